// Kernel-sum kernels and launch templates, shared by ksum.cu (d <= 8) and
// ksum_hi.cu (d >= 9), which instantiate them for disjoint dimensions so the
// two translation units compile in parallel.
#pragma once
// Kernel sums out_k = sum_j phi(|y_k - x_j|) a_j over the data points (Sec.
// 6.2: the product C gamma of the trend step, and c(x0)^T gamma of the
// prediction, eq. Spatial), optionally plus the trend k(y_k)^T beta.
//
// FP64 path: one thread per target; the data points and weights stream through
// shared memory in tiles of 128; FP64 throughout.
// Mixed path: four targets per thread; points as FP32 offsets from the data
// box centre (absolute error of a kernel value ~1e-7); kernel values in FP32,
// the weights split into two FP32 numbers, the sum over one tile of 256 points
// a cascaded FP32 sum (Sum2), the running sum over tiles in FP64.
// Distances are formed from coordinate differences (no |x|^2 + |y|^2 - 2 x.y
// cancellation).
//
// Source split: a grid of (target blocks) x (source chunks).  When there are
// too few target blocks to fill the GPU, each CTA sums one chunk of the data
// points and writes its partial sums to a work array; ksum_reduce_kernel adds
// the chunks in order (FP64) and the trend.  With one chunk the kernels write
// the result directly.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "ff.cuh"
#include "internal.h"
#include "matern.cuh"

namespace mlb {


struct TrendArgs {
    const double* beta;   // nullptr: no trend
    const int* alpha;     // p x d exponents
    int p;
    double lo[kMaxDim], hi[kMaxDim];
};

template <int D>
__device__ __forceinline__ void add_trend(double& acc, const double* y, const TrendArgs& tr) {
    double u[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double span = tr.hi[c] - tr.lo[c];
        u[c] = span > 0.0 ? 2.0 * (y[c] - tr.lo[c]) / span - 1.0 : 0.0;
    }
    for (int m = 0; m < tr.p; ++m) {
        double v = 1.0;
#pragma unroll
        for (int c = 0; c < D; ++c)
            for (int e = 0; e < tr.alpha[m * D + c]; ++e) v *= u[c];
        acc += tr.beta[m] * v;
    }
}

template <int D, bool DERIV>
__global__ void __launch_bounds__(128) ksum_f64_kernel(const double* __restrict__ tg, int64_t M,
                                                       const double* __restrict__ xs,
                                                       const double* __restrict__ a, int64_t N, KernelFn K,
                                                       KGeo geo, double* __restrict__ out, TrendArgs tr,
                                                       int64_t jchunk, double* __restrict__ part) {
    __shared__ double sx[128 * D];
    __shared__ double sa[128];
    const int64_t k = blockIdx.x * 128LL + threadIdx.x;
    double y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = k < M ? tg[k * D + c] * geo.sc[c] : 0.0;
    double acc = 0.0;
    const int64_t jb = blockIdx.y * jchunk, je = min(N, jb + jchunk);
    for (int64_t j0 = jb; j0 < je; j0 += 128) {
        const int nj = (int)(je - j0 < 128 ? je - j0 : 128);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nj * D; idx += 128) sx[idx] = xs[j0 * D + idx] * geo.sc[idx % D];
        if (threadIdx.x < nj) sa[threadIdx.x] = a[j0 + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            double r2 = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double df = y[c] - sx[j * D + c];
                r2 += df * df;
            }
            const double r = sqrt(r2);
            acc += kern_f64<DERIV>(r, K) * sa[j];
        }
    }
    if (k >= M) return;
    if (part) {
        part[blockIdx.y * M + k] = acc;
        return;
    }
    if (tr.beta) {
        // the trend is a polynomial in the caller's coordinates, not in the
        // scaled ones of an anisotropic distance
        double yy[D];
#pragma unroll
        for (int c = 0; c < D; ++c) yy[c] = tg[k * D + c];
        add_trend<D>(acc, yy, tr);
    }
    out[k] = acc;
}

// Mixed: FP32 kernel values, FP32 sum per tile of 256 points, FP64 across tiles.
// GEN = false: the half-integer Matern closed forms only (the hot loop of the
// matrix-free product carries no code for the other covariance kinds).
template <int D, int TPT, bool DERIV, int BS, bool GEN>
__global__ void __launch_bounds__(BS) ksum_f32_kernel(const double* __restrict__ tg, int64_t M,
                                                       const float* __restrict__ xs32,
                                                       const double* __restrict__ src64,
                                                       const double* __restrict__ a, int64_t N, KernelFn K,
                                                       KGeo ctr, double* __restrict__ out,
                                                       TrendArgs tr, int64_t jchunk, double* __restrict__ part) {
    constexpr int TS = 256;
    __shared__ float sx[TS * D];
    __shared__ float sa[TS];      // weights split as a = a_hi + a_lo
    __shared__ float sl[TS];
    const int64_t k0 = (blockIdx.x * (int64_t)BS + threadIdx.x) * TPT;
    float y[TPT][D];
#pragma unroll
    for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c)
            y[t][c] = k0 + t < M ? (float)((tg[(k0 + t) * D + c] - ctr.c[c]) * ctr.sc[c]) : 0.0f;
    double acc[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) acc[t] = 0.0;
    const int64_t jb = blockIdx.y * jchunk, je = min(N, jb + jchunk);
    for (int64_t j0 = jb; j0 < je; j0 += TS) {
        const int nj = (int)(je - j0 < TS ? je - j0 : TS);
        __syncthreads();
        if (xs32) {
            for (int idx = threadIdx.x; idx < nj * D; idx += BS) sx[idx] = xs32[j0 * D + idx];
        } else {
            for (int idx = threadIdx.x; idx < nj * D; idx += BS)
                sx[idx] = (float)((src64[j0 * D + idx] - ctr.c[idx % D]) * ctr.sc[idx % D]);
        }
        for (int idx = threadIdx.x; idx < nj; idx += BS) {
            const double w = a[j0 + idx];
            const float wh = (float)w;
            sa[idx] = wh;
            sl[idx] = (float)(w - (double)wh);
        }
        __syncthreads();
        float part[TPT], comp[TPT], low[TPT];
#pragma unroll
        for (int t = 0; t < TPT; ++t) part[t] = comp[t] = low[t] = 0.0f;
        for (int j = 0; j < nj; ++j) {
            float xj[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xj[c] = sx[j * D + c];
            const float aj = sa[j], alj = sl[j];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float r2 = 0.0f;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float df = y[t][c] - xj[c];
                    r2 = fmaf(df, df, r2);
                }
                const float r = sqrtf(r2);
                const float kv = GEN ? kern_f32<DERIV>(r, K)
                                     : (DERIV ? dmatern_dlogrho_f32(r, K.kind, K.scale32) : matern_f32(r, K.kind, K.scale32));
                sum2_add(part[t], comp[t], __fmul_rn(kv, aj));
                low[t] = fmaf(kv, alj, low[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t) acc[t] += (double)part[t] + ((double)low[t] + (double)comp[t]);
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t k = k0 + t;
        if (k >= M) continue;
        if (part) {
            part[blockIdx.y * M + k] = acc[t];
            continue;
        }
        double v = acc[t];
        if (tr.beta) {
            double yy[D];
#pragma unroll
            for (int c = 0; c < D; ++c) yy[c] = tg[k * D + c];
            add_trend<D>(v, yy, tr);
        }
        out[k] = v;
    }
}

// Mixed path, one-shot sums (trend step, prediction, gradient): kernel values
// in double-float (ff.cuh) from double-float coordinates, weights split into
// two FP32 numbers, the leading products in a cascaded sum (Sum2) over a tile
// of 128 points with their rounding errors (TwoProduct) and the cross terms in
// a plain FP32 sum, the running sum over tiles in FP64.  Two targets per thread.
template <int D, int TPT, bool DERIV>
__global__ void __launch_bounds__(128) ksum_ff_kernel(const double* __restrict__ tg, int64_t M,
                                                      const float* __restrict__ xh32,
                                                      const float* __restrict__ xl32,
                                                      const double* __restrict__ src64,
                                                      const double* __restrict__ a, int64_t N, KernelFn K,
                                                      KGeo ctr, double* __restrict__ out,
                                                      TrendArgs tr, int64_t jchunk, double* __restrict__ part) {
    constexpr int TS = 128;
    __shared__ float sxh[TS * D], sxl[TS * D];
    __shared__ float sah[TS], sal[TS];
    __shared__ float2 tab[64];
    ff_fill_exp2_table(tab);
    const ff sc = ff_from_double(K.scale);
    const int64_t k0 = (blockIdx.x * 128LL + threadIdx.x) * TPT;
    ff y[TPT][D];
#pragma unroll
    for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int c = 0; c < D; ++c)
            y[t][c] = ff_from_double(k0 + t < M ? (tg[(k0 + t) * D + c] - ctr.c[c]) * ctr.sc[c] : 0.0);
    double acc[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) acc[t] = 0.0;
    const int64_t jb = blockIdx.y * jchunk, je = min(N, jb + jchunk);
    for (int64_t j0 = jb; j0 < je; j0 += TS) {
        const int nj = (int)(je - j0 < TS ? je - j0 : TS);
        __syncthreads();
        if (xh32) {
            for (int idx = threadIdx.x; idx < nj * D; idx += 128) {
                sxh[idx] = xh32[j0 * D + idx];
                sxl[idx] = xl32[j0 * D + idx];
            }
        } else {
            for (int idx = threadIdx.x; idx < nj * D; idx += 128) {
                const ff v = ff_from_double((src64[j0 * D + idx] - ctr.c[idx % D]) * ctr.sc[idx % D]);
                sxh[idx] = v.h;
                sxl[idx] = v.l;
            }
        }
        for (int idx = threadIdx.x; idx < nj; idx += 128) {
            const ff w = ff_from_double(a[j0 + idx]);
            sah[idx] = w.h;
            sal[idx] = w.l;
        }
        __syncthreads();
        float part[TPT], comp[TPT], low[TPT];
#pragma unroll
        for (int t = 0; t < TPT; ++t) part[t] = comp[t] = low[t] = 0.0f;
        for (int j = 0; j < nj; ++j) {
            const float ah = sah[j], al = sal[j];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                ff r2 = {0.0f, 0.0f};
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    ff df = ff_two_sum(y[t][c].h, -sxh[j * D + c]);
                    df = ff_add(df, {__fsub_rn(y[t][c].l, sxl[j * D + c]), 0.0f});
                    r2 = ff_add(r2, ff_mul(df, df));
                }
                const ff r = ff_sqrt(r2);
                const ff kv = ff_kern<DERIV>(r, K, sc, tab);
                const float pr = __fmul_rn(kv.h, ah);
                sum2_add(part[t], comp[t], pr);
                low[t] = fmaf(kv.h, al, fmaf(kv.l, ah, __fadd_rn(low[t], fmaf(kv.h, ah, -pr))));
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t) acc[t] += (double)part[t] + ((double)low[t] + (double)comp[t]);
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t kk = k0 + t;
        if (kk >= M) continue;
        if (part) {
            part[blockIdx.y * M + kk] = acc[t];
            continue;
        }
        double v = acc[t];
        if (tr.beta) {
            double yy[D];
#pragma unroll
            for (int c = 0; c < D; ++c) yy[c] = tg[kk * D + c];
            add_trend<D>(v, yy, tr);
        }
        out[kk] = v;
    }
}

// out_k = sum over chunks of part[chunk][k] (in chunk order) + trend
template <int D>
__global__ void __launch_bounds__(256) ksum_reduce_kernel(const double* __restrict__ part, int splits, int64_t M,
                                                          const double* __restrict__ tg, double* __restrict__ out,
                                                          TrendArgs tr) {
    const int64_t k = blockIdx.x * 256LL + threadIdx.x;
    if (k >= M) return;
    double v = 0.0;
    for (int c = 0; c < splits; ++c) v += part[c * M + k];
    if (tr.beta) {
        double yy[D];
#pragma unroll
        for (int c = 0; c < D; ++c) yy[c] = tg[k * D + c];
        add_trend<D>(v, yy, tr);
    }
    out[k] = v;
}

// Source chunking for a grid of ctasM target blocks: about eight CTAs per SM in
// all, every chunk at least four tiles of TS points, the partial sums within
// the context's work array.  Returns the chunk length (a multiple of TS) and
// the number of chunks; one chunk means no split.
struct KsumSplit {
    int64_t chunk;
    int splits;
};

inline KsumSplit ksum_split(const mlb_ctx* ctx, int64_t ctasM, int64_t M, int64_t Ns, int TS) {
    int64_t want = (8LL * ctx->nsm + ctasM - 1) / std::max<int64_t>(ctasM, 1);
    want = std::min<int64_t>(want, Ns / (4LL * TS));
    want = std::min<int64_t>(want, ctx->ksum_part_cap / std::max<int64_t>(M, 1));
    want = std::min<int64_t>(want, 1024);
    if (want <= 1 || !ctx->ksum_part) return {std::max<int64_t>(Ns, 1), 1};
    int64_t chunk = (Ns + want - 1) / want;
    chunk = (chunk + TS - 1) / TS * TS;
    return {chunk, (int)((Ns + chunk - 1) / chunk)};
}

template <int D>
static void launch_reduce(mlb_ctx* ctx, const KsumSplit& sp, const double* tg, int64_t M, double* out,
                          const TrendArgs& tr) {
    if (sp.splits <= 1) return;
    ctx->launches += 1;     // the kernel sum's own launch is counted by its caller
    ksum_reduce_kernel<D><<<(unsigned)((M + 255) / 256), 256, 0, ctx->stream>>>(ctx->ksum_part, sp.splits, M, tg,
                                                                              out, tr);
}

// Launch shapes of the FP32 kernel sum (targets per thread x block size); the
// autotuner below picks one per device and dimension.  Every dimension has the
// default (4 targets, 128 threads); the common ones have all six.
constexpr int kKsumVariants = 6;
constexpr int kKsumVariantTC = kKsumFormTC;     // the tensor-core form (ksum_tc.cu), self sums only
static_assert(kKsumVariantTC == kKsumVariants, "the tensor-core form follows the launch shapes");
constexpr int kVarTpt[kKsumVariants] = {2, 4, 8, 2, 4, 8};
constexpr int kVarBs[kKsumVariants] = {128, 128, 128, 256, 256, 256};

constexpr bool tuned_dim(int D) { return D == 2 || D == 3 || D == 4 || D == 5 || D == 6 || D == 8 || D == 10; }

template <int D, bool DERIV, int TPT, int BS, bool GEN = false>
static void launch_f32_shape(mlb_ctx* ctx, const double* tg, int64_t M, const float* xs32, const double* src,
                             const double* a, int64_t Ns, const KernelFn& K, const KGeo& ctr, double* out,
                             const TrendArgs& tr) {
    const int64_t ctasM = (M + (int64_t)BS * TPT - 1) / ((int64_t)BS * TPT);
    const KsumSplit sp = ksum_split(ctx, ctasM, M, Ns, 256);
    const dim3 grid((unsigned)ctasM, (unsigned)sp.splits);
    ksum_f32_kernel<D, TPT, DERIV, BS, GEN><<<grid, BS, 0, ctx->stream>>>(tg, M, xs32, src, a, Ns, K, ctr, out,
                                                                     tr, sp.chunk,
                                                                     sp.splits > 1 ? ctx->ksum_part : nullptr);
    launch_reduce<D>(ctx, sp, tg, M, out, tr);
}

template <int D, bool DERIV>
static void launch_f32_variant(int v, mlb_ctx* ctx, const double* tg, int64_t M, const float* xs32,
                               const double* src, const double* a, int64_t Ns, const KernelFn& K,
                               const KGeo& ctr, double* out, const TrendArgs& tr) {
    if (K.kind > KIND_NU_5HALF) {
        launch_f32_shape<D, DERIV, 4, 128, true>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr);
        return;
    }
    if constexpr (tuned_dim(D) && !DERIV) {
        switch (v) {
            case 0: launch_f32_shape<D, DERIV, 2, 128>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr); return;
            case 2: launch_f32_shape<D, DERIV, 8, 128>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr); return;
            case 3: launch_f32_shape<D, DERIV, 2, 256>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr); return;
            case 4: launch_f32_shape<D, DERIV, 4, 256>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr); return;
            case 5: launch_f32_shape<D, DERIV, 8, 256>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr); return;
            default: break;
        }
    }
    launch_f32_shape<D, DERIV, 4, 128>(ctx, tg, M, xs32, src, a, Ns, K, ctr, out, tr);
}

template <int D, bool DERIV>
static void launch_ksum(mlb_ctx* ctx, const double* tg, int64_t M, const double* src, int64_t Ns,
                        const double* a, double* out, TrendArgs tr, bool accurate) {
    const KernelFn& K = ctx->kfn;
    const KGeo& geo = ctx->kgeo;
    if (ctx->opts.precision == MLB_MIXED && accurate) {
        constexpr int TPT = 2;
        const int64_t ctasM = (M + 128 * TPT - 1) / (128 * TPT);
        const KsumSplit sp = ksum_split(ctx, ctasM, M, Ns, 128);
        ksum_ff_kernel<D, TPT, DERIV><<<dim3((unsigned)ctasM, (unsigned)sp.splits), 128, 0, ctx->stream>>>(
            tg, M, src ? nullptr : ctx->kxs32, src ? nullptr : ctx->kxs32lo, src, a, Ns, K, geo, out, tr,
            sp.chunk, sp.splits > 1 ? ctx->ksum_part : nullptr);
        launch_reduce<D>(ctx, sp, tg, M, out, tr);
        return;
    }
    if (ctx->opts.precision == MLB_MIXED) {
        launch_f32_variant<D, DERIV>(DERIV ? 1 : ctx->ksum_variant, ctx, tg, M, src ? nullptr : ctx->kxs32, src,
                                     a, Ns, K, geo, out, tr);
        return;
    }
    const int64_t ctasM = (M + 127) / 128;
    const KsumSplit sp = ksum_split(ctx, ctasM, M, Ns, 128);
    ksum_f64_kernel<D, DERIV><<<dim3((unsigned)ctasM, (unsigned)sp.splits), 128, 0, ctx->stream>>>(
        tg, M, src ? src : ctx->xs, a, Ns, K, geo, out, tr, sp.chunk, sp.splits > 1 ? ctx->ksum_part : nullptr);
    launch_reduce<D>(ctx, sp, tg, M, out, tr);
}


}  // namespace mlb
