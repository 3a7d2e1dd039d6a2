// Diagonally preconditioned CG on C~_W g = Z_W (Sec. 5.2 remark on P_W,
// Sec. 6.2) and the trend step beta = (X^T X)^{-1} X^T (Z - C gamma)
// (eq. Spatial:eqn3).
//
// Vectors, inner products and updates are FP64.  The matrix-vector product
// streams the row panels of C~_W (HBM bound in FP32, FP64-pipe bound in FP64).
// Inner products are deterministic: every CTA writes its partial sums and the
// CTA that finishes last (a ticket count, no waiting) adds them in a fixed
// order, so one iteration is two or three launches: the product (whose last
// CTA forms alpha), the vector update (whose last CTA forms beta and the
// stopping test, and p for short vectors) and, for long vectors, the p
// update.  The scalars of the iteration live on the device; the host only
// reads the "done" flag between chunks of iterations, which are replayed as a
// captured CUDA graph.
// Stopping test: ||r_k||_2 <= rtol ||Z_W||_2 on the unpreconditioned
// residual r_k = Z_W - C~_W g_k (remark closing Sec. 6.2).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "matern.cuh"
#include "pcg_device.cuh"

namespace mlb {

constexpr int64_t kFusePMax = 16384;   // longest vector whose p update the last CTA does

// The symmetric FP32 product reads its vector as FP32 high and low parts
// (SymPanels::xh, xl); the kernels that write the PCG direction p also write
// those parts, so the product needs no conversion launch of its own.
__device__ __forceinline__ void store_split(float* xh, float* xl, int64_t k, double v) {
    if (!xh) return;
    const float h = (float)v;
    xh[k] = h;
    xl[k] = (float)(v - (double)h);
}

// the split buffers of the context's product, or nullptr when it reads none
static float* split_h(const mlb_ctx* ctx) { return (ctx->sym.vals && !ctx->opts.matrix_free) ? ctx->sym.xh : nullptr; }
static float* split_l(const mlb_ctx* ctx) { return (ctx->sym.vals && !ctx->opts.matrix_free) ? ctx->sym.xl : nullptr; }

// y = A x over the row panels, one CTA per panel (heaviest panels first).
// For every chunk of 256 columns the CTA stages the column indices' x values
// once in shared memory; each warp then streams its rows' values and
// multiplies against the staged chunk.  Only the values come from HBM.  To
// keep enough bytes in flight every lane issues the loads of four rows times
// four 16-byte segments before it consumes any of them (panels are padded to
// a width that is a multiple of 4, so every row starts 16-byte aligned).
// FP64 throughout: on GB300 the FP64 pipe, not HBM, bounds this product.
// Optionally part[block] = sum over the panel's rows of x_r y_r.
__global__ void __launch_bounds__(256) spmv_panel_f64_kernel(Panels pan, const double* __restrict__ vals,
                                                             const int* __restrict__ kcell,
                                                             const int64_t* __restrict__ wOff, int ncell,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             double* __restrict__ part, PcgState* st) {
    if (st && st->done) return;
    constexpr int CH = 256;
    __shared__ double xs[CH];     // the chunk's x values
    __shared__ double red[8];
    const int g = ncell - 1 - blockIdx.x;
    const int kc = kcell[g];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double dotp = 0.0;
    if (kc > 0) {
        const int n = pan.ncols[g];
        const int* ci = pan.colidx + pan.colOff[g];
        const double* v0 = vals + pan.valOff[g];
        const int64_t r0 = wOff[g];
        const int nrg = (kc + 31) / 32;          // groups of 4 rows per warp actually used
        // one DFMA per entry (the FP64 pipe bounds this kernel on GB300): each
        // lane chains its 8 products of a chunk, one add per chunk into the row
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
        for (int c0 = 0; c0 < n; c0 += CH) {
            const int m = min(CH, n - c0);
            __syncthreads();
            if (threadIdx.x < m) xs[threadIdx.x] = x[ci[c0 + threadIdx.x]];
            __syncthreads();
            if (m == CH) {
#pragma unroll
                for (int qb = 0; qb < 2; ++qb) {
                    if (qb >= nrg) break;
                    double2 v[4][4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = warp + 8 * (4 * qb + q);
                        const double* row = v0 + (int64_t)min(r, kc - 1) * n + c0 + 2 * lane;
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[q][u] = *reinterpret_cast<const double2*>(row + 64 * u);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = warp + 8 * (4 * qb + q);
                        double a = 0.0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = 2 * lane + 64 * u;
                            a = fma(v[q][u].x, xs[j], a);
                            a = fma(v[q][u].y, xs[j + 1], a);
                        }
                        if (r < kc) acc[4 * qb + q] += a;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = warp + 8 * q;
                    if (r < kc) {
                        const double* row = v0 + (int64_t)r * n + c0;
                        double a = 0.0;
                        for (int j = 2 * lane; j < m; j += 64) {
                            const double2 vv = *reinterpret_cast<const double2*>(row + j);
                            a = fma(vv.x, xs[j], a);
                            a = fma(vv.y, xs[j + 1], a);
                        }
                        acc[q] += a;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = warp + 8 * q;
            double a = acc[q];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0 && r < kc) {
                y[r0 + r] = a;
                dotp += x[r0 + r] * a;
            }
        }
    }
    if (part) {
        if (lane == 0) red[warp] = dotp;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s2 = 0.0;
            for (int i = 0; i < 8; ++i) s2 += red[i];
            part[blockIdx.x] = s2;
        }
        // inside the PCG the last CTA also forms alpha
        if (st && draw_last_ticket(st)) pcg_alpha_finish(part, gridDim.x, st);
    }
}

// FP32 panels: one CTA per work item of at most kItemRows rows and kSegCols
// columns of a panel (the heaviest items first, so that the uneven panels fill
// the SMs evenly and the last wave is short); the item writes its rows'
// partial products to its column segment's slice of ypart.  Each
// warp owns kItemRows / 8 rows and loads, per 256-column chunk, two 16-byte
// vectors of each of them before using any (128 bytes per lane in flight at
// 32-row items).  x is staged
// per chunk as FP32 high and low parts in a double buffer: the gather of the
// next chunk's x (column list -> x, an L2 round trip) is issued before the
// current chunk is multiplied and stored after it, so one barrier per chunk
// remains and the gather hides behind the value stream.  Products in FP32,
// each row's chunk sums in a cascaded FP32 sum (Sum2), the reduction in FP64.
// 64 registers, so four CTAs (32 warps) stay resident per SM.
__global__ void __launch_bounds__(256, 4) spmv_panel_f32_kernel(Panels pan, const float* __restrict__ vals,
                                                             const int* __restrict__ kcell,
                                                             const int64_t* __restrict__ wOff,
                                                             const double* __restrict__ x, int64_t nwav,
                                                             double* __restrict__ part, PcgState* st) {
    if (st && st->done) return;
    constexpr int CH = 256;
    __shared__ __align__(16) float xh[2][CH];
    __shared__ __align__(16) float xl[2][CH];
    __shared__ double red[8];
    const int4 wk = pan.work[blockIdx.x];           // cell, first row, first column, segment
    const int g = wk.x;
    const int rows = min(kItemRows, kcell[g] - wk.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nn = pan.ncols[g];                  // row stride of the panel
    const int cb = wk.z;
    const int n = min((int)nn, cb + kSegCols);        // end of this item's columns
    const int* ci = pan.colidx + pan.colOff[g];
    double* __restrict__ y = pan.ypart + (int64_t)wk.w * nwav;
    const float* v0 = vals + pan.valOff[g] + (int64_t)wk.y * nn;
    const int64_t r0 = wOff[g] + wk.y;
    constexpr int QR = kItemRows / 8;                  // rows per warp
    const int nq = min(QR, (rows - warp + 7) / 8);     // rows of this warp: warp, warp + 8, ...
    float acc[QR], err[QR];
#pragma unroll
    for (int q = 0; q < QR; ++q) acc[q] = err[q] = 0.0f;
    if (threadIdx.x < min(CH, n - cb)) {
        const double xv = x[ci[cb + threadIdx.x]];
        const float h = (float)xv;
        xh[0][threadIdx.x] = h;
        xl[0][threadIdx.x] = (float)(xv - (double)h);
    }
    __syncthreads();
    int buf = 0;
    for (int c0 = cb; c0 < n; c0 += CH) {
        const int m = min(CH, n - c0);
        const int cn = c0 + CH + threadIdx.x;
        // one thread per row asks the L2 for the row's next chunk (a bulk
        // prefetch, no registers held), so HBM streams it while this chunk's
        // loads and products run.  Rows start 16-byte aligned and the chunk
        // length is a multiple of 4 values, as the bulk copy requires.
        const int pc = c0 + CH;
        if (threadIdx.x < rows && pc < n)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(v0 + (int64_t)threadIdx.x * nn + pc),
                         "r"((unsigned)(min(CH, n - pc) * 4))
                         : "memory");
        const double xn = cn < n ? x[ci[cn]] : 0.0;
        const float* sh = xh[buf];
        const float* sl = xl[buf];
        if (m == CH) {
            float4 v[QR][2];
#pragma unroll
            for (int q = 0; q < QR; ++q) {
                const int r = min(warp + 8 * q, rows - 1);
                const float* row = v0 + (int64_t)r * nn + c0 + 4 * lane;
#pragma unroll
                for (int u = 0; u < 2; ++u) v[q][u] = *reinterpret_cast<const float4*>(row + 128 * u);
            }
#pragma unroll
            for (int q = 0; q < QR; ++q) {
                if (q < nq) {
                    float a = 0.0f;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = 4 * lane + 128 * u;
                        const float4 h = *reinterpret_cast<const float4*>(sh + j);
                        const float4 l = *reinterpret_cast<const float4*>(sl + j);
                        a += v[q][u].x * h.x + v[q][u].y * h.y + v[q][u].z * h.z + v[q][u].w * h.w;
                        a += v[q][u].x * l.x + v[q][u].y * l.y + v[q][u].z * l.z + v[q][u].w * l.w;
                    }
                    sum2_add(acc[q], err[q], a);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < QR; ++q) {
                if (q < nq) {
                    const float* row = v0 + (int64_t)(warp + 8 * q) * nn + c0;
                    float a = 0.0f;
                    for (int j = 4 * lane; j < m; j += 128) {
                        const float4 vv = *reinterpret_cast<const float4*>(row + j);
                        a += vv.x * (sh[j] + sl[j]) + vv.y * (sh[j + 1] + sl[j + 1]) +
                             vv.z * (sh[j + 2] + sl[j + 2]) + vv.w * (sh[j + 3] + sl[j + 3]);
                    }
                    sum2_add(acc[q], err[q], a);
                }
            }
        }
        if (cn < n) {
            const float h = (float)xn;
            xh[buf ^ 1][threadIdx.x] = h;
            xl[buf ^ 1][threadIdx.x] = (float)(xn - (double)h);
        }
        __syncthreads();
        buf ^= 1;
    }
    double dotp = 0.0;
#pragma unroll
    for (int q = 0; q < QR; ++q) {
        double a = (double)acc[q] + (double)err[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const int r = warp + 8 * q;
        if (lane == 0 && q < nq) {
            y[r0 + r] = a;
            dotp += x[r0 + r] * a;
        }
    }
    if (part) {
        if (lane == 0) red[warp] = dotp;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s2 = 0.0;
            for (int i = 0; i < 8; ++i) s2 += red[i];
            part[blockIdx.x] = s2;
        }
        // inside the PCG the last CTA also forms alpha
        if (st && draw_last_ticket(st)) pcg_alpha_finish(part, gridDim.x, st);
    }
}

// x = 0, r = b, z = r / diag, p = z; partials of r.z and b.b
__global__ void pcg_init_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ diag,
                                double* x, double* r, double* z, double* p, double* part, float* xh, float* xl) {
    double rz = 0.0, bb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double zi = diag ? bi / diag[i] : bi;
        x[i] = 0.0;
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        store_split(xh, xl, i, zi);
        rz += bi * zi;
        bb += bi * bi;
    }
    const double s1 = block_reduce(rz);
    const double s2 = block_reduce(bb);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[kVecBlocks + blockIdx.x] = s2;
    }
}

// The scalar kernels reduce the per-block partial sums with one CTA (strided
// per-thread sums, then a fixed-order tree), so their results are
// deterministic and they do not serialise on one thread's loads.
__global__ void __launch_bounds__(256) pcg_init_scalars(const double* part, PcgState* st) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < kVecBlocks; i += blockDim.x) {
        a += part[i];
        b += part[kVecBlocks + i];
    }
    const double rz = block_reduce(a);
    const double bb = block_reduce(b);
    if (threadIdx.x) return;
    st->rz = rz;
    st->bb = bb;
    st->rr = bb;
    st->it = 0;
    st->ticket = 0;
    st->status = ST_OK;
    st->done = bb == 0.0 ? 1 : 0;
}

__global__ void __launch_bounds__(256) pcg_alpha_kernel(const double* part, int nparts, PcgState* st) {
    if (st->done) return;
    double a = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += part[i];
    const double pq = block_reduce(a);
    if (threadIdx.x) return;
    st->pq = pq;
    if (!(pq > 0.0)) {
        st->status = ST_BREAKDOWN;
        st->done = 1;
        return;
    }
    st->alpha = st->rz / pq;
}

// The last CTA of a vector update: beta, the stopping test and (fuse_p)
// p = z + beta p, which is cheaper than another launch for short vectors.
__device__ void pcg_update_finish(int64_t n, PcgState* st, const double* part, double tol2, int maxit, int fuse_p,
                                  double* __restrict__ p, const double* z, float* xh, float* xl) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(part + i);
        b += __ldcg(part + kVecBlocks + i);
    }
    const double rrs = block_reduce(a);
    const double rzs = block_reduce(b);
    __shared__ double beta_s;
    __shared__ int go_on;
    if (threadIdx.x == 0) {
        st->it += 1;
        st->rr = rrs;
        st->beta = rzs / st->rz;
        st->rz = rzs;
        go_on = 0;
        if (rrs <= tol2 * st->bb) {
            st->done = 1;
        } else if (st->it >= maxit) {
            st->status = ST_NOCONV;
            st->done = 1;
        } else {
            go_on = 1;
        }
        beta_s = st->beta;
    }
    __syncthreads();
    if (fuse_p && go_on)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double v = __ldcg(z + i) + beta_s * p[i];
            p[i] = v;
            store_split(xh, xl, i, v);
        }
}

// x += alpha p, r -= alpha q, z = P^{-1} r and the partials of r.r and r.z;
// the last CTA then finishes the iteration (pcg_update_finish).
// With ypart != nullptr, q_i is the in-order sum of the FP32 product's
// segment partials (nseg[rowCell[i]] of them); otherwise q is read.
__global__ void pcg_update_xr_kernel(int64_t n, PcgState* st, double* __restrict__ p,
                                     const double* __restrict__ q, const double* __restrict__ ypart,
                                     const int* __restrict__ rowCell, const int* __restrict__ nseg,
                                     const double* __restrict__ diag,
                                     double* x, double* r, double* z, double* part, double tol2, int maxit,
                                     int fuse_p, float* xh, float* xl) {
    if (st->done) return;
    const double alpha = st->alpha;
    double rr = 0.0, rz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double qi;
        if (ypart) {
            const int ns = nseg[rowCell[i]];
            qi = 0.0;
            for (int sg = 0; sg < ns; ++sg) qi += ypart[sg * n + i];
        } else {
            qi = q[i];
        }
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * qi;
        r[i] = ri;
        const double zi = diag ? ri / diag[i] : ri;
        z[i] = zi;
        rr += ri * ri;
        rz += ri * zi;
    }
    const double s1 = block_reduce(rr);
    const double s2 = block_reduce(rz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[kVecBlocks + blockIdx.x] = s2;
    }
    if (!draw_last_ticket(st)) return;
    pcg_update_finish(n, st, part, tol2, maxit, fuse_p, p, z, xh, xl);
}

// The same update after the symmetric packed product: q_i is the sum of up to
// (segments + blocks above) partials, too many for one thread to read in
// sequence.  A CTA takes 32 consecutive elements at a time (one row block, so
// the slot count is uniform); its eight warps each add every eighth slot
// (reads coalesced along the elements), and warp 0 adds the eight sums in
// order and updates the vectors.  The order is fixed, so q is deterministic.
__global__ void __launch_bounds__(256) pcg_update_sym_kernel(int64_t n, PcgState* st, double* __restrict__ p,
                                                          SymPanels S, const double* __restrict__ diag,
                                                          double* x, double* r, double* z, double* part,
                                                          double tol2, int maxit, int fuse_p, float* xh,
                                                          float* xl) {
    if (st->done) return;
    __shared__ double qs[8][32];
    const double alpha = st->alpha;
    const int j = threadIdx.x & 31, g = threadIdx.x >> 5;
    double rr = 0.0, rz = 0.0;
    for (int64_t c0 = (int64_t)blockIdx.x * 32; c0 < n; c0 += (int64_t)gridDim.x * 32) {
        const int64_t i = c0 + j;
        qs[g][j] = i < n ? sym_q_slots(S, n, i, 0, g, 8) : 0.0;
        __syncthreads();
        if (g == 0 && i < n) {
            double qi = qs[0][j];
#pragma unroll
            for (int k = 1; k < 8; ++k) qi += qs[k][j];
            x[i] += alpha * p[i];
            const double ri = r[i] - alpha * qi;
            r[i] = ri;
            const double zi = diag ? ri / diag[i] : ri;
            z[i] = zi;
            rr += ri * ri;
            rz += ri * zi;
        }
        __syncthreads();
    }
    const double s1 = block_reduce(rr);
    const double s2 = block_reduce(rz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[kVecBlocks + blockIdx.x] = s2;
    }
    if (!draw_last_ticket(st)) return;
    pcg_update_finish(n, st, part, tol2, maxit, fuse_p, p, z, xh, xl);
}

__global__ void pcg_update_p_kernel(int64_t n, PcgState* st, const double* __restrict__ z, double* p, float* xh,
                                    float* xl) {
    if (st->done) return;
    const double beta = st->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = z[i] + beta * p[i];
        p[i] = v;
        store_split(xh, xl, i, v);
    }
}

// resid = Z - C gamma - eta gamma, then partial sums of X^T resid
__global__ void trend_partial_kernel(int64_t N, int p, const double* __restrict__ X, const double* __restrict__ Z,
                                     const double* __restrict__ Cg, const double* __restrict__ g, double eta,
                                     int64_t chunk, double* part) {
    const int64_t r0 = blockIdx.x * chunk, r1 = min(N, r0 + chunk);
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) acc += X[r * p + j] * (Z[r] - Cg[r] - eta * g[r]);
        part[(int64_t)blockIdx.x * p + j] = acc;
    }
}

// beta = (L L^T)^{-1} sum(part)
__global__ void trend_solve_kernel(const double* part, int nb, int p, const double* L, double* beta) {
    if (threadIdx.x) return;
    double y[128];
    for (int j = 0; j < p; ++j) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(int64_t)b * p + j];
        for (int k = 0; k < j; ++k) s -= L[j * p + k] * y[k];
        y[j] = s / L[j * p + j];
    }
    for (int j = p - 1; j >= 0; --j) {
        double s = y[j];
        for (int k = j + 1; k < p; ++k) s -= L[k * p + j] * y[k];
        y[j] = s / L[j * p + j];
    }
    for (int j = 0; j < p; ++j) beta[j] = y[j];
}

// y_i = sum over the column segments of row i's panel of ypart[s][i], in order
__global__ void seg_reduce_kernel(int64_t n, const int* __restrict__ rowCell, const int* __restrict__ nseg,
                                  const double* __restrict__ ypart, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ns = nseg[rowCell[i]];
        double v = 0.0;
        for (int sg = 0; sg < ns; ++sg) v += ypart[sg * n + i];
        y[i] = v;
    }
}

// out = C~_W u.  The FP32 product leaves its segment partials in ypart; inside
// the PCG (sum_in_update) the vector update sums them, elsewhere a reduction
// writes out.
static void launch_spmv(mlb_ctx* ctx, const double* u, double* out, double* part, PcgState* st,
                        bool sum_in_update = false) {
    if (ctx->sym.vals) {
        // inside the PCG the vector updates have already split p
        sym_launch(ctx, u, 1, part, st, sum_in_update);
        if (!sum_in_update) sym_reduce(ctx, out);
    } else if (ctx->pan.vals32) {
        if (ctx->pan.nwork == 0) {    // no wavelet rows: an empty product, a zero dot
            if (part) cudaMemsetAsync(part, 0, sizeof(double), ctx->stream);
            return;
        }
        spmv_panel_f32_kernel<<<ctx->pan.nwork, 256, 0, ctx->stream>>>(ctx->pan, ctx->pan.vals32, ctx->cells.k,
                                                                      ctx->cells.wOff, u, ctx->nwav, part, st);
        if (!sum_in_update) {
            seg_reduce_kernel<<<kVecBlocks, 256, 0, ctx->stream>>>(ctx->nwav, ctx->pan.rowCell, ctx->pan.nseg,
                                                                   ctx->pan.ypart, out);
            ctx->launches += 1;
        }
    } else
        spmv_panel_f64_kernel<<<ctx->ncell, 256, 0, ctx->stream>>>(ctx->pan, ctx->pan.vals, ctx->cells.k,
                                                                      ctx->cells.wOff, ctx->ncell, u, out, part, st);
}

// y += eta x; part[block] = sum x_i y_i (when part != nullptr)
__global__ void axpy_dot_kernel(int64_t n, double eta, const double* __restrict__ x, double* __restrict__ y,
                                double* part, PcgState* st) {
    if (st && st->done) return;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = y[i] + eta * x[i];
        y[i] = v;
        acc += x[i] * v;
    }
    const double s1 = block_reduce(acc);
    if (part && threadIdx.x == 0) part[blockIdx.x] = s1;
}

// Three-step product of Sec. 6.2: out = W (K (W^T u)) + eta u, with the
// kernel sum K a over all data points (no matrix is stored).
static mlb_status three_step(mlb_ctx* ctx, const double* u, double* out, double* part, PcgState* st) {
    double* a = ctx->vec + 8 * ctx->N;
    double* b = ctx->vec + 9 * ctx->N;
    mlb_status s = apply_Wt_dev(ctx, u, a);
    if (s != MLB_OK) return s;
    // the kernel sum of every iteration: FP32 kernel values on the mixed path
    s = kernel_sum_general(ctx, nullptr, ctx->N, nullptr, ctx->N, a, b, false, false, false);
    if (s != MLB_OK) return s;
    s = apply_W_dev(ctx, b, out);
    if (s != MLB_OK) return s;
    axpy_dot_kernel<<<kVecBlocks, 256, 0, ctx->stream>>>(ctx->nwav, ctx->theta.nugget, u, out, part, st);
    MLB_CHECK_LAUNCH(ctx, "axpy_dot_kernel");
    return MLB_OK;
}

mlb_status cw_matvec_dev(mlb_ctx* ctx, const double* u, double* out) {
    if (ctx->opts.matrix_free) return three_step(ctx, u, out, nullptr, nullptr);
    launch_spmv(ctx, u, out, nullptr, nullptr);
    MLB_CHECK_LAUNCH(ctx, "spmv_panel kernel");
    return MLB_OK;
}

static mlb_status launch_iteration(mlb_ctx* ctx, double* x, double* r, double* z, double* p, double* q,
                                   double tol2) {
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->nwav;
    const double* diag = ctx->opts.precond ? ctx->diag : nullptr;
    double* part2 = ctx->partial + std::max(max_work_items(ctx->ncell, ctx->N), (size_t)kVecBlocks);
    if (ctx->opts.matrix_free) {
        // the kernel sum, the transforms and the axpy run every iteration; once
        // converged, the kernels that check the flag return at once
        mlb_status s = three_step(ctx, p, q, ctx->partial, ctx->pcg);
        if (s != MLB_OK) return s;
        pcg_alpha_kernel<<<1, 256, 0, st>>>(ctx->partial, kVecBlocks, ctx->pcg);
        ctx->launches += 1;
    } else if (!ctx->sym.vals && ctx->pan.vals32 && ctx->pan.nwork == 0) {
        // no wavelet rows: nothing to iterate on
        return MLB_OK;
    } else {
        // the product's last CTA forms alpha; the FP32 product's segment
        // partials are summed by the update below
        launch_spmv(ctx, p, q, ctx->partial, ctx->pcg, true);
        ctx->launches += 1;
    }
    const bool segs = !ctx->opts.matrix_free && !ctx->sym.vals && ctx->pan.vals32;
    // short vectors: the last CTA of the update also forms p; long ones get a launch
    const int fuse_p = n <= kFusePMax ? 1 : 0;
    if (!ctx->opts.matrix_free && ctx->sym.vals)
        pcg_update_sym_kernel<<<kVecBlocks, 256, 0, st>>>(n, ctx->pcg, p, ctx->sym, diag, x, r, z, part2, tol2,
                                                          ctx->opts.pcg_maxit, fuse_p, split_h(ctx), split_l(ctx));
    else
        pcg_update_xr_kernel<<<kVecBlocks, 256, 0, st>>>(n, ctx->pcg, p, q, segs ? ctx->pan.ypart : nullptr,
                                                         ctx->pan.rowCell, ctx->pan.nseg, diag, x, r, z, part2, tol2,
                                                         ctx->opts.pcg_maxit, fuse_p, split_h(ctx), split_l(ctx));
    ctx->launches += 1;
    if (!fuse_p) {
        pcg_update_p_kernel<<<kVecBlocks, 256, 0, st>>>(n, ctx->pcg, z, p, split_h(ctx), split_l(ctx));
        ctx->launches += 1;
    }
    return MLB_OK;
}

// PCG on C~_W x = b; b and x are nwav vectors on the device, b must not alias
// the work vectors (vec + nwav .. vec + 5 nwav).
mlb_status pcg_run(mlb_ctx* ctx, const double* b, double* x, mlb_info* info) {
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->nwav;
    double* r = ctx->vec + n;
    double* z = ctx->vec + 2 * n;
    double* p = ctx->vec + 3 * n;
    double* q = ctx->vec + 4 * n;
    const double* diag = ctx->opts.precond ? ctx->diag : nullptr;
    pcg_init_kernel<<<kVecBlocks, 256, 0, st>>>(n, b, diag, x, r, z, p, ctx->partial, split_h(ctx), split_l(ctx));
    pcg_init_scalars<<<1, 256, 0, st>>>(ctx->partial, ctx->pcg);
    MLB_CHECK_LAUNCH(ctx, "pcg_init");
    ctx->launches += 1;
    const double tol2 = ctx->opts.pcg_rtol * ctx->opts.pcg_rtol;
    // graph, its instance and the timing events are released on every return
    struct Owned {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ~Owned() {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } own;
    MLB_CUDA(ctx, cudaEventCreate(&own.e0));
    MLB_CUDA(ctx, cudaEventCreate(&own.e1));
    MLB_CUDA(ctx, cudaEventRecord(own.e0, st));
    // one chunk of iterations as a CUDA graph, replayed until done
    const int chunk = ctx->opts.matrix_free ? 2 : 8;
    const int64_t l0 = ctx->launches;
    MLB_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) {
        mlb_status ls = launch_iteration(ctx, x, r, z, p, q, tol2);
        if (ls != MLB_OK) {
            cudaStreamEndCapture(st, &own.graph);
            return ls;
        }
    }
    MLB_CUDA(ctx, cudaStreamEndCapture(st, &own.graph));
    MLB_CUDA(ctx, cudaGraphInstantiate(&own.exec, own.graph, 0));
    const int64_t perChunk = ctx->launches - l0;   // kernels in one replay (capture counted them once)
    ctx->launches = l0;
    PcgState hs{};
    for (;;) {
        MLB_CUDA(ctx, cudaGraphLaunch(own.exec, st));
        ctx->launches += perChunk;
        MLB_CUDA(ctx, cudaMemcpyAsync(&hs, ctx->pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        if (hs.done) break;
    }
    MLB_CUDA(ctx, cudaEventRecord(own.e1, st));
    MLB_CUDA(ctx, cudaEventSynchronize(own.e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, own.e0, own.e1);
    if (info) {
        info->iterations = hs.it;
        info->converged = hs.status == ST_OK && hs.done;
        info->rel_residual = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
        info->ms_pcg = ms;
    }
    if (hs.status == ST_BREAKDOWN) return fail(ctx, MLB_EBREAKDOWN, "PCG breakdown: p^T C~_W p <= 0");
    if (hs.status == ST_NOCONV) return fail(ctx, MLB_ENOCONV, "PCG did not reach pcg_rtol within pcg_maxit");
    if (hs.status == ST_TIMEOUT) return fail(ctx, MLB_ETIMEOUT, "a bounded wait of the matrix product gave up");
    return MLB_OK;
}

mlb_status solve_dev(mlb_ctx* ctx, const double* Z_kd, mlb_info* info) {
    cudaStream_t st = ctx->stream;
    double* b = ctx->vec;
    double* x = ctx->gW;
    mlb_status s = apply_W_dev(ctx, Z_kd, b);
    if (s != MLB_OK) return s;
    mlb_info& I = ctx->last_info;
    const mlb_status ps = pcg_run(ctx, b, x, &I);
    if (ps != MLB_OK && ps != MLB_ENOCONV && ps != MLB_EBREAKDOWN) return ps;
    const std::string pmsg = ctx->err;
    I.nnz = ctx->pan.nnz;
    I.nnz_unique = ctx->pan.nnzUnique;
    I.col_total = ctx->sym.vals ? 0 : ctx->pan.colTotal;
    I.symmetric = ctx->sym.vals ? 1 : 0;
    I.product_variant = ctx->sym.vals ? ctx->sym_variant : 0;
    I.product_values = ctx->opts.matrix_free ? 0 : (ctx->sym.vals ? ctx->sym.stored : ctx->pan.stored);
    I.blocks = ctx->pan.blocks;
    I.ms_assemble = ctx->ms_assemble;
    // gamma = W^T g, then beta
    cudaEvent_t b0, b1;
    cudaEventCreate(&b0);
    cudaEventCreate(&b1);
    cudaEventRecord(b0, st);
    s = apply_Wt_dev(ctx, x, ctx->gamma);
    if (s != MLB_OK) return s;
    s = trend_dev(ctx, Z_kd);
    if (s != MLB_OK) return s;
    cudaEventRecord(b1, st);
    cudaEventSynchronize(b1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b0, b1);
    cudaEventDestroy(b0);
    cudaEventDestroy(b1);
    I.ms_beta = ms;
    I.launches = ctx->launches;
    if (info) *info = I;
    if (ps != MLB_OK) ctx->err = pmsg;
    return ps;
}

mlb_status trend_dev(mlb_ctx* ctx, const double* Z_kd) {
    cudaStream_t st = ctx->stream;
    double* Cg = ctx->vec + 5 * ctx->nwav;     // N entries
    mlb_status s = kernel_sum_dev(ctx, nullptr, ctx->N, ctx->gamma, Cg, false);
    if (s != MLB_OK) return s;
    const int nb = 64;
    const int64_t chunk = (ctx->N + nb - 1) / nb;
    double* part = ctx->partial;
    trend_partial_kernel<<<nb, 128, 0, st>>>(ctx->N, ctx->p, ctx->X, Z_kd, Cg, ctx->gamma, ctx->theta.nugget,
                                             chunk, part);
    trend_solve_kernel<<<1, 32, 0, st>>>(part, nb, ctx->p, ctx->XtXf, ctx->beta);
    MLB_CHECK_LAUNCH(ctx, "trend");
    return MLB_OK;
}

// ---- several right-hand sides at once (kriging MSE) ---------------------------
//
// kRhs independent diagonally preconditioned CG recurrences on the same FP32
// C~_W, sharing one pass over the panels per iteration: every value loaded
// feeds kRhs products, so the HBM traffic of an iteration is that of one
// product.  Vectors are stored right-hand side after right-hand side (kRhs x n).
// Each recurrence has its own scalars and stopping test; one that has stopped
// is carried along unchanged until all have.

__device__ __forceinline__ bool all_done(const PcgState* st) {
    bool d = true;
#pragma unroll
    for (int r = 0; r < kRhs; ++r) d = d && st[r].done;
    return d;
}

__global__ void __launch_bounds__(256, 2) spmm_panel_f32_kernel(Panels pan, const float* __restrict__ vals,
                                                             const int* __restrict__ kcell,
                                                             const int64_t* __restrict__ wOff,
                                                             const double* __restrict__ x, int64_t nwav,
                                                             double* __restrict__ ypart, double* __restrict__ part,
                                                             PcgState* st) {
    if (all_done(st)) return;
    constexpr int CH = 256;
    constexpr int QR = kItemRows / 8;
    __shared__ __align__(16) float xh[2][kRhs][CH];
    __shared__ __align__(16) float xl[2][kRhs][CH];
    __shared__ double red[8][kRhs];
    const int4 wk = pan.work[blockIdx.x];
    const int g = wk.x;
    const int rows = min(kItemRows, kcell[g] - wk.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nn = pan.ncols[g];
    const int cb = wk.z;
    const int n = min((int)nn, cb + kSegCols);
    const int* ci = pan.colidx + pan.colOff[g];
    const float* v0 = vals + pan.valOff[g] + (int64_t)wk.y * nn;
    const int64_t r0 = wOff[g] + wk.y;
    const int nq = min(QR, (rows - warp + 7) / 8);
    float acc[QR][kRhs], err[QR][kRhs];
#pragma unroll
    for (int q = 0; q < QR; ++q)
#pragma unroll
        for (int r = 0; r < kRhs; ++r) acc[q][r] = err[q][r] = 0.0f;
    if (threadIdx.x < min(CH, n - cb)) {
        const int c = ci[cb + threadIdx.x];
#pragma unroll
        for (int r = 0; r < kRhs; ++r) {
            const double xv = x[r * nwav + c];
            const float h = (float)xv;
            xh[0][r][threadIdx.x] = h;
            xl[0][r][threadIdx.x] = (float)(xv - (double)h);
        }
    }
    __syncthreads();
    int buf = 0;
    for (int c0 = cb; c0 < n; c0 += CH) {
        const int m = min(CH, n - c0);
        const int cn = c0 + CH + threadIdx.x;
        const int pc = c0 + CH;
        if (threadIdx.x < rows && pc < n)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(v0 + (int64_t)threadIdx.x * nn + pc),
                         "r"((unsigned)(min(CH, n - pc) * 4))
                         : "memory");
        double xn[kRhs];
        if (cn < n) {
            const int c = ci[cn];
#pragma unroll
            for (int r = 0; r < kRhs; ++r) xn[r] = x[r * nwav + c];
        }
        if (m == CH) {
            float4 v[QR][2];
#pragma unroll
            for (int q = 0; q < QR; ++q) {
                const int rr = min(warp + 8 * q, rows - 1);
                const float* row = v0 + (int64_t)rr * nn + c0 + 4 * lane;
#pragma unroll
                for (int u = 0; u < 2; ++u) v[q][u] = *reinterpret_cast<const float4*>(row + 128 * u);
            }
#pragma unroll
            for (int r = 0; r < kRhs; ++r) {
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    if (q < nq) {
                        float a = 0.0f;
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int j = 4 * lane + 128 * u;
                            const float4 h = *reinterpret_cast<const float4*>(&xh[buf][r][j]);
                            const float4 l = *reinterpret_cast<const float4*>(&xl[buf][r][j]);
                            a += v[q][u].x * h.x + v[q][u].y * h.y + v[q][u].z * h.z + v[q][u].w * h.w;
                            a += v[q][u].x * l.x + v[q][u].y * l.y + v[q][u].z * l.z + v[q][u].w * l.w;
                        }
                        sum2_add(acc[q][r], err[q][r], a);
                    }
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < QR; ++q) {
                if (q < nq) {
                    const float* row = v0 + (int64_t)(warp + 8 * q) * nn + c0;
#pragma unroll
                    for (int r = 0; r < kRhs; ++r) {
                        const float* sh = xh[buf][r];
                        const float* sl = xl[buf][r];
                        float a = 0.0f;
                        for (int j = 4 * lane; j < m; j += 128) {
                            const float4 vv = *reinterpret_cast<const float4*>(row + j);
                            a += vv.x * (sh[j] + sl[j]) + vv.y * (sh[j + 1] + sl[j + 1]) +
                                 vv.z * (sh[j + 2] + sl[j + 2]) + vv.w * (sh[j + 3] + sl[j + 3]);
                        }
                        sum2_add(acc[q][r], err[q][r], a);
                    }
                }
            }
        }
        if (cn < n) {
#pragma unroll
            for (int r = 0; r < kRhs; ++r) {
                const float h = (float)xn[r];
                xh[buf ^ 1][r][threadIdx.x] = h;
                xl[buf ^ 1][r][threadIdx.x] = (float)(xn[r] - (double)h);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    double dotp[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) dotp[r] = 0.0;
#pragma unroll
    for (int q = 0; q < QR; ++q) {
        const int row = warp + 8 * q;
#pragma unroll
        for (int r = 0; r < kRhs; ++r) {
            double a = (double)acc[q][r] + (double)err[q][r];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0 && q < nq) {
                ypart[((int64_t)r * pan.nsegMax + wk.w) * nwav + r0 + row] = a;
                dotp[r] += x[r * nwav + r0 + row] * a;
            }
        }
    }
    if (lane == 0)
#pragma unroll
        for (int r = 0; r < kRhs; ++r) red[warp][r] = dotp[r];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < kRhs; ++r) {
            double s2 = 0.0;
            for (int i = 0; i < 8; ++i) s2 += red[i][r];
            part[(int64_t)r * gridDim.x + blockIdx.x] = s2;
        }
    if (draw_last_ticket(st))
        for (int r = 0; r < kRhs; ++r)
            if (!st[r].done) pcg_alpha_finish(part + (int64_t)r * gridDim.x, gridDim.x, st + r);
}

// x_r += alpha_r p_r, r_r -= alpha_r q_r (q_r from the segment partials, or
// from the symmetric product's partials),
// z_r = P^{-1} r_r and the partials of r_r.r_r and r_r.z_r; the last CTA forms
// beta_r and the stopping test of every recurrence still running.
__global__ void pcg_update_multi_kernel(int64_t n, PcgState* st, const double* __restrict__ p,
                                        const double* __restrict__ ypart, int nsegMax,
                                        const int* __restrict__ rowCell, const int* __restrict__ nseg,
                                        SymPanels sym, const double* __restrict__ diag, double* x, double* rv,
                                        double* z, double* part, double tol2, int maxit) {
    if (all_done(st)) return;
    bool act[kRhs];
    double alpha[kRhs], rr[kRhs], rz[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) {
        act[r] = !st[r].done;
        alpha[r] = st[r].alpha;
        rr[r] = rz[r] = 0.0;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ns = sym.vals ? 0 : nseg[rowCell[i]];
        const double di = diag ? diag[i] : 1.0;
#pragma unroll
        for (int r = 0; r < kRhs; ++r) {
            if (!act[r]) continue;
            double qi = 0.0;
            if (sym.vals) qi = sym_q(sym, n, i, r);
            for (int sg = 0; sg < ns; ++sg) qi += ypart[((int64_t)r * nsegMax + sg) * n + i];
            const int64_t k = r * n + i;
            x[k] += alpha[r] * p[k];
            const double ri = rv[k] - alpha[r] * qi;
            rv[k] = ri;
            const double zi = diag ? ri / di : ri;
            z[k] = zi;
            rr[r] += ri * ri;
            rz[r] += ri * zi;
        }
    }
    for (int r = 0; r < kRhs; ++r) {
        const double s1 = block_reduce(rr[r]);
        const double s2 = block_reduce(rz[r]);
        if (threadIdx.x == 0) {
            part[(int64_t)(2 * r) * kVecBlocks + blockIdx.x] = s1;
            part[(int64_t)(2 * r + 1) * kVecBlocks + blockIdx.x] = s2;
        }
    }
    if (!draw_last_ticket(st)) return;
    for (int r = 0; r < kRhs; ++r) {
        if (!act[r]) continue;
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            a += __ldcg(part + (int64_t)(2 * r) * kVecBlocks + i);
            b += __ldcg(part + (int64_t)(2 * r + 1) * kVecBlocks + i);
        }
        const double rrs = block_reduce(a);
        const double rzs = block_reduce(b);
        if (threadIdx.x == 0) {
            PcgState& S = st[r];
            S.it += 1;
            S.rr = rrs;
            S.beta = rzs / S.rz;
            S.rz = rzs;
            if (rrs <= tol2 * S.bb) {
                S.done = 1;
            } else if (S.it >= maxit) {
                S.status = ST_NOCONV;
                S.done = 1;
            }
        }
    }
}

__global__ void pcg_update_p_multi_kernel(int64_t n, const PcgState* st, const double* __restrict__ z, double* p,
                                          float* xh, float* xl, int64_t xld) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int r = 0; r < kRhs; ++r)
            if (!st[r].done) {
                const double v = z[r * n + i] + st[r].beta * p[r * n + i];
                p[r * n + i] = v;
                store_split(xh, xl, r * xld + i, v);
            }
}

// x_r = 0, r_r = b_r, z_r = P^{-1} b_r, p_r = z_r; the scalars of every recurrence
__global__ void pcg_init_multi_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ diag,
                                      double* x, double* rv, double* z, double* p, double* part, float* xh, float* xl,
                                      int64_t xld) {
    double rz[kRhs], bb[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) rz[r] = bb[r] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int r = 0; r < kRhs; ++r) {
            const int64_t k = r * n + i;
            const double bi = b[k];
            const double zi = diag ? bi / diag[i] : bi;
            x[k] = 0.0;
            rv[k] = bi;
            z[k] = zi;
            p[k] = zi;
            store_split(xh, xl, r * xld + i, zi);
            rz[r] += bi * zi;
            bb[r] += bi * bi;
        }
    for (int r = 0; r < kRhs; ++r) {
        const double s1 = block_reduce(rz[r]);
        const double s2 = block_reduce(bb[r]);
        if (threadIdx.x == 0) {
            part[(int64_t)(2 * r) * kVecBlocks + blockIdx.x] = s1;
            part[(int64_t)(2 * r + 1) * kVecBlocks + blockIdx.x] = s2;
        }
    }
}

__global__ void __launch_bounds__(256) pcg_init_multi_scalars(const double* part, PcgState* st) {
    for (int r = 0; r < kRhs; ++r) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < kVecBlocks; i += blockDim.x) {
            a += part[(int64_t)(2 * r) * kVecBlocks + i];
            b += part[(int64_t)(2 * r + 1) * kVecBlocks + i];
        }
        const double rz = block_reduce(a);
        const double bb = block_reduce(b);
        if (threadIdx.x == 0) {
            PcgState& S = st[r];
            S.rz = rz;
            S.bb = bb;
            S.rr = bb;
            S.it = 0;
            S.ticket = 0;
            S.status = ST_OK;
            S.done = bb == 0.0 ? 1 : 0;
        }
    }
}

// work items of the FP32 product (symmetric storage or row panels)
static int product_items(const mlb_ctx* ctx) { return ctx->sym.vals ? ctx->sym.nwork : ctx->pan.nwork; }

size_t pcg_multi_work_doubles(const mlb_ctx* ctx) {
    const int64_t n = ctx->nwav;
    const int64_t nseg = ctx->sym.vals ? 0 : ctx->pan.nsegMax;   // the symmetric partials live in ctx->sym
    return (size_t)kRhs * (5 * n + nseg * n) + (size_t)kRhs * product_items(ctx) +
           (size_t)2 * kRhs * kVecBlocks + kRhs * (sizeof(PcgState) / sizeof(double) + 1);
}

// kRhs PCG solves C~_W x_r = b_r (b, x: kRhs x nwav, device) on the FP32
// panels of the mixed path; work: pcg_multi_work_doubles(ctx) doubles (device).
// iters (host, kRhs) receives each recurrence's iteration count.
mlb_status pcg_run_multi(mlb_ctx* ctx, const double* b, double* x, double* work, int* iters) {
    if (ctx->opts.matrix_free || !(ctx->sym.vals || (ctx->pan.vals32 && ctx->pan.nwork > 0)))
        return fail(ctx, MLB_EINVAL, "several right-hand sides need the assembled FP32 panels");
    if (ctx->sym.vals) {
        mlb_status rs = sym_reserve(ctx, kRhs);
        if (rs != MLB_OK) return rs;
    }
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->nwav;
    double* rv = work;
    double* z = rv + kRhs * n;
    double* p = z + kRhs * n;
    double* ypart = p + kRhs * n;
    double* part = ypart + (int64_t)kRhs * (ctx->sym.vals ? 0 : ctx->pan.nsegMax) * n;
    double* part2 = part + (int64_t)kRhs * product_items(ctx);
    PcgState* S = reinterpret_cast<PcgState*>(part2 + 2 * kRhs * kVecBlocks);
    const double* diag = ctx->opts.precond ? ctx->diag : nullptr;
    const double tol2 = ctx->opts.pcg_rtol * ctx->opts.pcg_rtol;
    pcg_init_multi_kernel<<<kVecBlocks, 256, 0, st>>>(n, b, diag, x, rv, z, p, part2, split_h(ctx), split_l(ctx),
                                                      ctx->sym.xld);
    pcg_init_multi_scalars<<<1, 256, 0, st>>>(part2, S);
    MLB_CHECK_LAUNCH(ctx, "pcg_init_multi");
    ctx->launches += 1;
    struct Owned {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ~Owned() {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        }
    } own;
    constexpr int chunk = 8;
    MLB_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) {
        if (ctx->sym.vals)
            sym_launch(ctx, p, kRhs, part, S, true);
        else
            spmm_panel_f32_kernel<<<ctx->pan.nwork, 256, 0, st>>>(ctx->pan, ctx->pan.vals32, ctx->cells.k,
                                                                 ctx->cells.wOff, p, n, ypart, part, S);
        pcg_update_multi_kernel<<<kVecBlocks, 256, 0, st>>>(n, S, p, ypart, ctx->pan.nsegMax, ctx->pan.rowCell,
                                                            ctx->pan.nseg, ctx->sym, diag, x, rv, z, part2, tol2,
                                                            ctx->opts.pcg_maxit);
        pcg_update_p_multi_kernel<<<kVecBlocks, 256, 0, st>>>(n, S, z, p, split_h(ctx), split_l(ctx), ctx->sym.xld);
    }
    MLB_CUDA(ctx, cudaStreamEndCapture(st, &own.graph));
    MLB_CUDA(ctx, cudaGraphInstantiate(&own.exec, own.graph, 0));
    PcgState hs[kRhs];
    for (;;) {
        MLB_CUDA(ctx, cudaGraphLaunch(own.exec, st));
        ctx->launches += 3 * chunk;
        MLB_CUDA(ctx, cudaMemcpyAsync(hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        bool done = true;
        for (int r = 0; r < kRhs; ++r) done = done && hs[r].done;
        if (done) break;
    }
    for (int r = 0; r < kRhs; ++r) {
        if (iters) iters[r] = hs[r].it;
        if (hs[r].status == ST_BREAKDOWN) return fail(ctx, MLB_EBREAKDOWN, "PCG breakdown: p^T C~_W p <= 0");
        if (hs[r].status == ST_NOCONV) return fail(ctx, MLB_ENOCONV, "PCG did not reach pcg_rtol within pcg_maxit");
        if (hs[r].status == ST_TIMEOUT)
            return fail(ctx, MLB_ETIMEOUT, "a bounded wait of the matrix product gave up");
    }
    return MLB_OK;
}

}  // namespace mlb
