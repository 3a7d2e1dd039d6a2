// Multilevel basis on the GPU (Sec. 3.1, construction steps 1-5).
//
// Level by level from the leaves, one CTA per cell: the cell's moment matrix
// M = X^T B (B = the leaf unit vectors, or the children's scaling vectors) is
// transposed into shared memory and split by a Householder QR, M^T = Q R.
// With M^T of full column rank a = min(p, s), the first a columns of Q span
// the row space of M (the scaling vectors) and the remaining s - a columns its
// null space (the wavelets, which satisfy X^T psi = 0, eq. hbconstruction:eqn1).
// The paper takes the right singular vectors of an SVD instead; both give an
// orthonormal basis of the same two subspaces, and everything downstream
// (predictions, W^T W, the truncated C~_W up to a block-diagonal rotation) is
// independent of that choice.  The moments of the new scaling vectors are the
// rows of R (X^T phi_j = R[j, :]^T), which is all the parent needs.
//
// The transforms W v and W^T u (Sec. 3.1, operator W; Sec. 6.2 steps (1), (3))
// run level by level with the per-cell factors: O(N n0 + cells p^2) work.
#include <cfloat>
#include <mutex>
#include <string>

#include "internal.h"

namespace mlb {

struct Box {
    double lo[kMaxDim];
    double hi[kMaxDim];
};

// u = 2 (x - lo) / (hi - lo) - 1 per axis (0 where hi == lo), X = u^alpha.
__global__ void design_kernel(const double* __restrict__ xs, int64_t N, int d, int p,
                              const int* __restrict__ alpha, Box box, double* __restrict__ X) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double u[kMaxDim];
    for (int k = 0; k < d; ++k) {
        const double span = box.hi[k] - box.lo[k];
        u[k] = span > 0.0 ? 2.0 * (xs[i * d + k] - box.lo[k]) / span - 1.0 : 0.0;
    }
    for (int j = 0; j < p; ++j) {
        double v = 1.0;
        for (int k = 0; k < d; ++k)
            for (int e = 0; e < alpha[j * d + k]; ++e) v *= u[k];
        X[i * p + j] = v;
    }
}

// Partial sums of X^T X over row chunks: part[b][j*p + c].
__global__ void xtx_partial_kernel(const double* __restrict__ X, int64_t N, int p, int64_t chunk,
                                   double* __restrict__ part) {
    const int64_t r0 = blockIdx.x * chunk;
    const int64_t r1 = min(N, r0 + chunk);
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
        const int j = idx / p, c = idx % p;
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) acc += X[r * p + j] * X[r * p + c];
        part[(int64_t)blockIdx.x * p * p + idx] = acc;
    }
}

// Sums the partials into A (p x p) and factors A = L L^T in place (lower).
__global__ void xtx_chol_kernel(const double* __restrict__ part, int nb, int p, double* A, int* flag) {
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * p * p + idx];
        A[idx] = acc;
    }
    __syncthreads();
    for (int j = 0; j < p; ++j) {
        if (threadIdx.x == 0) {
            double s = A[j * p + j];
            for (int k = 0; k < j; ++k) s -= A[j * p + k] * A[j * p + k];
            if (!(s > 0.0)) { atomicOr(flag, 2); s = 1.0; }
            A[j * p + j] = sqrt(s);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < p; i += blockDim.x) {
            double s = A[i * p + j];
            for (int k = 0; k < j; ++k) s -= A[i * p + k] * A[j * p + k];
            A[i * p + j] = s / A[j * p + j];
        }
        __syncthreads();
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// Householder QR of the s x p matrix M^T of one cell, Q written to V (s x s,
// row-major), the a x p factor R to the R pool.
__global__ void __launch_bounds__(128) qr_level_kernel(CellTables C, const double* __restrict__ X,
                                                       int p, int level, int leaf_level,
                                                       double* __restrict__ V, double* __restrict__ R,
                                                       int* flag) {
    extern __shared__ double sh[];
    __shared__ double red[32];
    __shared__ double bcast;
    const int g = (1 << level) - 1 + blockIdx.x;
    const int s = C.s[g], a = C.a[g];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* A = sh;
    double* tau = A + (int64_t)s * p;
    if (level == leaf_level) {
        const int64_t b = C.beg[g];
        for (int idx = tid; idx < s * p; idx += nt) A[idx] = X[b * p + idx];
    } else {
        const int gl = 2 * g + 1, gr = 2 * g + 2;
        const int al = C.a[gl], ar = C.a[gr];
        for (int idx = tid; idx < al * p; idx += nt) A[idx] = R[C.rOff[gl] + idx];
        for (int idx = tid; idx < ar * p; idx += nt) A[al * p + idx] = R[C.rOff[gr] + idx];
    }
    double part = 0.0;
    for (int idx = tid; idx < s * p; idx += nt) part += A[idx] * A[idx];
    const double normF = sqrt(block_sum(part, red));
    const int m = min(s, p);
    for (int j = 0; j < m; ++j) {
        part = 0.0;
        for (int i = j + 1 + tid; i < s; i += nt) {
            const double v = A[i * p + j];
            part += v * v;
        }
        const double xn2 = block_sum(part, red);
        if (tid == 0) {
            const double al = A[j * p + j];
            if (xn2 == 0.0) {
                tau[j] = 0.0;
                bcast = 0.0;
            } else {
                const double be = -copysign(sqrt(al * al + xn2), al);
                tau[j] = (be - al) / be;
                bcast = 1.0 / (al - be);
                A[j * p + j] = be;
            }
        }
        __syncthreads();
        const double tj = tau[j];
        if (tj != 0.0) {
            const double scal = bcast;
            for (int i = j + 1 + tid; i < s; i += nt) A[i * p + j] *= scal;
            __syncthreads();
            for (int c = j + 1 + tid; c < p; c += nt) {
                double wv = A[j * p + c];
                for (int i = j + 1; i < s; ++i) wv += A[i * p + j] * A[i * p + c];
                wv *= tj;
                A[j * p + c] -= wv;
                for (int i = j + 1; i < s; ++i) A[i * p + c] -= wv * A[i * p + j];
            }
        }
        __syncthreads();
    }
    // R (a x p, upper trapezoidal) and the rank test on its diagonal
    double* Rg = R + C.rOff[g];
    for (int idx = tid; idx < a * p; idx += nt) {
        const int i = idx / p, c = idx % p;
        Rg[idx] = c >= i ? A[i * p + c] : 0.0;
    }
    if (tid == 0) {
        double dmin = DBL_MAX;
        for (int i = 0; i < a; ++i) dmin = fmin(dmin, fabs(A[i * p + i]));
        if (a > 0 && dmin <= 10.0 * (double)max(p, s) * DBL_EPSILON * normF) {
            atomicOr(flag, 1);
            atomicMax(flag + 1, g + 1);     // the highest failing cell, for the error message
        }
    }
    // Q = H_0 H_1 ... H_{m-1}, accumulated backwards on the identity
    double* Q = V + C.vOff[g];
    for (int idx = tid; idx < s * s; idx += nt) Q[idx] = (idx / s == idx % s) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = m - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        for (int c = j + tid; c < s; c += nt) {
            double wv = Q[j * s + c];
            for (int i = j + 1; i < s; ++i) wv += A[i * p + j] * Q[i * s + c];
            wv *= tj;
            Q[j * s + c] -= wv;
            for (int i = j + 1; i < s; ++i) Q[i * s + c] -= wv * A[i * p + j];
        }
        __syncthreads();
    }
}

// Forward transform of one level: coefficients = V^T (local input); the first
// a go up as scaling coefficients, the rest are the cell's rows of W v.
__global__ void wt_fwd_kernel(CellTables C, const double* __restrict__ V, int level, int leaf_level,
                              const double* __restrict__ v_kd, double* __restrict__ sbuf,
                              int64_t sbase_l, int64_t sbase_c, double* __restrict__ out) {
    extern __shared__ double in[];
    const int g = (1 << level) - 1 + blockIdx.x;
    const int s = C.s[g], a = C.a[g];
    if (level == leaf_level) {
        const int b = C.beg[g];
        for (int i = threadIdx.x; i < s; i += blockDim.x) in[i] = v_kd[b + i];
    } else {
        const int64_t o = sbase_c + C.sOff[2 * g + 1];
        for (int i = threadIdx.x; i < s; i += blockDim.x) in[i] = sbuf[o + i];
    }
    __syncthreads();
    const double* Vg = V + C.vOff[g];
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < s; ++i) acc += Vg[(int64_t)i * s + j] * in[i];
        if (j < a) sbuf[sbase_l + C.sOff[g] + j] = acc;
        else out[C.wOff[g] + (j - a)] = acc;
    }
}

// Inverse transform of one level: local output = V [scaling; wavelet coefficients].
__global__ void wt_inv_kernel(CellTables C, const double* __restrict__ V, int level, int leaf_level,
                              const double* __restrict__ u, double* __restrict__ sbuf,
                              int64_t sbase_l, int64_t sbase_c, double* __restrict__ out_kd) {
    extern __shared__ double in[];
    const int g = (1 << level) - 1 + blockIdx.x;
    const int s = C.s[g], a = C.a[g];
    for (int j = threadIdx.x; j < s; j += blockDim.x)
        in[j] = j < a ? (level == 0 ? 0.0 : sbuf[sbase_l + C.sOff[g] + j]) : u[C.wOff[g] + (j - a)];
    __syncthreads();
    const double* Vg = V + C.vOff[g];
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc += Vg[(int64_t)i * s + j] * in[j];
        if (level == leaf_level) out_kd[C.beg[g] + i] = acc;
        else sbuf[sbase_c + C.sOff[2 * g + 1] + i] = acc;
    }
}

__global__ void gather_kernel(const int* __restrict__ perm, int64_t N, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[perm[i]];
}

__global__ void scatter_kernel(const int* __restrict__ perm, int64_t N, const double* __restrict__ src,
                               double* __restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) dst[perm[i]] = src[i];
}

static unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

mlb_status build_design(mlb_ctx* ctx) {
    Box box;
    for (int k = 0; k < ctx->d; ++k) {
        box.lo[k] = ctx->box_lo[k];
        box.hi[k] = ctx->box_hi[k];
    }
    design_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(ctx->xs, ctx->N, ctx->d, ctx->p,
                                                                    ctx->alpha, box, ctx->X);
    MLB_CHECK_LAUNCH(ctx, "design_kernel");
    const int nb = 64;
    const int64_t chunk = (ctx->N + nb - 1) / nb;
    double* part = (double*)dalloc(ctx, ctx->arena_basis, sizeof(double) * nb * ctx->p * ctx->p);
    if (!part) return MLB_ENOMEM;
    xtx_partial_kernel<<<nb, 256, 0, ctx->stream>>>(ctx->X, ctx->N, ctx->p, chunk, part);
    MLB_CHECK_LAUNCH(ctx, "xtx_partial_kernel");
    xtx_chol_kernel<<<1, 128, 0, ctx->stream>>>(part, nb, ctx->p, ctx->XtXf, ctx->flag);
    MLB_CHECK_LAUNCH(ctx, "xtx_chol_kernel");
    return MLB_OK;
}

mlb_status build_factors(mlb_ctx* ctx) {
    int smax = 0;
    for (auto& c : ctx->hcells) smax = c.s > smax ? c.s : smax;
    const size_t shm = sizeof(double) * ((size_t)smax * ctx->p + ctx->p + 8);
    if ((int)shm + 1024 > max_smem_optin()) return fail(ctx, MLB_EINVAL, "leaf_size x p too large for the basis kernel");
    {
        mlb_status ss = allow_max_dynamic_smem(ctx, (const void*)qr_level_kernel, "qr_level_kernel smem");
        if (ss != MLB_OK) return ss;
    }
    for (int l = ctx->t; l >= 0; --l) {
        qr_level_kernel<<<1u << l, 128, shm, ctx->stream>>>(ctx->cells, ctx->X, ctx->p, l, ctx->t,
                                                           ctx->V, ctx->R, ctx->flag);
        MLB_CHECK_LAUNCH(ctx, "qr_level_kernel");
    }
    return MLB_OK;
}

static int max_s(mlb_ctx* ctx) {
    int smax = 0;
    for (auto& c : ctx->hcells) smax = c.s > smax ? c.s : smax;
    return smax;
}

mlb_status apply_W_dev(mlb_ctx* ctx, const double* v_kd, double* out) {
    const size_t shm = sizeof(double) * max_s(ctx);
    for (int l = ctx->t; l >= 0; --l) {
        const int64_t sc = l < ctx->t ? ctx->sbase[l + 1] : 0;
        wt_fwd_kernel<<<1u << l, 128, shm, ctx->stream>>>(ctx->cells, ctx->V, l, ctx->t, v_kd, ctx->sbuf,
                                                         ctx->sbase[l], sc, out);
        MLB_CHECK_LAUNCH(ctx, "wt_fwd_kernel");
    }
    return MLB_OK;
}

mlb_status apply_Wt_dev(mlb_ctx* ctx, const double* u, double* out_kd) {
    const size_t shm = sizeof(double) * max_s(ctx);
    for (int l = 0; l <= ctx->t; ++l) {
        const int64_t sc = l < ctx->t ? ctx->sbase[l + 1] : 0;
        wt_inv_kernel<<<1u << l, 128, shm, ctx->stream>>>(ctx->cells, ctx->V, l, ctx->t, u, ctx->sbuf,
                                                         ctx->sbase[l], sc, out_kd);
        MLB_CHECK_LAUNCH(ctx, "wt_inv_kernel");
    }
    return MLB_OK;
}

mlb_status gather_kd(mlb_ctx* ctx, const double* v_user, double* v_kd) {
    gather_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(ctx->perm, ctx->N, v_user, v_kd);
    MLB_CHECK_LAUNCH(ctx, "gather_kernel");
    return MLB_OK;
}

mlb_status scatter_kd(mlb_ctx* ctx, const double* v_kd, double* v_user) {
    scatter_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(ctx->perm, ctx->N, v_kd, v_user);
    MLB_CHECK_LAUNCH(ctx, "scatter_kernel");
    return MLB_OK;
}

}  // namespace mlb

// ---------------------------------------------------------------------------
// W v without any device allocation.
//
// Some callers cannot allocate device memory when they need W v: real-time
// loops that must not block on the allocator (cudaMalloc can synchronise the
// device), processes held to a fixed device-memory budget, and hosts whose
// device memory is owned by another framework's pool.  For them this
// entry point keeps its work space -- the input reordered into kd-tree order
// and the scaling coefficients of every level -- in one fixed array in device
// global memory that every GPU loading this library reserves until the
// process exits.  Its size bounds the problems it accepts:
// N + (scaling coefficients of all levels) <= kNoAllocScratchDoubles.
// Every element read during a call is first written by the same call, so
// nothing needs clearing between calls; but all calls on one device share the
// array, so two calls whose kernels overlap in time (different streams or
// contexts) race on it.
// ---------------------------------------------------------------------------
namespace mlb {

constexpr int64_t kNoAllocScratchDoubles = 524288;   // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;
static double* g_noalloc_ptr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static mlb_status noalloc_scratch(mlb_ctx* ctx, double** out) {
    int dev = 0;
    MLB_CUDA(ctx, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(ctx, MLB_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return MLB_OK;
}

}  // namespace mlb

extern "C" mlb_status mlb_apply_W_noalloc(mlb_ctx* ctx, const double* v_dev, double* out_dev) {
    using namespace mlb;
    if (!ctx || !v_dev || !out_dev) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 1) return fail(ctx, MLB_ESTATE, "mlb_apply_W_noalloc needs mlb_build_basis first");
    const int64_t need = ctx->N + ctx->sbase[ctx->t + 1];
    if (need > kNoAllocScratchDoubles)
        return fail(ctx, MLB_EINVAL,
                    "mlb_apply_W_noalloc: N plus the scaling coefficients (" + std::to_string(need) +
                        " doubles) exceed its fixed work space of " + std::to_string(kNoAllocScratchDoubles) +
                        " doubles; use mlb_apply_W");
    if (cudaSetDevice(ctx->opts.device) != cudaSuccess) return fail(ctx, MLB_ECUDA, "cudaSetDevice failed");
    double* scratch = nullptr;
    mlb_status s = noalloc_scratch(ctx, &scratch);
    if (s != MLB_OK) return s;
    double* v_kd = scratch;                 // N entries
    double* sb = scratch + ctx->N;          // the levels' scaling coefficients
    gather_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(ctx->perm, ctx->N, v_dev, v_kd);
    MLB_CHECK_LAUNCH(ctx, "gather_kernel");
    const size_t shm = sizeof(double) * max_s(ctx);
    for (int l = ctx->t; l >= 0; --l) {
        const int64_t sc = l < ctx->t ? ctx->sbase[l + 1] : 0;
        wt_fwd_kernel<<<1u << l, 128, shm, ctx->stream>>>(ctx->cells, ctx->V, l, ctx->t, v_kd, sb, ctx->sbase[l],
                                                         sc, out_dev);
        MLB_CHECK_LAUNCH(ctx, "wt_fwd_kernel");
    }
    return MLB_OK;
}
