// Kernel sums out_k = sum_j phi(|y_k - x_j|) a_j over the data points (Sec.
// 6.2: the product C gamma of the trend step, and c(x0)^T gamma of the
// prediction, eq. Spatial), optionally plus the trend k(y_k)^T beta.
//
// One thread per target; the data points and weights stream through shared
// memory in tiles of 128.  Distances are formed from coordinate differences
// (no |x|^2 + |y|^2 - 2 x.y cancellation).  FP64 path: FP64 throughout.
#include <cmath>

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
__global__ void __launch_bounds__(128) ksum_f64_kernel(const double* __restrict__ tg, int64_t M,
                                                       const double* __restrict__ xs,
                                                       const double* __restrict__ a, int64_t N, int kind,
                                                       double scale, double* __restrict__ out, TrendArgs tr) {
    __shared__ double sx[128 * D];
    __shared__ double sa[128];
    const int64_t k = blockIdx.x * 128LL + threadIdx.x;
    double y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = k < M ? tg[k * D + c] : 0.0;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < N; j0 += 128) {
        const int nj = (int)(N - j0 < 128 ? N - j0 : 128);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nj * D; idx += 128) sx[idx] = xs[j0 * D + idx];
        if (threadIdx.x < nj) sa[threadIdx.x] = a[j0 + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            double r2 = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double df = y[c] - sx[j * D + c];
                r2 += df * df;
            }
            acc += matern_f64(sqrt(r2), kind, scale) * sa[j];
        }
    }
    if (k >= M) return;
    if (tr.beta) {
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
    out[k] = acc;
}

template <int D>
static void launch_ksum(mlb_ctx* ctx, const double* tg, int64_t M, const double* a, double* out, TrendArgs tr) {
    const int kind = nu_kind(ctx->theta.nu);
    const double scale = std::sqrt(2.0 * ctx->theta.nu) / ctx->theta.rho;
    const unsigned grid = (unsigned)((M + 127) / 128);
    ksum_f64_kernel<D><<<grid, 128, 0, ctx->stream>>>(tg, M, ctx->xs, a, ctx->N, kind, scale, out, tr);
}

mlb_status kernel_sum_dev(mlb_ctx* ctx, const double* targets, int64_t M, const double* a_kd, double* out,
                          bool add_trend) {
    if (M <= 0) return MLB_OK;
    TrendArgs tr{};
    tr.beta = add_trend ? ctx->beta : nullptr;
    tr.alpha = ctx->alpha;
    tr.p = ctx->p;
    for (int c = 0; c < ctx->d; ++c) {
        tr.lo[c] = ctx->box_lo[c];
        tr.hi[c] = ctx->box_hi[c];
    }
    const double* tg = targets ? targets : ctx->xs;
    switch (ctx->d) {
#define MLB_KSUM_CASE(DD) \
    case DD: launch_ksum<DD>(ctx, tg, M, a_kd, out, tr); break;
        MLB_KSUM_CASE(1) MLB_KSUM_CASE(2) MLB_KSUM_CASE(3) MLB_KSUM_CASE(4)
        MLB_KSUM_CASE(5) MLB_KSUM_CASE(6) MLB_KSUM_CASE(7) MLB_KSUM_CASE(8)
        MLB_KSUM_CASE(9) MLB_KSUM_CASE(10) MLB_KSUM_CASE(11) MLB_KSUM_CASE(12)
        MLB_KSUM_CASE(13) MLB_KSUM_CASE(14) MLB_KSUM_CASE(15) MLB_KSUM_CASE(16)
#undef MLB_KSUM_CASE
        default: return fail(ctx, MLB_EINVAL, "dimension d out of range 1..16");
    }
    MLB_CHECK_LAUNCH(ctx, "ksum_f64_kernel");
    return MLB_OK;
}

}  // namespace mlb
