// Gradient of the held-out loss L = (1/M) sum_k (Y-hat_k - y_k)^2 in log(rho)
// and log(nugget), by the adjoint of the saddle-point system of Sec. 5.2
// (eq. Spatial:problem).  The paper estimates theta by maximum likelihood and
// has no gradient of the predictor; the adjoint is written from its BLUP
// equations:
//
//   g_k = 2 (Y-hat_k - y_k) / M,  a = sum_k g_k c(x0_k),  b = sum_k g_k k(x0_k)
//   [[C, X], [X^T, 0]] [lambda; mu] = [a; b], solved the multilevel way:
//     lambda_0 = X (X^T X)^{-1} b          (X^T lambda_0 = b, W lambda_0 = 0)
//     C~_W lambda_W = W (a - C lambda_0)   (the same PCG as the forward solve)
//     lambda = lambda_0 + W^T lambda_W
//   dL/dlog(rho) = sum_k g_k (dc_k/dlog rho)^T gamma - lambda^T (dC/dlog rho) gamma
//   dL/dlog(eta) = -eta lambda^T gamma
//
// The derivative blocks enter only through kernel sums with d phi/d log(rho)
// evaluated on the fly (never a stored dC/drho or dC_W/drho).
#include <cmath>

#include "internal.h"

namespace mlb {

constexpr int kRedBlocks = 256;

__device__ double block_sum_all(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// g = 2 (yhat - y) / M; part[b] = sum of (yhat - y)^2 over the block's share
__global__ void residual_kernel(int64_t M, const double* __restrict__ yhat, const double* __restrict__ y,
                                double* __restrict__ g, double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        const double r = yhat[k] - y[k];
        g[k] = 2.0 * r / (double)M;
        acc += r * r;
    }
    const double s = block_sum_all(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* part) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * y[i];
    const double s = block_sum_all(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// b_m = sum_k g_k k_m(x0_k) (monomials of the box-scaled target coordinates)
__global__ void trend_adjoint_kernel(int64_t M, int d, int p, const double* __restrict__ tg,
                                     const double* __restrict__ g, const int* __restrict__ alpha,
                                     const double* __restrict__ lo, const double* __restrict__ hi,
                                     double* __restrict__ part) {
    extern __shared__ double acc[];    // p x blockDim.x
    for (int m = 0; m < p; ++m) acc[m * blockDim.x + threadIdx.x] = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        double u[kMaxDim];
        for (int c = 0; c < d; ++c) {
            const double span = hi[c] - lo[c];
            u[c] = span > 0.0 ? 2.0 * (tg[k * d + c] - lo[c]) / span - 1.0 : 0.0;
        }
        for (int m = 0; m < p; ++m) {
            double v = g[k];
            for (int c = 0; c < d; ++c)
                for (int e = 0; e < alpha[m * d + c]; ++e) v *= u[c];
            acc[m * blockDim.x + threadIdx.x] += v;
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < p; m += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += acc[m * blockDim.x + i];
        part[(int64_t)blockIdx.x * p + m] = s;
    }
}

// c = (L L^T)^{-1} sum_b part[b]  (p <= 128, one thread)
__global__ void small_solve_kernel(const double* part, int nb, int p, const double* L, double* c) {
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
    for (int j = 0; j < p; ++j) c[j] = y[j];
}

// lambda_0 = X c
__global__ void xc_kernel(int64_t N, int p, const double* __restrict__ X, const double* __restrict__ c,
                          double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int m = 0; m < p; ++m) s += X[i * p + m] * c[m];
    out[i] = s;
}

// rhs = a - (K lambda_0) - eta lambda_0
__global__ void rhs_kernel(int64_t N, const double* __restrict__ a, const double* __restrict__ Kl,
                           const double* __restrict__ l0, double eta, double* __restrict__ rhs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) rhs[i] = a[i] - Kl[i] - eta * l0[i];
}

__global__ void add_kernel(int64_t N, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) y[i] += x[i];
}

// out3 = [loss, dlogrho, dlognugget] from the four partial-sum arrays
__global__ void finish_kernel(const double* pl, const double* p1, const double* p2, const double* p3, int nb,
                              int64_t M, double eta, double* out3) {
    if (threadIdx.x) return;
    double l = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int b = 0; b < nb; ++b) {
        l += pl[b];
        t1 += p1[b];
        t2 += p2[b];
        t3 += p3[b];
    }
    out3[0] = l / (double)M;
    out3[1] = t1 - t2;
    out3[2] = -eta * t3;
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

mlb_status grad_dev(mlb_ctx* ctx, const double* tg, int64_t M, const double* y, double* out3) {
    cudaStream_t st = ctx->stream;
    const int64_t N = ctx->N, nw = ctx->nwav;
    const int p = ctx->p, d = ctx->d;
    Arena tmp;
    double* yhat = (double*)dalloc(ctx, tmp, sizeof(double) * M);
    double* g = (double*)dalloc(ctx, tmp, sizeof(double) * M);
    double* t1 = (double*)dalloc(ctx, tmp, sizeof(double) * M);
    double* a = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* l0 = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* Kl = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* lam = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* t2 = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* rw = (double*)dalloc(ctx, tmp, sizeof(double) * nw);
    double* lw = (double*)dalloc(ctx, tmp, sizeof(double) * nw);
    double* c = (double*)dalloc(ctx, tmp, sizeof(double) * 128);
    double* box = (double*)dalloc(ctx, tmp, sizeof(double) * 2 * kMaxDim);
    double* part = (double*)dalloc(ctx, tmp, sizeof(double) * (size_t)(4 * kRedBlocks + kRedBlocks * 128));
    mlb_status s = MLB_OK;
    if (!yhat || !g || !t1 || !a || !l0 || !Kl || !lam || !t2 || !rw || !lw || !c || !box || !part) {
        tmp.release();
        return fail(ctx, MLB_ENOMEM, "gradient work buffers");
    }
    double* pl = part;
    double* p1 = part + kRedBlocks;
    double* p2 = part + 2 * kRedBlocks;
    double* p3 = part + 3 * kRedBlocks;
    double* pb = part + 4 * kRedBlocks;
    double hb[2 * kMaxDim];
    for (int q = 0; q < d; ++q) {
        hb[q] = ctx->box_lo[q];
        hb[kMaxDim + q] = ctx->box_hi[q];
    }
    do {
        if (cudaMemcpyAsync(box, hb, sizeof(hb), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            s = fail(ctx, MLB_ECUDA, "copy");
            break;
        }
        // forward predictions and the loss residual
        if ((s = kernel_sum_general(ctx, tg, M, nullptr, N, ctx->gamma, yhat, true, false)) != MLB_OK) break;
        residual_kernel<<<kRedBlocks, 256, 0, st>>>(M, yhat, y, g, pl);
        // a = sum_k g_k c(x0_k): kernel sum at the data points over the targets
        if ((s = kernel_sum_general(ctx, nullptr, N, tg, M, g, a, false, false)) != MLB_OK) break;
        // b = sum_k g_k k(x0_k), lambda_0 = X (X^T X)^{-1} b
        trend_adjoint_kernel<<<kRedBlocks, 32, sizeof(double) * 32 * p, st>>>(M, d, p, tg, g, ctx->alpha, box,
                                                                            box + kMaxDim, pb);
        small_solve_kernel<<<1, 32, 0, st>>>(pb, kRedBlocks, p, ctx->XtXf, c);
        xc_kernel<<<nblk(N), 256, 0, st>>>(N, p, ctx->X, c, l0);
        MLB_CHECK_LAUNCH(ctx, "adjoint trend");
        ctx->launches += 3;
        // C~_W lambda_W = W (a - C lambda_0)
        if ((s = kernel_sum_dev(ctx, nullptr, N, l0, Kl, false)) != MLB_OK) break;
        rhs_kernel<<<nblk(N), 256, 0, st>>>(N, a, Kl, l0, ctx->theta.nugget, t2);
        MLB_CHECK_LAUNCH(ctx, "rhs_kernel");
        if ((s = apply_W_dev(ctx, t2, rw)) != MLB_OK) break;
        mlb_info ai{};
        s = pcg_run(ctx, rw, lw, &ai);
        if (s != MLB_OK) break;
        if ((s = apply_Wt_dev(ctx, lw, lam)) != MLB_OK) break;
        add_kernel<<<nblk(N), 256, 0, st>>>(N, l0, lam);
        // derivative kernel sums against gamma
        if ((s = kernel_sum_general(ctx, tg, M, nullptr, N, ctx->gamma, t1, false, true)) != MLB_OK) break;
        if ((s = kernel_sum_general(ctx, nullptr, N, nullptr, N, ctx->gamma, t2, false, true)) != MLB_OK) break;
        dot_kernel<<<kRedBlocks, 256, 0, st>>>(M, g, t1, p1);
        dot_kernel<<<kRedBlocks, 256, 0, st>>>(N, lam, t2, p2);
        dot_kernel<<<kRedBlocks, 256, 0, st>>>(N, lam, ctx->gamma, p3);
        finish_kernel<<<1, 32, 0, st>>>(pl, p1, p2, p3, kRedBlocks, M, ctx->theta.nugget, out3);
        MLB_CHECK_LAUNCH(ctx, "gradient reductions");
        ctx->launches += 5;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "gradient");
    } while (0);
    cudaStreamSynchronize(st);
    tmp.release();
    return s;
}

}  // namespace mlb

namespace mlb {

// part[b][m] = sum over the block's rows of X[r][m] v[r]
__global__ void xtv_kernel(int64_t N, int p, const double* __restrict__ X, const double* __restrict__ v,
                           int64_t chunk, double* __restrict__ part) {
    const int64_t r0 = blockIdx.x * chunk, r1 = min(N, r0 + chunk);
    for (int m = threadIdx.x; m < p; m += blockDim.x) {
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) acc += X[r * p + m] * v[r];
        part[(int64_t)blockIdx.x * p + m] = acc;
    }
}

// out = 1 - a.lambda - b.mu from the partials of a.lambda and the p-vectors b, mu
__global__ void mse_finish_kernel(const double* pa, int nb, const double* b, const double* mu, int p, double* out) {
    if (threadIdx.x) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += pa[i];
    double t = 0.0;
    for (int m = 0; m < p; ++m) t += b[m] * mu[m];
    *out = 1.0 - s - t;
}

// Kriging mean squared error at each target (the formula after eq. Spatial,
// unit variance): MSE(x0) = 1 - c^T lambda - k^T mu, where [lambda; mu] solves
// the saddle-point system [[C, X], [X^T, 0]] [lambda; mu] = [c(x0); k(x0)]
// (substituting lambda = C^{-1}(c - X mu) and X^T lambda = k gives the
// printed 1 + u^T (X^T C^{-1} X)^{-1} u - c^T C^{-1} c).  Solved the
// multilevel way, one target at a time:
//   lambda_0 = X (X^T X)^{-1} k,  C~_W lambda_W = W (c - C lambda_0),
//   lambda = lambda_0 + W^T lambda_W,  mu = (X^T X)^{-1} X^T (c - C lambda).
// The kernel sums run at the one-shot accuracy (double-float on the mixed
// path); the PCG is the context's (FP32 or FP64 C~_W), with kRhs targets per
// pass over the FP32 panels.
mlb_status mse_dev(mlb_ctx* ctx, const double* tg, int64_t M, double* out) {
    cudaStream_t st = ctx->stream;
    const int64_t N = ctx->N, nw = ctx->nwav;
    const int p = ctx->p, d = ctx->d;
    // on the FP32 panels kRhs targets share each pass over C~_W (one PCG
    // recurrence per target, one product for all); otherwise one at a time
    const bool multi = !ctx->opts.matrix_free && (ctx->sym.vals || (ctx->pan.vals32 && ctx->pan.nwork > 0));
    const int R = multi ? kRhs : 1;
    Arena tmp;
    double* A = (double*)dalloc(ctx, tmp, sizeof(double) * R * N);      // c(x0) per slot
    double* L0 = (double*)dalloc(ctx, tmp, sizeof(double) * R * N);     // lambda_0 per slot
    double* Bk = (double*)dalloc(ctx, tmp, sizeof(double) * R * 128);   // k(x0) per slot
    double* RW = (double*)dalloc(ctx, tmp, sizeof(double) * R * nw);    // right-hand sides W(c - C lambda_0)
    double* LW = (double*)dalloc(ctx, tmp, sizeof(double) * R * nw);    // lambda_W
    double* Kl = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* lam = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* t2 = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* small = (double*)dalloc(ctx, tmp, sizeof(double) * (3 * 128 + 8));
    double* box = (double*)dalloc(ctx, tmp, sizeof(double) * 2 * kMaxDim);
    double* part = (double*)dalloc(ctx, tmp, sizeof(double) * (size_t)(kRedBlocks * 128 + kRedBlocks));
    double* work = multi ? (double*)dalloc(ctx, tmp, sizeof(double) * pcg_multi_work_doubles(ctx)) : nullptr;
    if (!A || !L0 || !Bk || !RW || !LW || !Kl || !lam || !t2 || !small || !box || !part || (multi && !work)) {
        tmp.release();
        return fail(ctx, MLB_ENOMEM, "MSE work buffers");
    }
    double* one = small;            // the weight 1 of a single source
    double* c = small + 8;          // (X^T X)^{-1} k(x0)
    double* mu = c + 128;
    double* pa = part + (size_t)kRedBlocks * 128;
    double hb[2 * kMaxDim + 1];
    for (int q = 0; q < d; ++q) {
        hb[q] = ctx->box_lo[q];
        hb[kMaxDim + q] = ctx->box_hi[q];
    }
    hb[2 * kMaxDim] = 1.0;
    const int64_t chunk = (N + kRedBlocks - 1) / kRedBlocks;
    mlb_status s = MLB_OK;
    do {
        if (cudaMemcpyAsync(box, hb, sizeof(double) * 2 * kMaxDim, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(one, hb + 2 * kMaxDim, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            s = fail(ctx, MLB_ECUDA, "copy");
            break;
        }
        for (int64_t k0 = 0; k0 < M && s == MLB_OK; k0 += R) {
            // per slot: c(x0), k(x0), lambda_0 = X (X^T X)^{-1} k(x0) and the
            // right-hand side W (c(x0) - C lambda_0); slots past M repeat the
            // last target and are not reported
            for (int r = 0; r < R && s == MLB_OK; ++r) {
                const double* x0 = tg + std::min<int64_t>(k0 + r, M - 1) * d;
                double* a = A + (int64_t)r * N;
                double* l0 = L0 + (int64_t)r * N;
                double* b = Bk + r * 128;
                if ((s = kernel_sum_general(ctx, nullptr, N, x0, 1, one, a, false, false, true)) != MLB_OK) break;
                trend_adjoint_kernel<<<1, 32, sizeof(double) * 32 * p, st>>>(1, d, p, x0, one, ctx->alpha, box,
                                                                             box + kMaxDim, b);
                small_solve_kernel<<<1, 32, 0, st>>>(b, 1, p, ctx->XtXf, c);
                xc_kernel<<<nblk(N), 256, 0, st>>>(N, p, ctx->X, c, l0);
                MLB_CHECK_LAUNCH(ctx, "MSE trend part");
                ctx->launches += 2;
                if ((s = kernel_sum_general(ctx, nullptr, N, nullptr, N, l0, Kl, false, false, true)) != MLB_OK) break;
                rhs_kernel<<<nblk(N), 256, 0, st>>>(N, a, Kl, l0, ctx->theta.nugget, t2);
                MLB_CHECK_LAUNCH(ctx, "rhs_kernel");
                if ((s = apply_W_dev(ctx, t2, RW + (int64_t)r * nw)) != MLB_OK) break;
            }
            if (s != MLB_OK) break;
            // C~_W lambda_W = W (c(x0) - C lambda_0)
            if (multi) {
                if ((s = pcg_run_multi(ctx, RW, LW, work, nullptr)) != MLB_OK) break;
            } else {
                mlb_info ai{};
                if ((s = pcg_run(ctx, RW, LW, &ai)) != MLB_OK) break;
            }
            for (int r = 0; r < R && k0 + r < M && s == MLB_OK; ++r) {
                const double* a = A + (int64_t)r * N;
                // lambda = lambda_0 + W^T lambda_W; mu = (X^T X)^{-1} X^T (c(x0) - C lambda - eta lambda)
                if ((s = apply_Wt_dev(ctx, LW + (int64_t)r * nw, lam)) != MLB_OK) break;
                add_kernel<<<nblk(N), 256, 0, st>>>(N, L0 + (int64_t)r * N, lam);
                MLB_CHECK_LAUNCH(ctx, "add_kernel");
                if ((s = kernel_sum_general(ctx, nullptr, N, nullptr, N, lam, Kl, false, false, true)) != MLB_OK) break;
                rhs_kernel<<<nblk(N), 256, 0, st>>>(N, a, Kl, lam, ctx->theta.nugget, t2);
                xtv_kernel<<<kRedBlocks, 32, 0, st>>>(N, p, ctx->X, t2, chunk, part);
                small_solve_kernel<<<1, 32, 0, st>>>(part, kRedBlocks, p, ctx->XtXf, mu);
                dot_kernel<<<kRedBlocks, 256, 0, st>>>(N, a, lam, pa);
                mse_finish_kernel<<<1, 32, 0, st>>>(pa, kRedBlocks, Bk + r * 128, mu, p, out + k0 + r);
                MLB_CHECK_LAUNCH(ctx, "MSE reductions");
                ctx->launches += 4;
            }
        }
        if (s != MLB_OK) break;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "MSE");
    } while (0);
    cudaStreamSynchronize(st);
    tmp.release();
    return s;
}

}  // namespace mlb
