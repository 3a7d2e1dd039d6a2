// Multilevel log-likelihood (Sec. 5.1, the reduced likelihood for the full
// transform, n = 0):
//
//   l_W(theta) = -(N~/2) log(2 pi) - (1/2) log det C~_W - (1/2) Z_W^T C~_W^{-1} Z_W,
//
// with Z_W = W Z and N~ = N - p.  The quadratic form comes from the PCG solve
// of C~_W g = Z_W (Z_W . g).  The paper takes log det from a sparse Cholesky
// factorisation by a third-party package; here it is estimated by stochastic
// Lanczos quadrature (Ubaru, Chen and Saad, "Fast estimation of tr(f(A)) via
// stochastic Lanczos quadrature", SIAM J. Matrix Anal. Appl. 38 (2017)):
//
//   log det A = tr log A ~ (1/m) sum_i |v_i|^2 sum_j (e_1^T u_j)^2 log(theta_j),
//
// where, for each probe v_i = W z_i (z_i supplied by the caller in the data
// space, so that E[v v^T] = W W^T = I for z with identity covariance), k
// Lanczos steps on A = C~_W from v_i / |v_i| give the tridiagonal T_k with
// eigenpairs (theta_j, u_j).  The Lanczos vectors are fully reorthogonalised
// (classical Gram-Schmidt, twice), so the recurrence is stable and its result
// does not depend on the basis chosen inside each cell.  The k x k
// eigenproblem is solved on the host by cyclic Jacobi rotations (Golub and
// Van Loan, Matrix Computations, Sec. 8.5).
#include <cmath>
#include <vector>

#include "internal.h"

namespace mlb {

constexpr int kLzBlocks = 256;

__device__ double lz_block_sum(double v) {
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

// part[c * gridDim.x + b] = sum over block b's share of Q[c] . w, for c < nc
// (Q row-major, nc vectors of length n); blockIdx.y = c.
__global__ void lz_multidot_kernel(int64_t n, const double* __restrict__ Q, int64_t ldq,
                                   const double* __restrict__ w, double* __restrict__ part) {
    const int c = blockIdx.y;
    const double* q = Q + c * ldq;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += q[i] * w[i];
    const double s = lz_block_sum(acc);
    if (threadIdx.x == 0) part[(int64_t)c * gridDim.x + blockIdx.x] = s;
}

// coef[c] = sum over blocks of part[c][*], in order (one thread per c)
__global__ void lz_reduce_kernel(const double* __restrict__ part, int nb, int nc, double* __restrict__ coef) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)c * nb + b];
    coef[c] = s;
}

// w -= sum_{c < nc} coef[c] Q[c]
__global__ void lz_project_kernel(int64_t n, const double* __restrict__ Q, int64_t ldq, int nc,
                                  const double* __restrict__ coef, double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int c = 0; c < nc; ++c) s -= coef[c] * Q[c * ldq + i];
        w[i] = s;
    }
}

// out = w / sqrt(ww) (0 when ww == 0); beta = sqrt(ww)
__global__ void lz_normalize_kernel(int64_t n, const double* __restrict__ w, const double* __restrict__ ww,
                                    double* __restrict__ out, double* __restrict__ beta) {
    const double b = sqrt(fmax(*ww, 0.0));
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) *beta = b;
}

// Symmetric k x k eigenproblem by cyclic Jacobi; returns the eigenvalues and
// the first components of the normalised eigenvectors.
static void jacobi_eigen(std::vector<double> A, int k, std::vector<double>& theta, std::vector<double>& u0) {
    std::vector<double> V((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                const double a2 = A[(size_t)i * k + j] * A[(size_t)i * k + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[(size_t)p * k + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int r = 0; r < k; ++r) {     // A <- A J (columns p, q)
                    const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
                    A[(size_t)r * k + p] = c * arp - s * arq;
                    A[(size_t)r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {     // A <- J^T A (rows p, q)
                    const double apr = A[(size_t)p * k + r], aqr = A[(size_t)q * k + r];
                    A[(size_t)p * k + r] = c * apr - s * aqr;
                    A[(size_t)q * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {     // V <- V J
                    const double vrp = V[(size_t)r * k + p], vrq = V[(size_t)r * k + q];
                    V[(size_t)r * k + p] = c * vrp - s * vrq;
                    V[(size_t)r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    theta.assign(k, 0.0);
    u0.assign(k, 0.0);
    for (int j = 0; j < k; ++j) {
        theta[j] = A[(size_t)j * k + j];
        u0[j] = V[j];                            // row 0, column j
    }
}

static unsigned lz_grid(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < kLzBlocks ? (b > 0 ? b : 1) : kLzBlocks);
}

// log det C~_W by stochastic Lanczos quadrature with nprobe caller probes
// (device, nprobe x N in caller order) and `steps` Lanczos steps each.
mlb_status logdet_slq_dev(mlb_ctx* ctx, const double* probes, int nprobe, int steps, double* logdet) {
    cudaStream_t st = ctx->stream;
    const int64_t N = ctx->N, n = ctx->nwav;
    const int k = (int)std::min<int64_t>(steps, n);
    Arena tmp;
    double* Q = (double*)dalloc(ctx, tmp, sizeof(double) * (size_t)(k + 1) * n);
    double* w = (double*)dalloc(ctx, tmp, sizeof(double) * n);
    double* zk = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* part = (double*)dalloc(ctx, tmp, sizeof(double) * (size_t)kLzBlocks * (k + 1));
    double* coef = (double*)dalloc(ctx, tmp, sizeof(double) * (k + 2));
    double* ab = (double*)dalloc(ctx, tmp, sizeof(double) * 2 * (k + 1));    // alpha[0..k), beta[0..k)
    double* nrm = (double*)dalloc(ctx, tmp, sizeof(double) * 2);
    if (!Q || !w || !zk || !part || !coef || !ab || !nrm) {
        tmp.release();
        return fail(ctx, MLB_ENOMEM, "Lanczos work buffers");
    }
    double* alpha = ab;
    double* beta = ab + (k + 1);
    const unsigned g = lz_grid(n);
    double total = 0.0;
    mlb_status s = MLB_OK;
    for (int pi = 0; pi < nprobe && s == MLB_OK; ++pi) {
        // v = W z (the probe in the wavelet space), q_0 = v / |v|
        if ((s = gather_kd(ctx, probes + (int64_t)pi * N, zk)) != MLB_OK) break;
        if ((s = apply_W_dev(ctx, zk, w)) != MLB_OK) break;
        lz_multidot_kernel<<<dim3(g, 1), 256, 0, st>>>(n, w, n, w, part);
        lz_reduce_kernel<<<1, 32, 0, st>>>(part, g, 1, nrm);
        lz_normalize_kernel<<<g, 256, 0, st>>>(n, w, nrm, Q, nrm + 1);
        MLB_CHECK_LAUNCH(ctx, "Lanczos start");
        ctx->launches += 2;
        for (int j = 0; j < k; ++j) {
            double* qj = Q + (int64_t)j * n;
            if ((s = cw_matvec_dev(ctx, qj, w)) != MLB_OK) break;
            // alpha_j = q_j . w, then w -= sum_{c <= j} (q_c . w) q_c, twice: the
            // first pass removes alpha_j q_j and beta_{j-1} q_{j-1} with the rest
            lz_multidot_kernel<<<dim3(g, j + 1), 256, 0, st>>>(n, Q, n, w, part);
            lz_reduce_kernel<<<1, 128, 0, st>>>(part, g, j + 1, coef);
            cudaMemcpyAsync(alpha + j, coef + j, sizeof(double), cudaMemcpyDeviceToDevice, st);
            lz_project_kernel<<<g, 256, 0, st>>>(n, Q, n, j + 1, coef, w);
            lz_multidot_kernel<<<dim3(g, j + 1), 256, 0, st>>>(n, Q, n, w, part);
            lz_reduce_kernel<<<1, 128, 0, st>>>(part, g, j + 1, coef);
            lz_project_kernel<<<g, 256, 0, st>>>(n, Q, n, j + 1, coef, w);
            // beta_j = |w|, q_{j+1} = w / beta_j
            lz_multidot_kernel<<<dim3(g, 1), 256, 0, st>>>(n, w, n, w, part);
            lz_reduce_kernel<<<1, 32, 0, st>>>(part, g, 1, nrm);
            lz_normalize_kernel<<<g, 256, 0, st>>>(n, w, nrm, Q + (int64_t)(j + 1) * n, beta + j);
            MLB_CHECK_LAUNCH(ctx, "Lanczos step");
            ctx->launches += 8;
        }
        if (s != MLB_OK) break;
        std::vector<double> ha(k), hb(k), hv(1);
        MLB_CUDA(ctx, cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaMemcpyAsync(hb.data(), beta, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaMemcpyAsync(hv.data(), nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        // the coefficient of q_0 was computed as |v|; an invariant subspace
        // (beta_j ~ 0) ends the recurrence at j + 1 steps
        const double vnorm = hv[0];
        int kk = k;
        for (int j = 0; j < k - 1; ++j)
            if (!(hb[j] > 1e-12 * std::fabs(ha[j]))) {
                kk = j + 1;
                break;
            }
        std::vector<double> T((size_t)kk * kk, 0.0);
        for (int j = 0; j < kk; ++j) {
            T[(size_t)j * kk + j] = ha[j];
            if (j + 1 < kk) T[(size_t)j * kk + j + 1] = T[(size_t)(j + 1) * kk + j] = hb[j];
        }
        std::vector<double> theta, u0;
        jacobi_eigen(T, kk, theta, u0);
        double q = 0.0;
        for (int j = 0; j < kk; ++j) {
            if (!(theta[j] > 0.0)) {
                s = fail(ctx, MLB_EBREAKDOWN, "Lanczos: C~_W is not positive definite");
                break;
            }
            q += u0[j] * u0[j] * std::log(theta[j]);
        }
        total += vnorm * vnorm * q;
    }
    cudaStreamSynchronize(st);
    tmp.release();
    if (s == MLB_OK) *logdet = total / (double)std::max(nprobe, 1);
    return s;
}

}  // namespace mlb

using namespace mlb;

namespace {

__global__ void lz_dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * y[i];
    const double s = lz_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace

extern "C" mlb_status mlb_loglik(mlb_ctx* ctx, const double* Z, const double* probes, int nprobe, int steps,
                                 double* out3) {
    if (!ctx || !Z || !out3 || nprobe < 0 || (nprobe > 0 && !probes) || steps < 1 || steps > 100)
        return fail(ctx, MLB_EINVAL, "bad argument (1 <= steps <= 100)");
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "mlb_loglik needs mlb_assemble first");
    cudaSetDevice(ctx->opts.device);
    cudaStream_t st = ctx->stream;
    const int64_t N = ctx->N, n = ctx->nwav;
    Arena tmp;
    double* Zd = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* Zk = (double*)dalloc(ctx, tmp, sizeof(double) * N);
    double* ZW = (double*)dalloc(ctx, tmp, sizeof(double) * std::max<int64_t>(n, 1));
    double* gW = (double*)dalloc(ctx, tmp, sizeof(double) * std::max<int64_t>(n, 1));
    double* part = (double*)dalloc(ctx, tmp, sizeof(double) * kLzBlocks);
    double* pr = nprobe > 0 ? (double*)dalloc(ctx, tmp, sizeof(double) * (size_t)nprobe * N) : nullptr;
    if (!Zd || !Zk || !ZW || !gW || !part || (nprobe > 0 && !pr)) {
        tmp.release();
        return fail(ctx, MLB_ENOMEM, "likelihood work buffers");
    }
    mlb_status s = MLB_OK;
    double quad = 0.0, logdet = 0.0;
    do {
        if (cudaMemcpyAsync(Zd, Z, sizeof(double) * N, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            (nprobe > 0 &&
             cudaMemcpyAsync(pr, probes, sizeof(double) * (size_t)nprobe * N, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
            s = fail(ctx, MLB_ECUDA, "copy of Z or the probes failed");
            break;
        }
        // quadratic form Z_W^T C~_W^{-1} Z_W from the PCG solve
        if ((s = gather_kd(ctx, Zd, Zk)) != MLB_OK) break;
        if ((s = apply_W_dev(ctx, Zk, ZW)) != MLB_OK) break;
        mlb_info info{};
        if ((s = pcg_run(ctx, ZW, gW, &info)) != MLB_OK) break;
        const unsigned g = lz_grid(n);
        lz_dot_kernel<<<g, 256, 0, st>>>(n, ZW, gW, part);
        MLB_CHECK_LAUNCH(ctx, "lz_dot_kernel");
        std::vector<double> hp(g);
        MLB_CUDA(ctx, cudaMemcpyAsync(hp.data(), part, sizeof(double) * g, cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        for (double v : hp) quad += v;
        if (nprobe > 0 && (s = logdet_slq_dev(ctx, pr, nprobe, steps, &logdet)) != MLB_OK) break;
    } while (0);
    cudaStreamSynchronize(st);
    tmp.release();
    if (s != MLB_OK) return s;
    const double kLog2Pi = 1.8378770664093453;   // log(2 pi)
    out3[0] = -0.5 * ((double)n * kLog2Pi + logdet + quad);
    out3[1] = logdet;
    out3[2] = quad;
    return MLB_OK;
}
