// Diagonally preconditioned CG on C~_W g = Z_W (Sec. 5.2 remark on P_W,
// Sec. 6.2) and the trend step beta = (X^T X)^{-1} X^T (Z - C gamma)
// (eq. Spatial:eqn3).
//
// Vectors, inner products and updates are FP64.  The matrix-vector product is
// a warp-per-row pass over the row panels of C~_W (HBM bound).  Inner
// products are deterministic: every kernel writes per-block partial sums and
// a one-block kernel adds them in a fixed order.  The scalars of the
// iteration live on the device; the host only reads the "done" flag between
// chunks of iterations, which are replayed as a captured CUDA graph.
// Stopping test: ||r_k||_2 <= rtol ||Z_W||_2 on the unpreconditioned
// residual r_k = Z_W - C~_W g_k (remark closing Sec. 6.2).
#include <cmath>

#include "internal.h"

namespace mlb {

constexpr int kVecBlocks = 512;
constexpr int kSpmvBlocks = 1216;   // 8 x 152 SMs, grid-stride over rows

enum { ST_OK = 0, ST_BREAKDOWN = 1, ST_NOCONV = 2 };

__device__ double block_reduce(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += red[i];
    }
    __syncthreads();
    return s;   // valid in thread 0
}

// y = A x over the panels; optionally part[block] = sum_r x_r y_r.
__global__ void __launch_bounds__(256) spmv_kernel(Panels pan, const int64_t* __restrict__ wOff, int64_t nwav,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   double* __restrict__ part, const PcgState* st) {
    if (st && st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dotp = 0.0;
    for (int64_t r = warp; r < nwav; r += nwarp) {
        const int g = pan.rowCell[r];
        const int64_t i = r - wOff[g];
        const int n = pan.ncols[g];
        const double* v = pan.vals + pan.valOff[g] + i * n;
        const int* ci = pan.colidx + pan.colOff[g];
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += v[j] * x[ci[j]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            y[r] = acc;
            dotp += x[r] * acc;
        }
    }
    if (part) {
        const double s = block_reduce(dotp);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// x = 0, r = b, z = r / diag, p = z; partials of r.z and b.b
__global__ void pcg_init_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ diag,
                                double* x, double* r, double* z, double* p, double* part) {
    double rz = 0.0, bb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double zi = diag ? bi / diag[i] : bi;
        x[i] = 0.0;
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
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

__global__ void pcg_init_scalars(const double* part, PcgState* st) {
    if (threadIdx.x) return;
    double rz = 0.0, bb = 0.0;
    for (int i = 0; i < kVecBlocks; ++i) {
        rz += part[i];
        bb += part[kVecBlocks + i];
    }
    st->rz = rz;
    st->bb = bb;
    st->rr = bb;
    st->it = 0;
    st->status = ST_OK;
    st->done = bb == 0.0 ? 1 : 0;
}

__global__ void pcg_alpha_kernel(const double* part, int nparts, PcgState* st) {
    if (threadIdx.x || st->done) return;
    double pq = 0.0;
    for (int i = 0; i < nparts; ++i) pq += part[i];
    st->pq = pq;
    if (!(pq > 0.0)) {
        st->status = ST_BREAKDOWN;
        st->done = 1;
        return;
    }
    st->alpha = st->rz / pq;
}

__global__ void pcg_update_xr_kernel(int64_t n, const PcgState* st, const double* __restrict__ p,
                                     const double* __restrict__ q, const double* __restrict__ diag,
                                     double* x, double* r, double* z, double* part) {
    if (st->done) return;
    const double alpha = st->alpha;
    double rr = 0.0, rz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
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
}

__global__ void pcg_beta_kernel(const double* part, PcgState* st, double tol2, int maxit) {
    if (threadIdx.x || st->done) return;
    double rr = 0.0, rz = 0.0;
    for (int i = 0; i < kVecBlocks; ++i) {
        rr += part[i];
        rz += part[kVecBlocks + i];
    }
    st->it += 1;
    st->rr = rr;
    st->beta = rz / st->rz;
    st->rz = rz;
    if (rr <= tol2 * st->bb) {
        st->done = 1;
    } else if (st->it >= maxit) {
        st->status = ST_NOCONV;
        st->done = 1;
    }
}

__global__ void pcg_update_p_kernel(int64_t n, const PcgState* st, const double* __restrict__ z, double* p) {
    if (st->done) return;
    const double beta = st->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
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

mlb_status cw_matvec_dev(mlb_ctx* ctx, const double* u, double* out) {
    spmv_kernel<<<kSpmvBlocks, 256, 0, ctx->stream>>>(ctx->pan, ctx->cells.wOff, ctx->nwav, u, out, nullptr, nullptr);
    MLB_CHECK_LAUNCH(ctx, "spmv_kernel");
    return MLB_OK;
}

static void launch_iteration(mlb_ctx* ctx, double* x, double* r, double* z, double* p, double* q, double tol2) {
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->nwav;
    const double* diag = ctx->opts.precond ? ctx->diag : nullptr;
    spmv_kernel<<<kSpmvBlocks, 256, 0, st>>>(ctx->pan, ctx->cells.wOff, n, p, q, ctx->partial, ctx->pcg);
    pcg_alpha_kernel<<<1, 32, 0, st>>>(ctx->partial, kSpmvBlocks, ctx->pcg);
    pcg_update_xr_kernel<<<kVecBlocks, 256, 0, st>>>(n, ctx->pcg, p, q, diag, x, r, z, ctx->partial + kSpmvBlocks);
    pcg_beta_kernel<<<1, 32, 0, st>>>(ctx->partial + kSpmvBlocks, ctx->pcg, tol2, ctx->opts.pcg_maxit);
    pcg_update_p_kernel<<<kVecBlocks, 256, 0, st>>>(n, ctx->pcg, z, p);
}

mlb_status solve_dev(mlb_ctx* ctx, const double* Z_kd, mlb_info* info) {
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->nwav;
    double* b = ctx->vec;
    double* x = ctx->gW;
    double* r = ctx->vec + n;
    double* z = ctx->vec + 2 * n;
    double* p = ctx->vec + 3 * n;
    double* q = ctx->vec + 4 * n;
    mlb_status s = apply_W_dev(ctx, Z_kd, b);
    if (s != MLB_OK) return s;
    const double* diag = ctx->opts.precond ? ctx->diag : nullptr;
    pcg_init_kernel<<<kVecBlocks, 256, 0, st>>>(n, b, diag, x, r, z, p, ctx->partial);
    pcg_init_scalars<<<1, 32, 0, st>>>(ctx->partial, ctx->pcg);
    MLB_CHECK_LAUNCH(ctx, "pcg_init");
    const double tol2 = ctx->opts.pcg_rtol * ctx->opts.pcg_rtol;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    // one chunk of iterations as a CUDA graph, replayed until done
    const int chunk = 8;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MLB_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) launch_iteration(ctx, x, r, z, p, q, tol2);
    MLB_CUDA(ctx, cudaStreamEndCapture(st, &graph));
    MLB_CUDA(ctx, cudaGraphInstantiate(&exec, graph, 0));
    PcgState hs{};
    for (;;) {
        MLB_CUDA(ctx, cudaGraphLaunch(exec, st));
        ctx->launches += 5 * chunk;
        MLB_CUDA(ctx, cudaMemcpyAsync(&hs, ctx->pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        if (hs.done) break;
    }
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    mlb_info& I = ctx->last_info;
    I.iterations = hs.it;
    I.converged = hs.status == ST_OK && hs.done;
    I.rel_residual = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    I.nnz = ctx->pan.nnz;
    I.nnz_unique = ctx->pan.nnzUnique;
    I.blocks = ctx->pan.blocks;
    I.ms_assemble = ctx->ms_assemble;
    I.ms_pcg = ms;
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
    cudaEventElapsedTime(&ms, b0, b1);
    cudaEventDestroy(b0);
    cudaEventDestroy(b1);
    I.ms_beta = ms;
    I.launches = ctx->launches;
    if (info) *info = I;
    if (hs.status == ST_BREAKDOWN) return fail(ctx, MLB_EBREAKDOWN, "PCG breakdown: p^T C~_W p <= 0");
    if (hs.status == ST_NOCONV) return fail(ctx, MLB_ENOCONV, "PCG did not reach pcg_rtol within pcg_maxit");
    return MLB_OK;
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

}  // namespace mlb
