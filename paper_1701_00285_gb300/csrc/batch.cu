// Many independent BLUP problems in one call (the batched workload: problems
// of different sizes, dimensions and covariance parameters).
//
// Every problem gets its own context (basis, assembly, vectors).  The setup
// phases -- kd-tree and basis, assembly of C~_W, Z_W = W Z -- and the closing
// phases -- gamma = W^T gamma_W, the trend step, predictions -- run the
// single-problem kernels on a pool of streams driven by host threads.  The PCG
// phase, where a per-problem loop would be bound by kernel launches (five
// launches per iteration on systems of a few thousand unknowns), is one
// persistent launch: one CTA per problem runs its whole diagonally
// preconditioned CG (Sec. 5.2 remark, Sec. 6.2) with block-level reductions
// only -- no CTA waits for another.  Problems with more than kCtaRows
// unknowns would hold one SM for many iterations of a product that wants
// the whole GPU; they run the single-problem PCG (full-grid product, CUDA
// graph chunks) on the stream pool while the persistent launch runs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace mlb {

// largest system solved by one CTA of the persistent launch
constexpr int kCtaRows = 1024;

struct BatchPcgProblem {
    const double* vals64;      // panel values (FP64 path) or nullptr
    const float* vals32;       // panel values (mixed path) or nullptr
    const int* colidx;
    const int* ncols;
    const int64_t* valOff;
    const int64_t* colOff;
    const int* rowCell;
    const int64_t* wOff;
    const double* diag;        // nullptr: no preconditioner
    const double* b;
    double* x;
    double* r;
    double* z;
    double* p;
    double* q;
    int64_t n;
    double tol2;
    int maxit;
    int pad;
    PcgState* st;
};

__device__ double cta_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// q = A p by warp-per-row over the problem's panels; returns p.q (all
// threads).  p is staged in shared memory first (n <= kCtaRows), so the
// column gather reads shared memory and only the values and column indices
// stream from global memory, four at a time (panel rows start 16-byte
// aligned and hold a multiple of 4 columns).
__device__ double cta_spmv(const BatchPcgProblem& P, const double* __restrict__ pv, double* __restrict__ q,
                           double* xs, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t i = threadIdx.x; i < P.n; i += blockDim.x) xs[i] = pv[i];
    __syncthreads();
    double dot = 0.0;
    for (int64_t r = warp; r < P.n; r += nw) {
        const int g = P.rowCell[r];
        const int64_t i = r - P.wOff[g];
        const int n = P.ncols[g];
        const int* ci = P.colidx + P.colOff[g];
        double acc = 0.0;
        if (P.vals32) {
            // four 16-byte value and index loads per lane in flight before any is used
            const float* v = P.vals32 + P.valOff[g] + i * n;
            for (int j0 = 4 * lane; j0 < n; j0 += 512) {
                float4 a[4];
                int4 c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + 128 * u;
                    if (j < n) {
                        a[u] = *reinterpret_cast<const float4*>(v + j);
                        c[u] = *reinterpret_cast<const int4*>(ci + j);
                    } else {
                        a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        c[u] = make_int4(0, 0, 0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    acc += (double)a[u].x * xs[c[u].x] + (double)a[u].y * xs[c[u].y] + (double)a[u].z * xs[c[u].z] +
                           (double)a[u].w * xs[c[u].w];
            }
        } else {
            const double* v = P.vals64 + P.valOff[g] + i * n;
            for (int j = 4 * lane; j < n; j += 128) {
                const double2 a = *reinterpret_cast<const double2*>(v + j);
                const double2 b = *reinterpret_cast<const double2*>(v + j + 2);
                const int4 c = *reinterpret_cast<const int4*>(ci + j);
                acc += a.x * xs[c.x] + a.y * xs[c.y] + b.x * xs[c.z] + b.y * xs[c.w];
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            q[r] = acc;
            dot += xs[r] * acc;
        }
    }
    return cta_sum(dot, red);
}

// One CTA per problem; the iteration matches pcg_run: x0 = 0, stop when
// ||r_k||^2 <= tol^2 ||b||^2 on the recursive unpreconditioned residual.
__global__ void __launch_bounds__(512) batch_pcg_kernel(const BatchPcgProblem* __restrict__ probs) {
    __shared__ double red[32];
    __shared__ double xs[kCtaRows];
    const BatchPcgProblem P = probs[blockIdx.x];
    const int64_t n = P.n;
    double rz = 0.0, bb = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double bi = P.b[i];
        const double zi = P.diag ? bi / P.diag[i] : bi;
        P.x[i] = 0.0;
        P.r[i] = bi;
        P.z[i] = zi;
        P.p[i] = zi;
        rz += bi * zi;
        bb += bi * bi;
    }
    rz = cta_sum(rz, red);
    bb = cta_sum(bb, red);
    int it = 0, status = 0;
    double rr = bb;
    if (bb > 0.0) {
        while (true) {
            __syncthreads();
            const double pq = cta_spmv(P, P.p, P.q, xs, red);
            if (!(pq > 0.0)) {
                status = 1;
                break;
            }
            const double alpha = rz / pq;
            double rrl = 0.0, rzl = 0.0;
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                P.x[i] += alpha * P.p[i];
                const double ri = P.r[i] - alpha * P.q[i];
                P.r[i] = ri;
                const double zi = P.diag ? ri / P.diag[i] : ri;
                P.z[i] = zi;
                rrl += ri * ri;
                rzl += ri * zi;
            }
            rr = cta_sum(rrl, red);
            const double rzn = cta_sum(rzl, red);
            ++it;
            if (rr <= P.tol2 * bb) break;
            if (it >= P.maxit) {
                status = 2;
                break;
            }
            const double beta = rzn / rz;
            rz = rzn;
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) P.p[i] = P.z[i] + beta * P.p[i];
        }
    }
    if (threadIdx.x == 0) {
        P.st->it = it;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->status = status;
        P.st->done = 1;
    }
}

}  // namespace mlb

using namespace mlb;

namespace {

thread_local std::string g_batch_err;
thread_local double g_batch_phase_ms[3] = {0.0, 0.0, 0.0};
thread_local int64_t g_batch_launches = 0;

double ms_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

struct Job {
    mlb_batch_problem* prob;
    mlb_ctx* ctx = nullptr;
    mlb_status status = MLB_OK;
    double* Zd = nullptr;     // device Z (caller order) and kd order
};

mlb_status setup_one(Job& j, const mlb_opts& o, cudaStream_t st) {
    mlb_batch_problem& P = *j.prob;
    mlb_status s = mlb_create(&o, &j.ctx);
    if (s != MLB_OK) return s;
    mlb_set_stream(j.ctx, st);
    s = mlb_build_basis(j.ctx, P.points, P.n, P.d, P.w);
    if (s != MLB_OK) return s;
    // the persistent launch reads the row panels of the systems it solves
    j.ctx->allow_sym = j.ctx->nwav > kCtaRows;
    s = mlb_assemble(j.ctx, &P.theta, P.tau_factor);
    if (s != MLB_OK) return s;
    mlb_ctx* c = j.ctx;
    double* Zu = c->vec + 7 * c->N;
    double* Zkd = c->vec + 6 * c->N;
    MLB_CUDA(c, cudaMemcpyAsync(Zu, P.Z, sizeof(double) * c->N, cudaMemcpyHostToDevice, st));
    s = gather_kd(c, Zu, Zkd);
    if (s != MLB_OK) return s;
    return apply_W_dev(c, Zkd, c->vec);
}

mlb_status finish_one(Job& j) {
    mlb_ctx* c = j.ctx;
    mlb_batch_problem& P = *j.prob;
    PcgState hs{};
    MLB_CUDA(c, cudaMemcpyAsync(&hs, c->pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, c->stream));
    MLB_CUDA(c, cudaStreamSynchronize(c->stream));
    P.iterations = hs.it;
    mlb_status s = apply_Wt_dev(c, c->gW, c->gamma);
    if (s != MLB_OK) return s;
    s = trend_dev(c, c->vec + 6 * c->N);
    if (s != MLB_OK) return s;
    c->state = 3;
    if (P.beta) {
        MLB_CUDA(c, cudaMemcpyAsync(P.beta, c->beta, sizeof(double) * c->p, cudaMemcpyDeviceToHost, c->stream));
    }
    if (P.m > 0) s = mlb_predict(c, P.targets, P.m, P.yhat);
    if (s != MLB_OK) return s;
    if (hs.status == 1) return fail(c, MLB_EBREAKDOWN, "PCG breakdown");
    if (hs.status == 2) return fail(c, MLB_ENOCONV, "PCG not converged");
    return MLB_OK;
}

// f(job, thread) over the listed jobs that are still OK, on `threads` host threads
template <typename F>
void run_listed(std::vector<Job>& jobs, const std::vector<int>& list, int threads, F f) {
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t]() {
            for (int k = next.fetch_add(1); k < (int)list.size(); k = next.fetch_add(1)) {
                Job& j = jobs[list[k]];
                if (j.status == MLB_OK) j.status = f(j, t);
            }
        });
    for (auto& th : pool) th.join();
}

template <typename F>
void run_parallel(std::vector<Job>& jobs, int threads, F f) {
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t]() {
            for (int i = next.fetch_add(1); i < (int)jobs.size(); i = next.fetch_add(1))
                if (jobs[i].status == MLB_OK) jobs[i].status = f(jobs[i], t);
        });
    for (auto& th : pool) th.join();
}

}  // namespace

extern "C" const char* mlb_batch_last_error(void) { return g_batch_err.c_str(); }

extern "C" int64_t mlb_batch_last_launches(void) { return g_batch_launches; }

extern "C" void mlb_batch_last_phase_ms(double* out) {
    if (out)
        for (int i = 0; i < 3; ++i) out[i] = g_batch_phase_ms[i];
}

extern "C" mlb_status mlb_batch_solve(const mlb_opts* opts, mlb_batch_problem* probs, int count, int host_threads,
                                      double* ms_out) {
    g_batch_err.clear();
    if (!probs || count < 1) return MLB_EINVAL;
    mlb_opts o;
    if (opts) o = *opts;
    else mlb_default_opts(&o);
    if (o.matrix_free) return MLB_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    if (cudaSetDevice(o.device) != cudaSuccess) return MLB_ECUDA;
    const int threads = std::max(1, std::min(host_threads > 0 ? host_threads : 8, 64));
    std::vector<cudaStream_t> streams(threads);
    for (auto& s : streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return MLB_ECUDA;
    std::vector<Job> jobs(count);
    for (int i = 0; i < count; ++i) {
        jobs[i].prob = &probs[i];
        probs[i].status = MLB_OK;
        probs[i].iterations = 0;
    }
    // phase 1: basis, assembly, Z_W
    for (double& v : g_batch_phase_ms) v = 0.0;
    g_batch_launches = 0;
    auto tp = std::chrono::steady_clock::now();
    run_parallel(jobs, threads, [&](Job& j, int t) {
        cudaSetDevice(o.device);
        return setup_one(j, o, streams[t]);
    });
    for (auto& s : streams) cudaStreamSynchronize(s);
    g_batch_phase_ms[0] = ms_since(tp);
    tp = std::chrono::steady_clock::now();
    // phase 2: the small systems in one persistent launch (largest first, so
    // the longest CTAs start first), the large ones on the stream pool
    std::vector<int> order, big;
    for (int i = 0; i < count; ++i)
        if (jobs[i].status == MLB_OK) (jobs[i].ctx->nwav > kCtaRows ? big : order).push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].ctx->nwav > jobs[b].ctx->nwav; });
    std::vector<BatchPcgProblem> hp;
    for (int i : order) {
        mlb_ctx* c = jobs[i].ctx;
        BatchPcgProblem b{};
        b.vals64 = c->pan.vals32 ? nullptr : c->pan.vals;
        b.vals32 = c->pan.vals32;
        b.colidx = c->pan.colidx;
        b.ncols = c->pan.ncols;
        b.valOff = c->pan.valOff;
        b.colOff = c->pan.colOff;
        b.rowCell = c->pan.rowCell;
        b.wOff = c->cells.wOff;
        b.diag = o.precond ? c->diag : nullptr;
        b.n = c->nwav;
        b.b = c->vec;
        b.x = c->gW;
        b.r = c->vec + b.n;
        b.z = c->vec + 2 * b.n;
        b.p = c->vec + 3 * b.n;
        b.q = c->vec + 4 * b.n;
        b.tol2 = o.pcg_rtol * o.pcg_rtol;
        b.maxit = o.pcg_maxit;
        b.st = c->pcg;
        hp.push_back(b);
    }
    mlb_status first = MLB_OK;
    BatchPcgProblem* dp = nullptr;
    cudaStream_t ps = nullptr;
    if (!hp.empty()) {
        if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&dp, sizeof(BatchPcgProblem) * hp.size()) != cudaSuccess) {
            first = MLB_ENOMEM;
            g_batch_err = "stream or problem table for the persistent PCG";
        }
        if (first == MLB_OK) {
            cudaError_t e = cudaMemcpyAsync(dp, hp.data(), sizeof(BatchPcgProblem) * hp.size(),
                                            cudaMemcpyHostToDevice, ps);
            if (e == cudaSuccess) {
                batch_pcg_kernel<<<(unsigned)hp.size(), 512, 0, ps>>>(dp);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) {
                first = MLB_ECUDA;
                g_batch_err = std::string("batch_pcg_kernel: ") + cudaGetErrorString(e);
            }
        }
    }
    if (first == MLB_OK && !big.empty())
        run_listed(jobs, big, threads, [&](Job& j, int t) {
            cudaSetDevice(o.device);
            mlb_set_stream(j.ctx, streams[t]);
            mlb_info inf{};
            const mlb_status s = pcg_run(j.ctx, j.ctx->vec, j.ctx->gW, &inf);
            // breakdown and non-convergence are reported per problem by finish_one
            return (s == MLB_EBREAKDOWN || s == MLB_ENOCONV) ? MLB_OK : s;
        });
    if (ps) {
        const cudaError_t e = cudaStreamSynchronize(ps);
        if (e != cudaSuccess && first == MLB_OK) {
            first = MLB_ECUDA;
            g_batch_err = std::string("batch_pcg_kernel: ") + cudaGetErrorString(e);
        }
        cudaStreamDestroy(ps);
    }
    if (dp) cudaFree(dp);
    const int64_t persistent = (first == MLB_OK && !hp.empty()) ? 1 : 0;
    g_batch_phase_ms[1] = ms_since(tp);
    tp = std::chrono::steady_clock::now();
    // phase 3: gamma, trend, predictions
    if (first == MLB_OK)
        run_parallel(jobs, threads, [&](Job& j, int) {
            cudaSetDevice(o.device);
            return finish_one(j);
        });
    g_batch_launches = persistent;
    for (int i = 0; i < count; ++i) {
        if (jobs[i].ctx) g_batch_launches += jobs[i].ctx->launches;
        probs[i].status = jobs[i].status;
        if (first == MLB_OK && jobs[i].status != MLB_OK) {
            first = jobs[i].status;
            g_batch_err = "problem " + std::to_string(i) + ": " + (jobs[i].ctx ? jobs[i].ctx->err : std::string("context"));
        }
        if (jobs[i].ctx) mlb_destroy(jobs[i].ctx);
    }
    for (auto& s : streams) cudaStreamDestroy(s);
    g_batch_phase_ms[2] = ms_since(tp);
    if (ms_out)
        *ms_out = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return first;
}
