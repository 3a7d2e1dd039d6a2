// C ABI of libmlblup: context, call order, argument checks, the kd-tree
// (Algorithms 1-3) and the cell tables, and the host <-> device copies of the
// host-pointer entry points.  Every numerical step runs in the kernels of
// basis.cu, assemble.cu, solve.cu and ksum.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <numeric>

#include "internal.h"
#include "matern.cuh"

namespace mlb {

void Arena::release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
}

mlb_status fail(mlb_ctx* ctx, mlb_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

mlb_status cuda_fail(mlb_ctx* ctx, cudaError_t e, const char* where) {
    cudaGetLastError();   // a non-sticky error must not be reported again by the next launch check
    return fail(ctx, e == cudaErrorMemoryAllocation ? MLB_ENOMEM : MLB_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

int max_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 48 * 1024;
}

mlb_status allow_max_dynamic_smem(mlb_ctx* ctx, const void* func, const char* name) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem_optin() - (int)fa.sharedSizeBytes);
    return e == cudaSuccess ? MLB_OK : cuda_fail(ctx, e, name);
}

void dfree(mlb_ctx* ctx, Arena& a, void* p) {
    if (!p) return;
    for (size_t i = 0; i < a.ptrs.size(); ++i)
        if (a.ptrs[i] == p) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(p);
            a.ptrs.erase(a.ptrs.begin() + i);
            return;
        }
}

void* dalloc(mlb_ctx* ctx, Arena& a, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 8;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
        return nullptr;
    }
    a.ptrs.push_back(p);
    return p;
}

// Total-degree exponents, graded, lexicographically decreasing within a degree.
static void exponents(int d, int w, std::vector<int>& out) {
    std::vector<int> cur(d, 0);
    for (int deg = 0; deg <= w; ++deg) {
        // recursive enumeration: first coordinate from deg down to 0
        std::vector<int> stack;
        std::function<void(int, int)> rec = [&](int k, int rem) {
            if (k == d - 1) {
                cur[k] = rem;
                out.insert(out.end(), cur.begin(), cur.end());
                return;
            }
            for (int a = rem; a >= 0; --a) {
                cur[k] = a;
                rec(k + 1, rem - a);
            }
        };
        rec(0, deg);
    }
}

static int depth_for(int64_t N, int n0) {
    int t = 0;
    while ((N + (1LL << t) - 1) / (1LL << t) > n0) ++t;
    return t;
}

// Algorithms 1-3: level by level; a cell splits at the median of its points
// ordered by (coordinate on the axis of largest population variance, caller
// index); the first floor(s/2) go left.  Every cell splits down to the common
// depth t at which all cells hold at most n0 points.
static void build_tree_host(const double* pts, int64_t N, int d, int n0, int t, std::vector<int>& perm,
                            std::vector<int>& beg, std::vector<int>& end) {
    perm.resize(N);
    std::iota(perm.begin(), perm.end(), 0);
    const int ncell = (1 << (t + 1)) - 1;
    beg.assign(ncell, 0);
    end.assign(ncell, 0);
    beg[0] = 0;
    end[0] = (int)N;
    std::vector<double> mean(d), var(d);
    for (int l = 0; l < t; ++l) {
        for (int k = 0; k < (1 << l); ++k) {
            const int g = (1 << l) - 1 + k;
            const int b = beg[g], e = end[g], n = e - b;
            for (int c = 0; c < d; ++c) {
                double s = 0.0;
                for (int i = b; i < e; ++i) s += pts[(int64_t)perm[i] * d + c];
                mean[c] = s / n;
                double v = 0.0;
                for (int i = b; i < e; ++i) {
                    const double df = pts[(int64_t)perm[i] * d + c] - mean[c];
                    v += df * df;
                }
                var[c] = v / n;
            }
            int axis = 0;
            for (int c = 1; c < d; ++c)
                if (var[c] > var[axis]) axis = c;
            std::sort(perm.begin() + b, perm.begin() + e, [&](int i, int j) {
                const double xi = pts[(int64_t)i * d + axis], xj = pts[(int64_t)j * d + axis];
                return xi < xj || (xi == xj && i < j);
            });
            const int h = n / 2;
            beg[2 * g + 1] = b;
            end[2 * g + 1] = b + h;
            beg[2 * g + 2] = b + h;
            end[2 * g + 2] = e;
        }
    }
}

// Helper for the host-pointer inspection calls: H2D input, device op, D2H output.
template <typename F>
mlb_status host_roundtrip(mlb_ctx* ctx, const double* in, int64_t nin, double* out, int64_t nout, F op) {
    cudaSetDevice(ctx->opts.device);
    double *din = nullptr, *dout = nullptr;
    MLB_CUDA(ctx, cudaMalloc(&din, sizeof(double) * std::max<int64_t>(nin, 1)));
    if (cudaMalloc(&dout, sizeof(double) * std::max<int64_t>(nout, 1)) != cudaSuccess) {
        cudaFree(din);
        return fail(ctx, MLB_ENOMEM, "cudaMalloc failed");
    }
    mlb_status s = MLB_OK;
    if (nin && cudaMemcpyAsync(din, in, sizeof(double) * nin, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        s = fail(ctx, MLB_ECUDA, "copy failed");
    if (s == MLB_OK) s = op(din, dout);
    if (s == MLB_OK) {
        cudaError_t e = cudaMemcpyAsync(out, dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "copy back");
    }
    cudaStreamSynchronize(ctx->stream);   // an error path may leave work queued on the buffers
    cudaFree(din);
    cudaFree(dout);
    return s;
}

}  // namespace mlb

using namespace mlb;

extern "C" {

void mlb_default_opts(mlb_opts* o) {
    if (!o) return;
    o->precision = MLB_FP64;
    o->leaf_size = 64;
    o->pcg_rtol = 1e-10;
    o->pcg_maxit = 20000;
    o->precond = 1;
    o->matrix_free = 0;
    o->device = 0;
}

const char* mlb_status_string(mlb_status s) {
    switch (s) {
        case MLB_OK: return "ok";
        case MLB_EINVAL: return "invalid argument";
        case MLB_ERANK: return "rank deficient";
        case MLB_ENOCONV: return "PCG not converged";
        case MLB_EBREAKDOWN: return "PCG breakdown";
        case MLB_ENOMEM: return "out of device memory";
        case MLB_ECUDA: return "CUDA error";
        case MLB_ETIMEOUT: return "device wait timed out";
        case MLB_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char* mlb_last_error(const mlb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mlb_status mlb_create(const mlb_opts* opts, mlb_ctx** out) {
    if (!out) return MLB_EINVAL;
    *out = nullptr;
    mlb_opts o;
    if (opts) o = *opts;
    else mlb_default_opts(&o);
    if (o.leaf_size < 1 || o.pcg_maxit < 1 || !(o.pcg_rtol > 0) || (o.precision != MLB_FP64 && o.precision != MLB_MIXED))
        return MLB_EINVAL;
    if (cudaSetDevice(o.device) != cudaSuccess) {
        cudaGetLastError();
        return MLB_ECUDA;
    }
    mlb_ctx* ctx = new mlb_ctx();
    ctx->opts = o;
    if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return MLB_ECUDA;
    }
    ctx->stream = ctx->own_stream;
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, o.device);
    *out = ctx;
    return MLB_OK;
}

void mlb_destroy(mlb_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->opts.device);
    cudaStreamSynchronize(ctx->stream);
    ctx->arena_solve.release();
    ctx->arena_asm.release();
    ctx->arena_basis.release();
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

mlb_status mlb_set_stream(mlb_ctx* ctx, void* s) {
    if (!ctx) return MLB_EINVAL;
    ctx->stream = s ? (cudaStream_t)s : ctx->own_stream;
    return MLB_OK;
}

static mlb_status build_basis_host(mlb_ctx* ctx, const double* pts, int64_t N, int d, int w) {
    cudaSetDevice(ctx->opts.device);
    if (d < 1 || d > kMaxDim || w < 0 || N < 2 || N > (1LL << 30))
        return fail(ctx, MLB_EINVAL, "need 1 <= d <= 16, w >= 0, 2 <= N < 2^30");
    for (int64_t i = 0; i < N * d; ++i)
        if (!std::isfinite(pts[i])) return fail(ctx, MLB_EINVAL, "non-finite point coordinate");
    std::vector<int> ex;
    exponents(d, w, ex);
    const int p = (int)(ex.size() / d);
    if (p > 128) return fail(ctx, MLB_EINVAL, "p = binom(d+w, w) must be <= 128");
    if (N <= p) return fail(ctx, MLB_EINVAL, "need N > p");
    cudaStreamSynchronize(ctx->stream);
    ctx->arena_solve.release();
    ctx->arena_asm.release();
    ctx->arena_basis.release();
    ctx->state = 0;
    ctx->N = N;
    ctx->d = d;
    ctx->w = w;
    ctx->p = p;
    const int n0 = ctx->opts.leaf_size;
    const int t = depth_for(N, n0);
    if (t > 20) return fail(ctx, MLB_EINVAL, "tree deeper than 20 levels");
    ctx->t = t;
    const int ncell = (1 << (t + 1)) - 1;
    ctx->ncell = ncell;
    std::vector<int> beg, end;
    build_tree_host(pts, N, d, n0, t, ctx->hperm, beg, end);
    for (int c = 0; c < d; ++c) {
        ctx->box_lo[c] = INFINITY;
        ctx->box_hi[c] = -INFINITY;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) {
            ctx->box_lo[c] = std::min(ctx->box_lo[c], pts[i * d + c]);
            ctx->box_hi[c] = std::max(ctx->box_hi[c], pts[i * d + c]);
        }
    // cell tables
    auto& H = ctx->hcells;
    H.assign(ncell, HostCell{});
    ctx->sumA.assign(t + 1, 0);
    ctx->sumK.assign(t + 1, 0);
    for (int l = t; l >= 0; --l) {
        for (int k = 0; k < (1 << l); ++k) {
            const int g = (1 << l) - 1 + k;
            HostCell& c = H[g];
            c.beg = beg[g];
            c.end = end[g];
            c.s = l == t ? c.end - c.beg : H[2 * g + 1].a + H[2 * g + 2].a;
            c.a = std::min(p, c.s);
            c.k = c.s - c.a;
            c.sOff = ctx->sumA[l];
            c.wLoc = ctx->sumK[l];
            ctx->sumA[l] += c.a;
            ctx->sumK[l] += c.k;
        }
    }
    if (H[0].a != p) return fail(ctx, MLB_ERANK, "fewer than p scaling vectors reach the root");
    ctx->levelBase.assign(t + 1, 0);
    for (int l = t - 1; l >= 0; --l) ctx->levelBase[l] = ctx->levelBase[l + 1] + ctx->sumK[l + 1];
    ctx->sbase.assign(t + 2, 0);
    for (int l = 0; l <= t; ++l) ctx->sbase[l + 1] = ctx->sbase[l] + ctx->sumA[l];
    int64_t vo = 0, ro = 0;
    for (int g = 0; g < ncell; ++g) {
        int l = 0;
        while ((1 << (l + 1)) - 1 <= g) ++l;
        H[g].vOff = vo;
        H[g].rOff = ro;
        H[g].wOff = ctx->levelBase[l] + H[g].wLoc;
        vo += (int64_t)H[g].s * H[g].s;
        ro += (int64_t)H[g].a * p;
    }
    ctx->nwav = N - p;
    std::vector<int> rowCell(ctx->nwav);
    for (int g = 0; g < ncell; ++g)
        for (int i = 0; i < H[g].k; ++i) rowCell[H[g].wOff + i] = g;
    // device buffers
    Arena& A = ctx->arena_basis;
    std::vector<double> xs(N * d);
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) xs[i * d + c] = pts[(int64_t)ctx->hperm[i] * d + c];
    ctx->xs = (double*)dalloc(ctx, A, sizeof(double) * N * d);
    ctx->xs32 = (float*)dalloc(ctx, A, sizeof(float) * N * d);
    ctx->xl32 = (float*)dalloc(ctx, A, sizeof(float) * N * d);
    ctx->xs32lo = (float*)dalloc(ctx, A, sizeof(float) * N * d);
    ctx->xl32lo = (float*)dalloc(ctx, A, sizeof(float) * N * d);
    ctx->leafctr = (double*)dalloc(ctx, A, sizeof(double) * ncell * d);
    ctx->perm = (int*)dalloc(ctx, A, sizeof(int) * N);
    ctx->alpha = (int*)dalloc(ctx, A, sizeof(int) * p * d);
    ctx->X = (double*)dalloc(ctx, A, sizeof(double) * N * p);
    ctx->XtXf = (double*)dalloc(ctx, A, sizeof(double) * p * p);
    ctx->V = (double*)dalloc(ctx, A, sizeof(double) * vo);
    ctx->R = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(ro, 1));
    ctx->sbuf = (double*)dalloc(ctx, A, sizeof(double) * ctx->sbase[t + 1]);
    ctx->flag = (int*)dalloc(ctx, A, sizeof(int) * 4);
    ctx->pan.rowCell = (int*)dalloc(ctx, A, sizeof(int) * ctx->nwav);
    ctx->gW = (double*)dalloc(ctx, A, sizeof(double) * ctx->nwav);
    ctx->gamma = (double*)dalloc(ctx, A, sizeof(double) * N);
    ctx->beta = (double*)dalloc(ctx, A, sizeof(double) * p);
    ctx->vec = (double*)dalloc(ctx, A, sizeof(double) * 10 * N);
    ctx->ksum_part_cap = std::max<int64_t>(8 * N, 1 << 16);
    ctx->ksum_part = (double*)dalloc(ctx, A, sizeof(double) * ctx->ksum_part_cap);
    ctx->partial = (double*)dalloc(ctx, A, sizeof(double) * (max_work_items(ncell, N) + 16384));
    ctx->pcg = (PcgState*)dalloc(ctx, A, sizeof(PcgState));
    CellTables& C = ctx->cells;
    C.beg = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    C.end = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    C.s = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    C.a = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    C.k = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    C.vOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    C.rOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    C.wOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    C.sOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    C.wLoc = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    C.lo = (double*)dalloc(ctx, A, sizeof(double) * ncell * d);
    C.hi = (double*)dalloc(ctx, A, sizeof(double) * ncell * d);
    C.diam = (double*)dalloc(ctx, A, sizeof(double) * ncell);
    {
        const void* need[] = {ctx->xs, ctx->xs32, ctx->xl32, ctx->xs32lo, ctx->xl32lo, ctx->leafctr, ctx->perm, ctx->alpha, ctx->X, ctx->XtXf, ctx->V, ctx->R, ctx->sbuf,
                              ctx->flag, ctx->pan.rowCell, ctx->gW, ctx->gamma, ctx->beta, ctx->vec,
                              ctx->partial, ctx->ksum_part, ctx->pcg, C.beg, C.end, C.s, C.a, C.k, C.vOff, C.rOff, C.wOff,
                              C.sOff, C.wLoc, C.lo, C.hi, C.diam};
        for (const void* q : need)
            if (!q) return fail(ctx, MLB_ENOMEM, ctx->err);
    }
    std::vector<int> ib(ncell), ie(ncell), is(ncell), ia(ncell), ik(ncell);
    std::vector<int64_t> vOff(ncell), rOff(ncell), wOff(ncell), sOff(ncell), wLoc(ncell);
    std::vector<double> lo((size_t)ncell * d), hi((size_t)ncell * d), diam(ncell);
    for (int g = 0; g < ncell; ++g) {
        const HostCell& c = H[g];
        ib[g] = c.beg; ie[g] = c.end; is[g] = c.s; ia[g] = c.a; ik[g] = c.k;
        vOff[g] = c.vOff; rOff[g] = c.rOff; wOff[g] = c.wOff; sOff[g] = c.sOff; wLoc[g] = c.wLoc;
        for (int q = 0; q < d; ++q) {
            double mn = INFINITY, mx = -INFINITY;
            for (int i = c.beg; i < c.end; ++i) {
                mn = std::min(mn, xs[(int64_t)i * d + q]);
                mx = std::max(mx, xs[(int64_t)i * d + q]);
            }
            lo[(size_t)g * d + q] = mn;
            hi[(size_t)g * d + q] = mx;
        }
        // diagonal accumulated axis by axis (no contraction: -ffp-contract=off)
        double acc = 0.0;
        for (int q = 0; q < d; ++q) {
            const double span = hi[(size_t)g * d + q] - lo[(size_t)g * d + q];
            acc = acc + span * span;
        }
        diam[g] = std::sqrt(acc);
    }
    // tau_{i,j} = c sqrt(Dbar_i Dbar_j): every cell carries its level's mean
    // diagonal, summed cell by cell in order
    for (int l = 0; l <= t; ++l) {
        double acc = 0.0;
        const int first = (1 << l) - 1, n = 1 << l;
        for (int k = 0; k < n; ++k) acc = acc + diam[first + k];
        const double mean = acc / (double)n;
        for (int k = 0; k < n; ++k) diam[first + k] = mean;
    }
    // FP32 coordinates of the mixed path: offsets from the data box centre, and
    // offsets from the box centre of the point's leaf
    std::vector<float> x32((size_t)N * d), xl((size_t)N * d), x32lo((size_t)N * d), xllo((size_t)N * d);
    std::vector<double> ctr((size_t)ncell * d);
    for (int g = 0; g < ncell; ++g)
        for (int q = 0; q < d; ++q) ctr[(size_t)g * d + q] = 0.5 * (lo[(size_t)g * d + q] + hi[(size_t)g * d + q]);
    for (int k = 0; k < (1 << t); ++k) {
        const int g = (1 << t) - 1 + k;
        for (int i = H[g].beg; i < H[g].end; ++i)
            for (int q = 0; q < d; ++q) {
                const double v = xs[(size_t)i * d + q];
                const double og = v - 0.5 * (ctx->box_lo[q] + ctx->box_hi[q]);
                const double ol = v - ctr[(size_t)g * d + q];
                x32[(size_t)i * d + q] = (float)og;
                x32lo[(size_t)i * d + q] = (float)(og - (double)(float)og);
                xl[(size_t)i * d + q] = (float)ol;
                xllo[(size_t)i * d + q] = (float)(ol - (double)(float)ol);
            }
    }
    cudaStream_t st = ctx->stream;
#define UP(dst, src, n) MLB_CUDA(ctx, cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st))
    UP(ctx->xs32, x32.data(), sizeof(float) * N * d);
    UP(ctx->xl32, xl.data(), sizeof(float) * N * d);
    UP(ctx->xs32lo, x32lo.data(), sizeof(float) * N * d);
    UP(ctx->xl32lo, xllo.data(), sizeof(float) * N * d);
    UP(ctx->leafctr, ctr.data(), sizeof(double) * ncell * d);
    UP(ctx->xs, xs.data(), sizeof(double) * N * d);
    UP(ctx->perm, ctx->hperm.data(), sizeof(int) * N);
    UP(ctx->alpha, ex.data(), sizeof(int) * p * d);
    UP(ctx->pan.rowCell, rowCell.data(), sizeof(int) * ctx->nwav);
    UP(C.beg, ib.data(), sizeof(int) * ncell);
    UP(C.end, ie.data(), sizeof(int) * ncell);
    UP(C.s, is.data(), sizeof(int) * ncell);
    UP(C.a, ia.data(), sizeof(int) * ncell);
    UP(C.k, ik.data(), sizeof(int) * ncell);
    UP(C.vOff, vOff.data(), sizeof(int64_t) * ncell);
    UP(C.rOff, rOff.data(), sizeof(int64_t) * ncell);
    UP(C.wOff, wOff.data(), sizeof(int64_t) * ncell);
    UP(C.sOff, sOff.data(), sizeof(int64_t) * ncell);
    UP(C.wLoc, wLoc.data(), sizeof(int64_t) * ncell);
    UP(C.lo, lo.data(), sizeof(double) * ncell * d);
    UP(C.hi, hi.data(), sizeof(double) * ncell * d);
    UP(C.diam, diam.data(), sizeof(double) * ncell);
#undef UP
    MLB_CUDA(ctx, cudaMemsetAsync(ctx->flag, 0, sizeof(int) * 4, st));
    mlb_status s = build_design(ctx);
    if (s != MLB_OK) return s;
    s = build_factors(ctx);
    if (s != MLB_OK) return s;
    int hflag[4] = {0, 0, 0, 0};
    MLB_CUDA(ctx, cudaMemcpyAsync(hflag, ctx->flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    MLB_CUDA(ctx, cudaStreamSynchronize(st));
    if (hflag[0] & 1) {
        const int g = hflag[1] - 1;
        std::string where;
        if (g >= 0 && g < ncell) {
            int l = 0;
            while ((1 << (l + 1)) - 1 <= g) ++l;
            where = " (cell " + std::to_string(g) + " of level " + std::to_string(l) + ": " +
                    std::to_string(H[g].s) + " vectors, " + std::to_string(p) + " moments)";
        }
        return fail(ctx, MLB_ERANK, "a local moment matrix is rank deficient" + where);
    }
    if (hflag[0] & 2) return fail(ctx, MLB_ERANK, "X^T X is not positive definite");
    ctx->state = 1;
    return MLB_OK;
}

mlb_status mlb_build_basis(mlb_ctx* ctx, const double* points, int64_t N, int d, int w) {
    if (!ctx || !points) return fail(ctx, MLB_EINVAL, "null argument");
    ctx->err.clear();
    return build_basis_host(ctx, points, N, d, w);
}

mlb_status mlb_build_basis_dev(mlb_ctx* ctx, const double* points_dev, int64_t N, int d, int w) {
    if (!ctx || !points_dev || N < 1 || d < 1 || d > kMaxDim) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    cudaSetDevice(ctx->opts.device);
    std::vector<double> h((size_t)N * d);
    MLB_CUDA(ctx, cudaMemcpyAsync(h.data(), points_dev, sizeof(double) * N * d, cudaMemcpyDeviceToHost, ctx->stream));
    MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return build_basis_host(ctx, h.data(), N, d, w);
}

mlb_status mlb_assemble(mlb_ctx* ctx, const mlb_theta* th, double tau_factor) {
    if (!ctx || !th) return fail(ctx, MLB_EINVAL, "null argument");
    ctx->err.clear();
    if (ctx->state < 1) return fail(ctx, MLB_ESTATE, "mlb_assemble needs mlb_build_basis first");
    if (th->family != MLB_MATERN && th->family != MLB_GAUSSIAN)
        return fail(ctx, MLB_EINVAL, "family must be MLB_MATERN or MLB_GAUSSIAN");
    if (th->family == MLB_MATERN && !(th->nu >= 0.2 && th->nu <= 30.0))
        return fail(ctx, MLB_EINVAL, "Matern smoothness nu must lie in [0.2, 30]");
    if (!(th->rho > 0) || !std::isfinite(th->rho) || !(th->nugget >= 0) || !std::isfinite(th->nugget))
        return fail(ctx, MLB_EINVAL, "need rho > 0 and nugget >= 0, finite");
    if (th->naxis != 0 && th->naxis != ctx->d)
        return fail(ctx, MLB_EINVAL, "naxis must be 0 (Euclidean) or the dimension d");
    for (int k = 0; k < th->naxis; ++k)
        if (!(th->axis[k] > 0) || !std::isfinite(th->axis[k]))
            return fail(ctx, MLB_EINVAL, "axis weights must be positive and finite");
    if (!(tau_factor >= 0)) return fail(ctx, MLB_EINVAL, "tau_factor must be >= 0 or INFINITY");
    cudaSetDevice(ctx->opts.device);
    cudaStreamSynchronize(ctx->stream);
    ctx->arena_asm.release();
    {
        int* rc = ctx->pan.rowCell;
        ctx->pan = Panels{};
        ctx->pan.rowCell = rc;
        ctx->sym = SymPanels{};
        ctx->diag = nullptr;
    }
    ctx->theta = *th;
    ctx->tau_factor = tau_factor;
    ctx->state = 1;
    {
        mlb_status ks = setup_kernel_fn(ctx);
        if (ks != MLB_OK) return ks;
    }
    if (ctx->opts.matrix_free) {
        if (!std::isinf(tau_factor)) return fail(ctx, MLB_EINVAL, "the three-step product needs tau = INFINITY");
        // the kernel sum runs in every PCG iteration: pick its launch shape now,
        // outside the graph capture of the solve
        mlb_status ts = tune_kernel_sum(ctx);
        if (ts != MLB_OK) return ts;
        ctx->state = 2;
        return MLB_OK;
    }
    for (auto& c : ctx->hcells)
        if (c.s > kTile) return fail(ctx, MLB_EINVAL, "assembled path needs leaf_size <= 64 and 2p <= 64");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    mlb_status s = assemble_dev(ctx);
    cudaEventRecord(e1, ctx->stream);
    if (s == MLB_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "assemble");
    }
    float ms = 0.f;
    if (s == MLB_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MLB_OK) return s;
    ctx->ms_assemble = ms;
    ctx->state = 2;
    return MLB_OK;
}

static mlb_status solve_common(mlb_ctx* ctx, const double* Z_dev_user, mlb_info* info) {
    double* Zkd = ctx->vec + 6 * ctx->N;
    mlb_status s = gather_kd(ctx, Z_dev_user, Zkd);
    if (s != MLB_OK) return s;
    s = solve_dev(ctx, Zkd, info);
    if (s == MLB_OK || s == MLB_ENOCONV || s == MLB_EBREAKDOWN) ctx->state = 3;
    return s;
}

mlb_status mlb_solve(mlb_ctx* ctx, const double* Z, double* beta_out, mlb_info* info) {
    if (!ctx || !Z) return fail(ctx, MLB_EINVAL, "null argument");
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "mlb_solve needs mlb_assemble first");
    cudaSetDevice(ctx->opts.device);
    double* Zu = ctx->vec + 7 * ctx->N;
    MLB_CUDA(ctx, cudaMemcpyAsync(Zu, Z, sizeof(double) * ctx->N, cudaMemcpyHostToDevice, ctx->stream));
    mlb_status s = solve_common(ctx, Zu, info);
    if (ctx->state == 3 && beta_out) {
        MLB_CUDA(ctx, cudaMemcpyAsync(beta_out, ctx->beta, sizeof(double) * ctx->p, cudaMemcpyDeviceToHost, ctx->stream));
        MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return s;
}

mlb_status mlb_solve_dev(mlb_ctx* ctx, const double* Z_dev, double* beta_dev, mlb_info* info) {
    if (!ctx || !Z_dev) return fail(ctx, MLB_EINVAL, "null argument");
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "mlb_solve needs mlb_assemble first");
    cudaSetDevice(ctx->opts.device);
    mlb_status s = solve_common(ctx, Z_dev, info);
    if (ctx->state == 3 && beta_dev)
        MLB_CUDA(ctx, cudaMemcpyAsync(beta_dev, ctx->beta, sizeof(double) * ctx->p, cudaMemcpyDeviceToDevice, ctx->stream));
    return s;
}

mlb_status mlb_predict_dev(mlb_ctx* ctx, const double* targets_dev, int64_t M, double* yhat_dev) {
    if (!ctx || (M > 0 && (!targets_dev || !yhat_dev)) || M < 0) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    if (ctx->state < 3) return fail(ctx, MLB_ESTATE, "mlb_predict needs mlb_solve first");
    cudaSetDevice(ctx->opts.device);
    return kernel_sum_dev(ctx, targets_dev, M, ctx->gamma, yhat_dev, true);
}

mlb_status mlb_predict(mlb_ctx* ctx, const double* targets, int64_t M, double* yhat_out) {
    if (!ctx || (M > 0 && (!targets || !yhat_out)) || M < 0) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    if (ctx->state < 3) return fail(ctx, MLB_ESTATE, "mlb_predict needs mlb_solve first");
    if (M == 0) return MLB_OK;
    cudaSetDevice(ctx->opts.device);
    double *tg = nullptr, *y = nullptr;
    MLB_CUDA(ctx, cudaMalloc(&tg, sizeof(double) * M * ctx->d));
    if (cudaMalloc(&y, sizeof(double) * M) != cudaSuccess) {
        cudaFree(tg);
        return fail(ctx, MLB_ENOMEM, "cudaMalloc failed");
    }
    mlb_status s = MLB_OK;
    if (cudaMemcpyAsync(tg, targets, sizeof(double) * M * ctx->d, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        s = fail(ctx, MLB_ECUDA, "copy of targets failed");
    if (s == MLB_OK) s = kernel_sum_dev(ctx, tg, M, ctx->gamma, y, true);
    if (s == MLB_OK) {
        cudaError_t e = cudaMemcpyAsync(yhat_out, y, sizeof(double) * M, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "predict");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tg);
    cudaFree(y);
    return s;
}

mlb_status mlb_get_sizes(const mlb_ctx* ctx, int64_t* N, int* d, int* p, int* t, int64_t* nwav) {
    if (!ctx) return MLB_EINVAL;
    if (ctx->state < 1) return MLB_ESTATE;
    if (N) *N = ctx->N;
    if (d) *d = ctx->d;
    if (p) *p = ctx->p;
    if (t) *t = ctx->t;
    if (nwav) *nwav = ctx->nwav;
    return MLB_OK;
}

mlb_status mlb_get_perm(mlb_ctx* ctx, int32_t* perm) {
    if (!ctx || !perm) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 1) return fail(ctx, MLB_ESTATE, "no basis");
    std::memcpy(perm, ctx->hperm.data(), sizeof(int) * ctx->N);
    return MLB_OK;
}

mlb_status mlb_get_gamma(mlb_ctx* ctx, double* gamma) {
    if (!ctx || !gamma) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 3) return fail(ctx, MLB_ESTATE, "no solution");
    return host_roundtrip(ctx, nullptr, 0, gamma, ctx->N,
                          [&](double*, double* dout) { return scatter_kd(ctx, ctx->gamma, dout); });
}

mlb_status mlb_apply_W(mlb_ctx* ctx, const double* v, double* out) {
    if (!ctx || !v || !out) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 1) return fail(ctx, MLB_ESTATE, "no basis");
    double* tmp = ctx->vec + 5 * ctx->N;
    return host_roundtrip(ctx, v, ctx->N, out, ctx->nwav, [&](double* din, double* dout) {
        mlb_status s = gather_kd(ctx, din, tmp);
        return s == MLB_OK ? apply_W_dev(ctx, tmp, dout) : s;
    });
}

mlb_status mlb_apply_Wt(mlb_ctx* ctx, const double* u, double* out) {
    if (!ctx || !u || !out) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 1) return fail(ctx, MLB_ESTATE, "no basis");
    double* tmp = ctx->vec + 5 * ctx->N;
    return host_roundtrip(ctx, u, ctx->nwav, out, ctx->N, [&](double* din, double* dout) {
        mlb_status s = apply_Wt_dev(ctx, din, tmp);
        return s == MLB_OK ? scatter_kd(ctx, tmp, dout) : s;
    });
}

mlb_status mlb_cw_matvec(mlb_ctx* ctx, const double* u, double* out) {
    if (!ctx || !u || !out) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "no assembly");
    mlb_status s = host_roundtrip(ctx, u, ctx->nwav, out, ctx->nwav,
                                  [&](double* din, double* dout) { return cw_matvec_dev(ctx, din, dout); });
    if (s == MLB_OK && ctx->sym.err) {
        // the product's bounded waits report here (host_roundtrip has synchronised)
        int e = 0;
        MLB_CUDA(ctx, cudaMemcpyAsync(&e, ctx->sym.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (e) {
            MLB_CUDA(ctx, cudaMemsetAsync(ctx->sym.err, 0, sizeof(int), ctx->stream));
            MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            return fail(ctx, MLB_ETIMEOUT, "a bounded wait of the matrix product gave up");
        }
    }
    return s;
}

mlb_status mlb_cw_matvec_dev(mlb_ctx* ctx, const double* u_dev, double* out_dev) {
    if (!ctx || !u_dev || !out_dev) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "no assembly");
    cudaSetDevice(ctx->opts.device);
    return cw_matvec_dev(ctx, u_dev, out_dev);
}

mlb_status mlb_get_info(const mlb_ctx* ctx, mlb_info* info) {
    if (!ctx || !info) return MLB_EINVAL;
    if (ctx->state < 2) return MLB_ESTATE;
    mlb_info I{};
    if (ctx->state >= 3) I = ctx->last_info;
    I.nnz = ctx->pan.nnz;
    I.nnz_unique = ctx->pan.nnzUnique;
    I.blocks = ctx->pan.blocks;
    I.col_total = ctx->sym.vals ? 0 : ctx->pan.colTotal;
    I.symmetric = ctx->sym.vals ? 1 : 0;
    I.product_values = ctx->opts.matrix_free ? 0 : (ctx->sym.vals ? ctx->sym.stored : ctx->pan.stored);
    I.ms_assemble = ctx->ms_assemble;
    I.launches = ctx->launches;
    I.product_variant = ctx->sym.vals ? ctx->sym_variant : (ctx->opts.matrix_free ? ctx->ksum_variant : 0);
    *info = I;
    return MLB_OK;
}

mlb_status mlb_set_product_variant(mlb_ctx* ctx, int variant) {
    if (!ctx) return MLB_EINVAL;
    if (ctx->state >= 2 && ctx->opts.matrix_free && ctx->opts.precision == MLB_MIXED) {
        // the matrix-free product: the kernel sum's launch shape, or its tensor-core form
        if (variant < 0 || variant > kKsumFormTC) return fail(ctx, MLB_EINVAL, "variant must be 0..6");
        if (variant == kKsumFormTC && !ksum_tc_supported(ctx))
            return fail(ctx, MLB_EINVAL, "no tensor-core kernel sum for this dimension and covariance");
        ctx->ksum_variant = variant;
        return MLB_OK;
    }
    if (ctx->state < 2 || !ctx->sym.vals) return fail(ctx, MLB_ESTATE, "no symmetric storage in this assembly");
    if (variant != 0 && variant != 1) return fail(ctx, MLB_EINVAL, "variant must be 0 or 1");
    ctx->sym_variant = variant;
    return MLB_OK;
}

mlb_status mlb_get_launch_count(const mlb_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return MLB_EINVAL;
    *count = ctx->launches;
    return MLB_OK;
}

mlb_status mlb_get_pattern(mlb_ctx* ctx, int i, int j, uint8_t* flags) {
    if (!ctx || !flags) return fail(ctx, MLB_EINVAL, "null argument");
    if (ctx->state < 2 || ctx->opts.matrix_free) return fail(ctx, MLB_ESTATE, "no assembled matrix");
    if (i < 0 || j < 0 || i > ctx->t || j > ctx->t) return fail(ctx, MLB_EINVAL, "level out of range");
    cudaSetDevice(ctx->opts.device);
    const int ni = 1 << i, nj = 1 << j;
    std::vector<int> row(nj);
    for (int m = 0; m < ni; ++m) {
        const int64_t gm = ni - 1 + m;
        MLB_CUDA(ctx, cudaMemcpyAsync(row.data(), ctx->pan.bcol + gm * ctx->ncell + (nj - 1), sizeof(int) * nj,
                                      cudaMemcpyDeviceToHost, ctx->stream));
        MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int q = 0; q < nj; ++q) flags[(int64_t)m * nj + q] = row[q] >= 0 ? 1 : 0;
    }
    return MLB_OK;
}

mlb_status mlb_kernel_sum(mlb_ctx* ctx, const double* targets, int64_t M, const double* a, double* out) {
    if (!ctx || !targets || !a || !out || M < 1) return fail(ctx, MLB_EINVAL, "bad argument");
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "needs mlb_assemble (theta)");
    cudaSetDevice(ctx->opts.device);
    double* akd = ctx->vec + 5 * ctx->N;
    double* au = ctx->vec + 4 * ctx->N;
    MLB_CUDA(ctx, cudaMemcpyAsync(au, a, sizeof(double) * ctx->N, cudaMemcpyHostToDevice, ctx->stream));
    mlb_status s = gather_kd(ctx, au, akd);
    if (s != MLB_OK) return s;
    return host_roundtrip(ctx, targets, M * ctx->d, out, M,
                          [&](double* din, double* dout) { return kernel_sum_dev(ctx, din, M, akd, dout, false); });
}

mlb_status mlb_mse_dev(mlb_ctx* ctx, const double* targets_dev, int64_t M, double* out_dev) {
    if (!ctx || !targets_dev || !out_dev || M < 1) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "mlb_mse needs mlb_assemble first");
    cudaSetDevice(ctx->opts.device);
    return mse_dev(ctx, targets_dev, M, out_dev);
}

mlb_status mlb_mse(mlb_ctx* ctx, const double* targets, int64_t M, double* mse_out) {
    if (!ctx || !targets || !mse_out || M < 1) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    if (ctx->state < 2) return fail(ctx, MLB_ESTATE, "mlb_mse needs mlb_assemble first");
    cudaSetDevice(ctx->opts.device);
    double *tg = nullptr, *o = nullptr;
    mlb_status s = MLB_OK;
    if (cudaMalloc(&tg, sizeof(double) * M * ctx->d) != cudaSuccess || cudaMalloc(&o, sizeof(double) * M) != cudaSuccess)
        s = fail(ctx, MLB_ENOMEM, "cudaMalloc failed");
    if (s == MLB_OK &&
        cudaMemcpyAsync(tg, targets, sizeof(double) * M * ctx->d, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        s = fail(ctx, MLB_ECUDA, "copy of targets failed");
    if (s == MLB_OK) s = mse_dev(ctx, tg, M, o);
    if (s == MLB_OK) {
        cudaError_t e = cudaMemcpyAsync(mse_out, o, sizeof(double) * M, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "MSE copy");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tg);
    cudaFree(o);
    return s;
}

mlb_status mlb_grad(mlb_ctx* ctx, const double* targets, int64_t M, const double* y_obs, double* loss_out,
                    double* dlogrho_out, double* dlognugget_out) {
    if (!ctx || !targets || !y_obs || M < 1) return fail(ctx, MLB_EINVAL, "bad argument");
    ctx->err.clear();
    if (ctx->state < 3) return fail(ctx, MLB_ESTATE, "mlb_grad needs mlb_solve first");
    cudaSetDevice(ctx->opts.device);
    double *tg = nullptr, *y = nullptr, *o3 = nullptr;
    mlb_status s = MLB_OK;
    if (cudaMalloc(&tg, sizeof(double) * M * ctx->d) != cudaSuccess || cudaMalloc(&y, sizeof(double) * M) != cudaSuccess ||
        cudaMalloc(&o3, sizeof(double) * 3) != cudaSuccess)
        s = fail(ctx, MLB_ENOMEM, "cudaMalloc failed");
    if (s == MLB_OK && (cudaMemcpyAsync(tg, targets, sizeof(double) * M * ctx->d, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
                        cudaMemcpyAsync(y, y_obs, sizeof(double) * M, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess))
        s = fail(ctx, MLB_ECUDA, "copy of targets failed");
    if (s == MLB_OK) s = grad_dev(ctx, tg, M, y, o3);
    double h[3] = {0, 0, 0};
    if (s == MLB_OK) {
        cudaError_t e = cudaMemcpyAsync(h, o3, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "gradient copy");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tg);
    cudaFree(y);
    cudaFree(o3);
    if (s != MLB_OK) return s;
    if (loss_out) *loss_out = h[0];
    if (dlogrho_out) *dlogrho_out = h[1];
    if (dlognugget_out) *dlognugget_out = h[2];
    return MLB_OK;
}

}  // extern "C"
