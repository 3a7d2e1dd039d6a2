// Symmetric packed FP32 storage of a complete C~_W and its one-pass product
// (mixed path).
//
// C~_W is symmetric: its entries are psi_m^T C psi_q and the distance
// criterion of Sec. 4.1 is symmetric in the two cells, so Alg. 7 computes the
// blocks j >= i only and mirrors the others (remark after Alg. 6).  When every
// pair of cells is admissible (tau = infinity) the matrix is dense, and the
// PCG product -- HBM bound on the FP32 path -- would stream every value twice
// if both triangles were stored.  Here each symmetric pair is stored once:
//
//   rows in blocks of kSymRows; block b keeps columns b kSymRows .. nwav - 1
//   (its diagonal square in full, and everything to the right of it),
//   row-major, row stride sym_width(nwav, b).
//
// One CTA per work item (block b, segment of kSymSeg columns) streams its
// values once and applies each value twice: to the block's rows (B x, row
// sums) and, for the columns right of the diagonal square, to the columns'
// rows (B^T x, column sums).  Row sums go to rowpart[segment], column sums to
// colpart[block]; the consumer (the PCG update, or sym_reduce) adds them in a
// fixed order, so the product is deterministic.  The dot product p^T q the
// PCG needs is linear in the partials, so every item adds its share and the
// last CTA of the launch forms alpha as on the row-panel path.
#include <algorithm>
#include <utility>
#include <vector>

#include "internal.h"
#include "pcg_device.cuh"

namespace mlb {

constexpr int kSymChunk = 256;   // columns staged per step (one per thread)

// FP64 row panels of a complete pattern (the panel column of an entry is its
// global wavelet column) -> packed FP32 upper blocks.  One warp per stored row.
__global__ void sym_pack_kernel(Panels pan, const int* __restrict__ rowCell, const int64_t* __restrict__ wOff,
                                int64_t n, SymPanels S) {
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t i = w0; i < n; i += nw) {
        const int b = (int)(i / kSymRows);
        const int64_t row0 = (int64_t)b * kSymRows;
        const int64_t W = sym_width(n, b);
        const int g = rowCell[i];
        const double* src = pan.vals + pan.valOff[g] + (i - wOff[g]) * (int64_t)pan.ncols[g];
        float* dst = S.vals + S.off[b] + (i - row0) * W;
        for (int64_t c = lane; c < W; c += 32) {
            const int64_t j = row0 + c;
            dst[c] = j < n ? (float)src[j] : 0.0f;
        }
    }
}

// The product of nrhs vectors (x: nrhs x n, right-hand side after
// right-hand side; CTA blockIdx.x serves item blockIdx.x / nrhs for
// right-hand side blockIdx.x % nrhs, so the CTAs that read one item's values
// run side by side and share them through L2).
//
// Per 256-column chunk each warp owns 16 rows of the block (warp, warp + 8,
// ...) and each lane two float4 column groups (4 lane and 128 + 4 lane); it
// loads four rows' values at a time (eight 16-byte loads in flight per lane)
// and applies each value to the row sum (against the staged x of the chunk)
// and to the column sum (against the staged x of the row).  x enters as FP32
// high and low parts (x = h + l to about 2^-48), products and sums are FP32,
// and the partials leave in FP64.  Column sums cross the eight warps through
// a double-buffered shared array, so one barrier per chunk remains.  One
// thread per row asks the L2 for that row's next chunk (bulk prefetch) while
// the current one is multiplied.
__global__ void __launch_bounds__(256, 2) sym_spmv_f32_kernel(SymPanels S, int64_t n, const double* __restrict__ x,
                                                           int nrhs, double* __restrict__ part, PcgState* st) {
    constexpr int CH = kSymChunk;
    constexpr int RW = kSymRows / 8;    // rows per warp
    constexpr int G = 4;                // rows loaded together
    __shared__ __align__(16) float xrh[kSymRows];
    __shared__ __align__(16) float xrl[kSymRows];
    __shared__ __align__(16) float xch[2][CH];
    __shared__ __align__(16) float xcl[2][CH];
    __shared__ __align__(16) float cred[2][8][CH];
    const int rhs = (int)(blockIdx.x % (unsigned)nrhs);
    const int item = (int)(blockIdx.x / (unsigned)nrhs);
    PcgState* ps = st ? st + rhs : nullptr;
    if (ps && ps->done) return;
    const int2 wk = S.work[item];
    const int b = wk.x;
    const int64_t row0 = (int64_t)b * kSymRows;
    const int rows = (int)min((int64_t)kSymRows, n - row0);
    const int64_t W = sym_width(n, b);
    const int64_t cs = row0 + (int64_t)wk.y * kSymSeg;      // first column of the item
    const int64_t ce = min(row0 + W, cs + kSymSeg);          // end of its columns (padded width)
    const int64_t diagEnd = row0 + kSymRows;                 // columns below: the diagonal square
    const double* __restrict__ xv = x + (int64_t)rhs * n;
    const float* __restrict__ vb = S.vals + S.off[b];        // row r, column c: vb[r W + c - row0]
    double* __restrict__ colpart = S.colpart + ((int64_t)rhs * S.nblk + b) * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kSymRows) {
        const double xr = tid < rows ? xv[row0 + tid] : 0.0;
        const float h = (float)xr;
        xrh[tid] = h;
        xrl[tid] = (float)(xr - (double)h);
    }
    {
        const int64_t c = cs + tid;
        const double xc = (c < ce && c < n) ? xv[c] : 0.0;
        const float h = (float)xc;
        xch[0][tid] = h;
        xcl[0][tid] = (float)(xc - (double)h);
    }
    __syncthreads();
    float racc[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) racc[k] = 0.0f;
    double dotp = 0.0;
    const int j0 = 4 * lane, j1 = 128 + 4 * lane;
    int buf = 0;
    for (int64_t c0 = cs; c0 < ce; c0 += CH) {
        const int m = (int)min((int64_t)CH, ce - c0);          // a multiple of 4
        const int64_t pc = c0 + CH;
        // rows start 16-byte aligned and the chunk is a multiple of 4 values,
        // as the bulk prefetch requires
        if (tid < rows && pc < ce)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vb + (int64_t)tid * W + (pc - row0)),
                         "r"((unsigned)(min((int64_t)CH, ce - pc) * 4))
                         : "memory");
        const int64_t cn = pc + tid;
        const double xn = (cn < ce && cn < n) ? xv[cn] : 0.0;
        const bool ok0 = j0 < m, ok1 = j1 < m;
        const float4 h0 = *reinterpret_cast<const float4*>(&xch[buf][j0]);
        const float4 l0 = *reinterpret_cast<const float4*>(&xcl[buf][j0]);
        const float4 h1 = *reinterpret_cast<const float4*>(&xch[buf][j1]);
        const float4 l1 = *reinterpret_cast<const float4*>(&xcl[buf][j1]);
        const float* vc = vb + (c0 - row0);
        float ca[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ca[k] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < RW; k0 += G) {
            float4 v[G][2];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int r = min(warp + 8 * (k0 + q), rows - 1);
                const float* rp = vc + (int64_t)r * W;
                v[q][0] = ok0 ? __ldg(reinterpret_cast<const float4*>(rp + j0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                v[q][1] = ok1 ? __ldg(reinterpret_cast<const float4*>(rp + j1)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int r = warp + 8 * (k0 + q);
                const float4 a = v[q][0], c = v[q][1];
                float s = 0.0f;
                s = fmaf(a.x, h0.x, s); s = fmaf(a.y, h0.y, s); s = fmaf(a.z, h0.z, s); s = fmaf(a.w, h0.w, s);
                s = fmaf(c.x, h1.x, s); s = fmaf(c.y, h1.y, s); s = fmaf(c.z, h1.z, s); s = fmaf(c.w, h1.w, s);
                s = fmaf(a.x, l0.x, s); s = fmaf(a.y, l0.y, s); s = fmaf(a.z, l0.z, s); s = fmaf(a.w, l0.w, s);
                s = fmaf(c.x, l1.x, s); s = fmaf(c.y, l1.y, s); s = fmaf(c.z, l1.z, s); s = fmaf(c.w, l1.w, s);
                racc[k0 + q] += s;
                const float wh = xrh[r], wl = xrl[r];     // zero past the block's last row
                ca[0] = fmaf(a.x, wh, fmaf(a.x, wl, ca[0]));
                ca[1] = fmaf(a.y, wh, fmaf(a.y, wl, ca[1]));
                ca[2] = fmaf(a.z, wh, fmaf(a.z, wl, ca[2]));
                ca[3] = fmaf(a.w, wh, fmaf(a.w, wl, ca[3]));
                ca[4] = fmaf(c.x, wh, fmaf(c.x, wl, ca[4]));
                ca[5] = fmaf(c.y, wh, fmaf(c.y, wl, ca[5]));
                ca[6] = fmaf(c.z, wh, fmaf(c.z, wl, ca[6]));
                ca[7] = fmaf(c.w, wh, fmaf(c.w, wl, ca[7]));
            }
        }
        *reinterpret_cast<float4*>(&cred[buf][warp][j0]) = make_float4(ca[0], ca[1], ca[2], ca[3]);
        *reinterpret_cast<float4*>(&cred[buf][warp][j1]) = make_float4(ca[4], ca[5], ca[6], ca[7]);
        {
            const float h = (float)xn;
            xch[buf ^ 1][tid] = h;
            xcl[buf ^ 1][tid] = (float)(xn - (double)h);
        }
        __syncthreads();
        // one thread per column: the eight warps' sums, for the columns right
        // of the diagonal square (the square's transpose is its own rows)
        const int64_t c = c0 + tid;
        if (tid < m && c >= diagEnd && c < n) {
            float s = 0.0f;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += cred[buf][w][tid];
            const double sd = (double)s;
            colpart[c] = sd;
            dotp += xv[c] * sd;
        }
        buf ^= 1;
    }
    double* __restrict__ rowpart = S.rowpart + ((int64_t)rhs * S.nsegMax + wk.y) * n;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        float a = racc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const int r = warp + 8 * k;
        if (lane == 0 && r < rows) {
            const double q = (double)a;
            rowpart[row0 + r] = q;
            dotp += xv[row0 + r] * q;
        }
    }
    if (part) {
        const double s = block_reduce(dotp);
        if (tid == 0) part[(int64_t)rhs * S.nwork + item] = s;
        // inside the PCG the last CTA of this right-hand side forms alpha
        if (ps && draw_last_ticket(ps, (unsigned)S.nwork))
            pcg_alpha_finish(part + (int64_t)rhs * S.nwork, S.nwork, ps);
    }
}

__global__ void sym_reduce_kernel(SymPanels S, int64_t n, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = sym_q(S, n, i, 0);
}

mlb_status sym_reserve(mlb_ctx* ctx, int nrhs) {
    SymPanels& S = ctx->sym;
    if (nrhs <= S.nrhs) return MLB_OK;
    dfree(ctx->arena_asm, S.rowpart);
    dfree(ctx->arena_asm, S.colpart);
    S.rowpart = S.colpart = nullptr;
    S.nrhs = 0;
    const int64_t n = ctx->nwav;
    S.rowpart = (double*)dalloc(ctx, ctx->arena_asm, sizeof(double) * (size_t)nrhs * S.nsegMax * n);
    S.colpart = (double*)dalloc(ctx, ctx->arena_asm, sizeof(double) * (size_t)nrhs * S.nblk * n);
    if (!S.rowpart || !S.colpart) return fail(ctx, MLB_ENOMEM, "symmetric product partials");
    S.nrhs = nrhs;
    return MLB_OK;
}

// Packs the FP64 panels of a complete pattern (nwav > 0) into the symmetric
// FP32 storage; the caller frees the FP64 panels afterwards.
mlb_status build_sym(mlb_ctx* ctx) {
    SymPanels& S = ctx->sym;
    S = SymPanels{};
    const int64_t n = ctx->nwav;
    if (n <= 0) return fail(ctx, MLB_EINVAL, "symmetric storage needs wavelet rows");
    S.nblk = (int)((n + kSymRows - 1) / kSymRows);
    std::vector<int64_t> off(S.nblk);
    std::vector<std::pair<int64_t, int2>> items;
    int64_t tot = 0;
    for (int b = 0; b < S.nblk; ++b) {
        const int64_t rows = std::min<int64_t>(kSymRows, n - (int64_t)b * kSymRows);
        const int64_t W = sym_width(n, b);
        off[b] = tot;
        tot += rows * W;
        const int ns = sym_nseg(n, b);
        S.nsegMax = std::max(S.nsegMax, ns);
        for (int s = 0; s < ns; ++s) {
            const int64_t cols = std::min<int64_t>(kSymSeg, W - (int64_t)s * kSymSeg);
            items.push_back({-rows * cols, make_int2(b, s)});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& c) { return a.first < c.first; });
    std::vector<int2> work;
    for (auto& it : items) work.push_back(it.second);
    if (work.size() > max_work_items(ctx->ncell, ctx->N)) return fail(ctx, MLB_EINVAL, "symmetric work table bound");
    S.nwork = (int)work.size();
    S.stored = tot;
    Arena& A = ctx->arena_asm;
    S.vals = (float*)dalloc(ctx, A, sizeof(float) * tot);
    S.off = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * S.nblk);
    S.work = (int2*)dalloc(ctx, A, sizeof(int2) * work.size());
    if (!S.vals || !S.off || !S.work) return fail(ctx, MLB_ENOMEM, "symmetric storage");
    cudaStream_t st = ctx->stream;
    MLB_CUDA(ctx, cudaMemcpyAsync(S.off, off.data(), sizeof(int64_t) * S.nblk, cudaMemcpyHostToDevice, st));
    MLB_CUDA(ctx, cudaMemcpyAsync(S.work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, st));
    const int64_t warps = std::min<int64_t>(n, (int64_t)std::max(ctx->nsm, 1) * 64);
    sym_pack_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(ctx->pan, ctx->pan.rowCell, ctx->cells.wOff,
                                                                         n, S);
    MLB_CHECK_LAUNCH(ctx, "sym_pack_kernel");
    // the host vectors above go out of scope: wait for their copies
    MLB_CUDA(ctx, cudaStreamSynchronize(st));
    return sym_reserve(ctx, 1);
}

void sym_launch(mlb_ctx* ctx, const double* x, int nrhs, double* part, PcgState* st) {
    const SymPanels& S = ctx->sym;
    sym_spmv_f32_kernel<<<(unsigned)(S.nwork * nrhs), 256, 0, ctx->stream>>>(S, ctx->nwav, x, nrhs, part, st);
}

void sym_reduce(mlb_ctx* ctx, double* out) {
    sym_reduce_kernel<<<kVecBlocks, 256, 0, ctx->stream>>>(ctx->sym, ctx->nwav, out);
    ctx->launches += 1;
}

}  // namespace mlb
