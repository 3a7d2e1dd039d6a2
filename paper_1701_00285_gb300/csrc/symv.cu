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
//   (its diagonal square in full, and everything to the right of it), cut
//   into tiles of kSymTile columns, each tile stored contiguously with the
//   block's rows one after the other (row r, column c of block b at
//   off[b] + (c / kSymTile) rows kSymTile + r kSymTile + c % kSymTile,
//   c counted from b kSymRows).
//
// One CTA per work item (block b, segment of S.seg columns) streams its
// values once and applies each value twice: to the block's rows (B x, row
// sums) and, for the columns right of the diagonal square, to the columns'
// rows (B^T x, column sums).  Row sums go to rowpart[segment], column sums to
// colpart[block]; the consumer (the PCG update, or sym_reduce) adds them in a
// fixed order, so the product is deterministic.  The dot product p^T q the
// PCG needs is linear in the partials, so every item adds its share and the
// last CTA of the launch forms alpha as on the row-panel path.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "bulk.cuh"
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
        const int64_t rows = min((int64_t)kSymRows, n - row0);
        const double* src = pan.vals + pan.valOff[g] + (i - wOff[g]) * (int64_t)pan.ncols[g];
        float* dst = S.vals + S.off[b] + (i - row0) * kSymTile;
        for (int64_t c = lane; c < W; c += 32) {
            const int64_t j = row0 + c;
            dst[(c / kSymTile) * rows * kSymTile + c % kSymTile] = j < n ? (float)src[j] : 0.0f;
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
// a double-buffered shared array, so one barrier per chunk remains.  The
// partials are FP32 sums and are stored as such (FP64 storage would add
// bytes, not digits); the consumer adds them in FP64.  One
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
    const int64_t cs = row0 + (int64_t)wk.y * S.seg;      // first column of the item
    const int64_t ce = min(row0 + W, cs + S.seg);          // end of its columns (padded width)
    const int64_t diagEnd = row0 + kSymRows;                 // columns below: the diagonal square
    const double* __restrict__ xv = x + (int64_t)rhs * n;
    const float* __restrict__ vb = S.vals + S.off[b];        // the block's first tile
    const int64_t tstride = (int64_t)rows * kSymTile;         // values per tile
    float* __restrict__ colpart = S.colpart + ((int64_t)rhs * S.nblk + b) * n;
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
        // the next chunk's tiles, one contiguous bulk prefetch each (tiles
        // start 16-byte aligned and hold a multiple of 4 values)
        if (tid < (int)min((int64_t)(CH / kSymTile), (ce - pc) / kSymTile))
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vb + ((pc - row0) / kSymTile + tid) * tstride),
                         "r"((unsigned)(tstride * 4))
                         : "memory");
        const int64_t cn = pc + tid;
        const double xn = (cn < ce && cn < n) ? xv[cn] : 0.0;
        const bool ok0 = j0 < m, ok1 = j1 < m;
        const float4 h0 = *reinterpret_cast<const float4*>(&xch[buf][j0]);
        const float4 l0 = *reinterpret_cast<const float4*>(&xcl[buf][j0]);
        const float4 h1 = *reinterpret_cast<const float4*>(&xch[buf][j1]);
        const float4 l1 = *reinterpret_cast<const float4*>(&xcl[buf][j1]);
        // lane columns 4 lane and 128 + 4 lane of the chunk: tiles lane / 16
        // and 2 + lane / 16 of it, column 4 (lane % 16) of the tile
        const float* vc0 = vb + ((c0 - row0) / kSymTile + (lane >> 4)) * tstride + 4 * (lane & 15);
        const float* vc1 = vc0 + 2 * tstride;
        float ca[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ca[k] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < RW; k0 += G) {
            float4 v[G][2];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int r = min(warp + 8 * (k0 + q), rows - 1);
                v[q][0] = ok0 ? __ldg(reinterpret_cast<const float4*>(vc0 + r * kSymTile)) : make_float4(0.f, 0.f, 0.f, 0.f);
                v[q][1] = ok1 ? __ldg(reinterpret_cast<const float4*>(vc1 + r * kSymTile)) : make_float4(0.f, 0.f, 0.f, 0.f);
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
            colpart[c] = s;
            dotp += xv[c] * sd;
        }
        buf ^= 1;
    }
    float* __restrict__ rowpart = S.rowpart + ((int64_t)rhs * S.nsegCap + wk.y) * n;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        float a = racc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const int r = warp + 8 * k;
        if (lane == 0 && r < rows) {
            const double q = (double)a;
            rowpart[row0 + r] = a;
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

// ---- the same product as a bulk-copy pipeline ------------------------------
//
// One producer warp streams the item through a ring of kStages shared-memory
// stages, each one tile (128 rows x kStCols columns, contiguous in global
// memory: a single 32 KB bulk copy) plus the matching FP32 high and low parts
// of x, completion counted in bytes on the stage's "full" mbarrier.  Eight
// consumer warps take the stages in order; warp w owns rows w + 8k and every
// lane two columns of the stage, so a warp reads 256 contiguous bytes of a
// row per shared load.  The values reach shared memory without passing
// through registers, so the bytes in flight are set by the ring (three 33 KB
// stages per CTA, two CTAs per SM), not by the consumers' registers.
// Each consumer warp leaves its column sums of a stage in its own row of the
// stage's column array and releases the stage on its "empty" mbarrier; the
// producer, which waits for that release before refilling the slot anyway,
// adds the eight warps' column sums in a fixed order and writes them out, so
// the consumers never wait for one another.  Every wait is bounded
// (bulk.cuh): one that gives up sets bit 0 of S.err (and, inside the PCG, the
// status ST_TIMEOUT), and the producer then waits (bounded) for its copies in
// flight before the CTA ends.
constexpr int kStCols = kSymTile;   // one stage = one tile of the block
constexpr int kStages = 3;
constexpr int kStageFloats = kSymRows * kStCols + 2 * kStCols;
constexpr size_t kBulkSmem = sizeof(float) * ((size_t)kStages * kStageFloats + (size_t)kStages * 8 * kStCols) +
                             sizeof(uint64_t) * 2 * kStages;

// x (nrhs x n, FP64) -> FP32 high and low parts (nrhs x xld, zero past n)
__global__ void xsplit_kernel(int64_t n, int nrhs, const double* __restrict__ x, int64_t xld, float* __restrict__ xh,
                              float* __restrict__ xl, const PcgState* st) {
    const int64_t tot = (int64_t)nrhs * xld;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = k / xld, i = k - r * xld;
        if (st && st[r].done) continue;
        const double v = i < n ? x[r * n + i] : 0.0;
        const float h = (float)v;
        xh[k] = h;
        xl[k] = (float)(v - (double)h);
    }
}

__device__ __forceinline__ void set_timeout(const SymPanels& S, PcgState* ps) {
    atomicOr(S.err, 1);
    if (ps) {
        ps->status = ST_TIMEOUT;
        ps->done = 1;
    }
}

__global__ void __launch_bounds__(288, 2) sym_spmv_bulk_kernel(SymPanels S, int64_t n, const double* __restrict__ x,
                                                             int nrhs, double* __restrict__ part, PcgState* st) {
    extern __shared__ __align__(128) unsigned char smraw[];
    float* stg = reinterpret_cast<float*>(smraw);                             // kStages x kStageFloats
    float* cred = stg + kStages * kStageFloats;                               // [kStages][8][kStCols]
    uint64_t* full = reinterpret_cast<uint64_t*>(cred + kStages * 8 * kStCols);
    uint64_t* empty = full + kStages;
    const int rhs = (int)(blockIdx.x % (unsigned)nrhs);
    const int item = (int)(blockIdx.x / (unsigned)nrhs);
    PcgState* ps = st ? st + rhs : nullptr;
    if (ps && ps->done) return;
    const int2 wk = S.work[item];
    const int b = wk.x;
    const int64_t row0 = (int64_t)b * kSymRows;
    const int rows = (int)min((int64_t)kSymRows, n - row0);
    const int64_t W = sym_width(n, b);
    const int64_t cs = row0 + (int64_t)wk.y * S.seg;
    const int64_t ce = min(row0 + W, cs + S.seg);
    const int64_t diagEnd = row0 + kSymRows;
    const int nst = (int)((ce - cs) / kStCols);                                // whole tiles
    const double* __restrict__ xv = x + (int64_t)rhs * n;
    const float* __restrict__ xh = S.xh + (int64_t)rhs * S.xld;
    const float* __restrict__ xl = S.xl + (int64_t)rhs * S.xld;
    const float* __restrict__ vb = S.vals + S.off[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 8);
        }
        mbar_fence_init();
    }
    __syncthreads();
    double dotp = 0.0;
    if (warp == 8) {
        // producer.  Tiles start 16-byte aligned and hold a multiple of 16
        // bytes, as the bulk copy requires.
        float* __restrict__ colpart = S.colpart + ((int64_t)rhs * S.nblk + b) * n;
        // column sums of stage s (its slot released by all eight warps): the
        // warps' sums in order, the x of the columns from the stage itself
        auto finish = [&](int s) {
            const int slot = s % kStages;
            const float* cr = cred + slot * 8 * kStCols + 2 * lane;
            float2 a = *reinterpret_cast<const float2*>(cr);
#pragma unroll
            for (int w = 1; w < 8; ++w) {
                const float2 t = *reinterpret_cast<const float2*>(cr + w * kStCols);
                a.x += t.x;
                a.y += t.y;
            }
            const float* sx = stg + slot * kStageFloats + kSymRows * kStCols;
            const int64_t c = cs + (int64_t)s * kStCols + 2 * lane;
            if (c >= diagEnd && c < n) {
                colpart[c] = a.x;
                dotp += ((double)sx[2 * lane] + (double)sx[kStCols + 2 * lane]) * (double)a.x;
            }
            if (c + 1 >= diagEnd && c + 1 < n) {
                colpart[c + 1] = a.y;
                dotp += ((double)sx[2 * lane + 1] + (double)sx[kStCols + 2 * lane + 1]) * (double)a.y;
            }
        };
        int issued = 0, done = 0;
        bool ok = true;
        for (int s = 0; s < nst; ++s) {
            const int slot = s % kStages, round = s / kStages;
            if (round > 0) {
                if (!mbar_wait(&empty[slot], (round - 1) & 1)) {
                    ok = false;
                    break;
                }
                finish(s - kStages);
                done = s - kStages + 1;
                __syncwarp();
            }
            const int64_t c0 = cs + (int64_t)s * kStCols;
            const unsigned rb = (unsigned)kStCols * 4u;                 // x parts of the tile
            const unsigned tb = (unsigned)rows * rb;                     // the tile
            float* dst = stg + slot * kStageFloats;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[slot], tb + 2 * rb);
                bulk_g2s(dst, vb + (c0 - row0) / kStCols * (int64_t)rows * kStCols, tb, &full[slot]);
                bulk_g2s(dst + kSymRows * kStCols, xh + c0, rb, &full[slot]);
                bulk_g2s(dst + kSymRows * kStCols + kStCols, xl + c0, rb, &full[slot]);
            }
            __syncwarp();
            issued = s + 1;
        }
        for (int s = done; ok && s < issued; ++s) {
            if (!mbar_wait(&empty[s % kStages], (s / kStages) & 1)) {
                ok = false;
                break;
            }
            finish(s);
        }
        if (!ok) {
            if (lane == 0) set_timeout(S, ps);
            // the copies this CTA has in flight land before it ends
            for (int s = max(0, issued - kStages); s < issued; ++s) mbar_wait(&full[s % kStages], (s / kStages) & 1);
        }
    } else {
        float xrh[16], xrl[16], racc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int r = warp + 8 * k;
            xrh[k] = r < rows ? xh[row0 + r] : 0.0f;
            xrl[k] = r < rows ? xl[row0 + r] : 0.0f;
            racc[k] = 0.0f;
        }
        bool ok = true;
        for (int s = 0; s < nst; ++s) {
            const int slot = s % kStages;
            if (!mbar_wait(&full[slot], (s / kStages) & 1)) {
                ok = false;
                break;
            }
            const float* sv = stg + slot * kStageFloats;
            const float2 h = *reinterpret_cast<const float2*>(sv + kSymRows * kStCols + 2 * lane);
            const float2 l = *reinterpret_cast<const float2*>(sv + kSymRows * kStCols + kStCols + 2 * lane);
            // four interleaved column accumulators (rows k mod 4) keep the
            // dependent FMA chains short
            float ca[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) ca[q][0] = ca[q][1] = 0.0f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (warp + 8 * k < rows) {           // warp-uniform
                    const float2 v = *reinterpret_cast<const float2*>(sv + (warp + 8 * k) * kStCols + 2 * lane);
                    racc[k] = fmaf(v.x, h.x, fmaf(v.y, h.y, fmaf(v.x, l.x, fmaf(v.y, l.y, racc[k]))));
                    ca[k & 3][0] = fmaf(v.x, xrh[k], fmaf(v.x, xrl[k], ca[k & 3][0]));
                    ca[k & 3][1] = fmaf(v.y, xrh[k], fmaf(v.y, xrl[k], ca[k & 3][1]));
                }
            }
            *reinterpret_cast<float2*>(cred + (slot * 8 + warp) * kStCols + 2 * lane) =
                make_float2((ca[0][0] + ca[1][0]) + (ca[2][0] + ca[3][0]), (ca[0][1] + ca[1][1]) + (ca[2][1] + ca[3][1]));
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        if (!ok) {
            if (lane == 0) set_timeout(S, ps);
        } else {
            float* __restrict__ rowpart = S.rowpart + ((int64_t)rhs * S.nsegCap + wk.y) * n;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = racc[k];
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                const int r = warp + 8 * k;
                if (lane == 0 && r < rows) {
                    const double q = (double)a;
                    rowpart[row0 + r] = a;
                    dotp += xv[row0 + r] * q;
                }
            }
        }
    }
    if (part) {
        const double sdot = block_reduce(dotp);
        if (tid == 0) part[(int64_t)rhs * S.nwork + item] = sdot;
        if (ps && draw_last_ticket(ps, (unsigned)S.nwork))
            pcg_alpha_finish(part + (int64_t)rhs * S.nwork, S.nwork, ps);
    }
}

// y = q of right-hand side 0, in the order of the PCG update
// (pcg_update_sym_kernel): eight warps per 32 elements, every eighth slot each
__global__ void __launch_bounds__(256) sym_reduce_kernel(SymPanels S, int64_t n, double* __restrict__ y) {
    __shared__ double qs[8][32];
    const int j = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (int64_t c0 = (int64_t)blockIdx.x * 32; c0 < n; c0 += (int64_t)gridDim.x * 32) {
        const int64_t i = c0 + j;
        qs[g][j] = i < n ? sym_q_slots(S, n, i, 0, g, 8) : 0.0;
        __syncthreads();
        if (g == 0 && i < n) {
            double q = qs[0][j];
#pragma unroll
            for (int k = 1; k < 8; ++k) q += qs[k][j];
            y[i] = q;
        }
        __syncthreads();
    }
}

static mlb_status tune_sym(mlb_ctx* ctx);

// Partial buffers for nrhs simultaneous products of the current plan.
mlb_status sym_reserve(mlb_ctx* ctx, int nrhs) {
    SymPanels& S = ctx->sym;
    if (nrhs <= S.nrhs && S.nsegMax <= S.nsegCap) return MLB_OK;
    nrhs = std::max(nrhs, S.nrhs);
    Arena& A = ctx->arena_asm;
    for (void* q : {(void*)S.rowpart, (void*)S.colpart, (void*)S.xh, (void*)S.xl}) dfree(ctx, A, q);
    S.rowpart = S.colpart = nullptr;
    S.xh = S.xl = nullptr;
    S.nrhs = 0;
    const int64_t n = ctx->nwav;
    S.xld = sym_width(n, 0);
    S.nsegCap = S.nsegMax;
    S.rowpart = (float*)dalloc(ctx, A, sizeof(float) * (size_t)nrhs * S.nsegCap * n);
    S.colpart = (float*)dalloc(ctx, A, sizeof(float) * (size_t)nrhs * S.nblk * n);
    S.xh = (float*)dalloc(ctx, A, sizeof(float) * (size_t)nrhs * S.xld);
    S.xl = (float*)dalloc(ctx, A, sizeof(float) * (size_t)nrhs * S.xld);
    if (!S.rowpart || !S.colpart || !S.xh || !S.xl) return fail(ctx, MLB_ENOMEM, "symmetric product partials");
    // entries past nwav stay zero: the writers of the split vectors stop at nwav
    MLB_CUDA(ctx, cudaMemsetAsync(S.xh, 0, sizeof(float) * (size_t)nrhs * S.xld, ctx->stream));
    MLB_CUDA(ctx, cudaMemsetAsync(S.xl, 0, sizeof(float) * (size_t)nrhs * S.xld, ctx->stream));
    S.nrhs = nrhs;
    return MLB_OK;
}

// Work list of the product for items of `seg` columns: (block, segment),
// heaviest first, so the last wave of CTAs is short.
static mlb_status sym_plan(mlb_ctx* ctx, int seg) {
    SymPanels& S = ctx->sym;
    const int64_t n = ctx->nwav;
    std::vector<std::pair<int64_t, int2>> items;
    int nsegMax = 0;
    for (int b = 0; b < S.nblk; ++b) {
        const int64_t rows = std::min<int64_t>(kSymRows, n - (int64_t)b * kSymRows);
        const int64_t W = sym_width(n, b);
        const int ns = sym_nseg(n, b, seg);
        nsegMax = std::max(nsegMax, ns);
        for (int s = 0; s < ns; ++s) {
            const int64_t cols = std::min<int64_t>(seg, W - (int64_t)s * seg);
            items.push_back({-rows * cols, make_int2(b, s)});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& c) { return a.first < c.first; });
    std::vector<int2> work;
    for (auto& it : items) work.push_back(it.second);
    if (work.size() > max_work_items(ctx->ncell, ctx->N)) return fail(ctx, MLB_EINVAL, "symmetric work table bound");
    Arena& A = ctx->arena_asm;
    if (!S.work || (int)work.size() > S.nworkCap) {
        dfree(ctx, A, S.work);
        S.work = (int2*)dalloc(ctx, A, sizeof(int2) * work.size());
        if (!S.work) return fail(ctx, MLB_ENOMEM, "symmetric work table");
        S.nworkCap = (int)work.size();
    }
    S.nwork = (int)work.size();
    S.seg = seg;
    S.nsegMax = nsegMax;
    MLB_CUDA(ctx, cudaMemcpyAsync(S.work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, ctx->stream));
    MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // `work` goes out of scope
    return sym_reserve(ctx, std::max(1, S.nrhs));
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
    int64_t tot = 0;
    for (int b = 0; b < S.nblk; ++b) {
        off[b] = tot;
        tot += std::min<int64_t>(kSymRows, n - (int64_t)b * kSymRows) * sym_width(n, b);
    }
    S.stored = tot;
    Arena& A = ctx->arena_asm;
    S.vals = (float*)dalloc(ctx, A, sizeof(float) * tot);
    S.off = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * S.nblk);
    S.err = (int*)dalloc(ctx, A, sizeof(int));
    if (!S.vals || !S.off || !S.err) return fail(ctx, MLB_ENOMEM, "symmetric storage");
    cudaStream_t st = ctx->stream;
    MLB_CUDA(ctx, cudaMemsetAsync(S.err, 0, sizeof(int), st));
    MLB_CUDA(ctx, cudaMemcpyAsync(S.off, off.data(), sizeof(int64_t) * S.nblk, cudaMemcpyHostToDevice, st));
    const int64_t warps = std::min<int64_t>(n, (int64_t)std::max(ctx->nsm, 1) * 64);
    sym_pack_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(ctx->pan, ctx->pan.rowCell, ctx->cells.wOff,
                                                                         n, S);
    MLB_CHECK_LAUNCH(ctx, "sym_pack_kernel");
    return tune_sym(ctx);   // synchronises the stream before `off` goes out of scope
}

void sym_launch(mlb_ctx* ctx, const double* x, int nrhs, double* part, PcgState* st, bool presplit) {
    const SymPanels& S = ctx->sym;
    if (ctx->sym_variant == 1) {
        if (!presplit) {
            xsplit_kernel<<<kVecBlocks, 256, 0, ctx->stream>>>(ctx->nwav, nrhs, x, S.xld, S.xh, S.xl, st);
            ctx->launches += 1;
        }
        sym_spmv_bulk_kernel<<<(unsigned)(S.nwork * nrhs), 288, kBulkSmem, ctx->stream>>>(S, ctx->nwav, x, nrhs,
                                                                                          part, st);
    } else {
        sym_spmv_f32_kernel<<<(unsigned)(S.nwork * nrhs), 256, 0, ctx->stream>>>(S, ctx->nwav, x, nrhs, part, st);
    }
}

// Chooses the form of the product (0: plain loads with L2 prefetch, 1:
// bulk-copy pipeline) and the columns per work item (2,048, 1,024 or 512:
// fewer, longer items against a shorter last wave) by timing every pair on
// the context's own matrix (CUDA events on its stream, outside any capture),
// cached per (device, size bucket) for the rest of the process.
static std::mutex g_sym_mutex;
static std::map<std::pair<int, int>, std::pair<int, int>> g_sym_cache;

static mlb_status tune_sym(mlb_ctx* ctx) {
    MLB_CUDA(ctx, cudaFuncSetAttribute(sym_spmv_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBulkSmem));
    int dev = 0;
    cudaGetDevice(&dev);
    int bucket = 0;
    while ((1LL << (bucket + 1)) <= ctx->nwav) ++bucket;
    const auto key = std::make_pair(dev, bucket);
    {
        std::lock_guard<std::mutex> lock(g_sym_mutex);
        auto it = g_sym_cache.find(key);
        if (it != g_sym_cache.end()) {
            ctx->sym_variant = it->second.first;
            return sym_plan(ctx, it->second.second);
        }
    }
    double* u = ctx->vec + 3 * ctx->nwav;
    MLB_CUDA(ctx, cudaMemsetAsync(u, 0, sizeof(double) * ctx->nwav, ctx->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> bestc(0, 2048);
    mlb_status s = MLB_OK;
    for (int seg : {2048, 1024, 512}) {
        if ((s = sym_plan(ctx, seg)) != MLB_OK) break;
        for (int v = 0; v < 2; ++v) {
            ctx->sym_variant = v;
            sym_launch(ctx, u, 1, nullptr, nullptr);
            cudaEventRecord(e0, ctx->stream);
            for (int k = 0; k < 3; ++k) sym_launch(ctx, u, 1, nullptr, nullptr);
            cudaEventRecord(e1, ctx->stream);
            ctx->launches += 4;
            const cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                s = cuda_fail(ctx, e, "symmetric product tuning");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bestc = std::make_pair(v, seg);
            }
        }
        if (s != MLB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MLB_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_sym_mutex);
        g_sym_cache[key] = bestc;
    }
    ctx->sym_variant = bestc.first;
    return sym_plan(ctx, bestc.second);
}

void sym_reduce(mlb_ctx* ctx, double* out) {
    sym_reduce_kernel<<<kVecBlocks, 256, 0, ctx->stream>>>(ctx->sym, ctx->nwav, out);
    ctx->launches += 1;
}

}  // namespace mlb
