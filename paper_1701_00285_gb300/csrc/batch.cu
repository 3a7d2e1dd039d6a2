// Many independent BLUP problems in one call (the batched workload: problems
// of different sizes, dimensions and covariance parameters).
//
// Every problem gets its own context (basis, assembly, vectors).  The setup
// phases -- kd-tree and basis, assembly of C~_W, Z_W = W Z -- and the closing
// phases -- gamma = W^T gamma_W, the trend step, predictions -- run the
// single-problem kernels on a pool of streams driven by host threads.  The PCG
// phase, where a per-problem loop would be bound by kernel launches (five
// launches per iteration on systems of a few thousand unknowns), is one
// persistent launch over all problems: each problem's diagonally
// preconditioned CG (Sec. 5.2 remark, Sec. 6.2) is a chain of phases (the
// product q = C~_W p, the update of x, r, z), each phase cut into row chunks
// that any CTA may take.  The CTA finishing a phase's last chunk reduces the
// chunks' partial sums in chunk order and opens the next phase, so the
// result does not depend on which CTA did what, and no CTA waits for
// another: CTAs without work take chunks of other problems.  A long-running
// problem therefore gets the whole GPU once the others are done.  Systems
// too wide to stage their search direction in shared memory run the
// single-problem PCG on the stream pool meanwhile.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "bulk.cuh"
#include "pcg_device.cuh"

namespace mlb {

// The persistent PCG takes systems of at most kFlowCols unknowns: every
// chunk of a product stages the search direction in shared memory, 8 bytes
// per column.
constexpr int kFlowCols = 12288;
constexpr int kFlowThreads = 256;
constexpr int kFlowWarps = kFlowThreads / 32;
constexpr int kUpdRows = 128;                  // rows per chunk of the vector phases
constexpr int kFlowDenseRows = 16;             // rows per product chunk, complete patterns (4 rows x 2 column halves per warp pair)
constexpr int64_t kProdValues = 1 << 18;       // panel values per product chunk, truncated patterns
constexpr int kFlowSymSeg = 512;               // columns per product chunk, symmetric storage (8 tiles)
// shared scratch of a symmetric chunk, in doubles: p on the rows and columns
// in FP64 and in FP32 high and low parts, and eight warps' column sums
constexpr int kFlowSymSmem = (kSymRows + kFlowSymSeg) + (kSymRows + kFlowSymSeg) + 8 * 256 / 2;
constexpr int kFlowSpan = 2048;                // columns summed in FP32 before the FP64 sum

// One problem of the persistent launch: its panels (row panels of C~_W, FP32
// or FP64), its vectors and the chunking of its phases.
struct FlowProblem {
    const float* vals32;       // panel values (mixed path) or nullptr
    const double* vals64;      // panel values (FP64 path) or nullptr
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
    double* p0;                // search directions of even iterations
    double* p1;                // and of odd ones
    double* q;
    double* part;              // per chunk of the current phase: its partial sums
    // symmetric FP32 storage (mixed precision, complete pattern): the chunks
    // of a product are (row block, column segment) pairs
    const float* symVals;      // nullptr: row panels
    const int64_t* symOff;     // per row block: offset of its first value
    const int2* symItem;       // per chunk: (block, segment)
    float* rowpart;            // nsegSym x n: a segment's sums over the block's rows
    float* colpart;            // nblk x n: a block's sums over the columns right of its square
    PcgState* st;
    double tol2;
    int n;
    int width;                 // staged columns: n rounded up to the panels' padding
    int dense;                 // every panel holds all n columns in order (no index lists)
    int prodRows;              // rows per product chunk
    int nprod, nupd;           // chunks of a product phase and of a vector phase
    int maxit;
};

// Scheduling state of one problem.  Phases are numbered by epoch: 0 sets up
// the residual, 2i + 1 is the product of iteration i, 2i + 2 its update.
// `ticket` hands out the chunks of the current epoch (epoch << 32 | next
// chunk); the CTA that finishes the epoch's last chunk reduces the partial
// sums, sets the scalars and opens the next epoch.  No CTA ever waits for
// another one: a CTA without work looks at other problems.
struct FlowCtl {
    unsigned long long ticket;
    unsigned done;             // chunks of the current epoch finished
    int finished;              // set when the problem's solve ended (the search needs no flag:
                               // a finished problem shows no open chunk)
    double rz, bb, rr, alpha, beta;
    int it;                    // iterations completed
};

struct FlowGlobal {
    unsigned long long hot;    // (iterations << 32 | problem) of the longest-running problem
    int remaining;             // problems not finished
    unsigned progress;         // epochs opened or problems finished, all problems
    int err;                   // set when no problem made progress for kWaitCycles
};

__device__ __forceinline__ unsigned flow_chunks(const FlowProblem& P, unsigned e) {
    return (e & 1u) ? (unsigned)P.nprod : (unsigned)P.nupd;
}

__device__ __forceinline__ double* flow_dir(const FlowProblem& P, int it) { return (it & 1) ? P.p1 : P.p0; }

// Fixed-order CTA sum of two values (all threads get both).
__device__ __forceinline__ double2 flow_sum2(double a, double b, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[wid] = a;
        red[kFlowWarps + wid] = b;
    }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < kFlowWarps; ++i) {
        sa += red[i];
        sb += red[kFlowWarps + i];
    }
    return make_double2(sa, sb);
}

// Epoch 0, rows [r0, r1): x = 0, r = b, z = D^-1 b, p_0 = z; partials b.z, b.b.
__device__ void flow_init(const FlowProblem& P, int c, double* red) {
    const int r0 = c * kUpdRows, r1 = min(P.n, r0 + kUpdRows);
    double rz = 0.0, bb = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += kFlowThreads) {
        const double bi = P.b[i];
        const double zi = P.diag ? bi / P.diag[i] : bi;
        P.x[i] = 0.0;
        P.r[i] = bi;
        P.z[i] = zi;
        P.p0[i] = zi;
        rz += bi * zi;
        bb += bi * bi;
    }
    const double2 s = flow_sum2(rz, bb, red);
    if (threadIdx.x == 0) {
        P.part[2 * c] = s.x;
        P.part[2 * c + 1] = s.y;
    }
}

// Epoch 2i + 1, rows [r0, r1): p_i = z + beta p_(i-1) (p_0 as set up), staged
// in shared memory (FP32 high and low parts for FP32 panels), q = C~_W p_i on
// the chunk's rows; partial p_i.q.  Complete patterns: 16 rows per chunk, see
// below.  Truncated patterns: a warp per row through its column list, FP32
// sums over each lane's 16 values of a 512-column step, the steps in FP64.
__device__ void flow_product(const FlowProblem& P, int it, double beta, int c, double* red, double* vstage,
                             bool staged, double* hsum, int64_t* rowoff) {
    const int r0 = c * P.prodRows, r1 = min(P.n, r0 + P.prodRows);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = P.width;
    double* pnew = flow_dir(P, it);
    const double* pold = flow_dir(P, it + 1);     // p_(i-1): the other buffer
    const bool mixed = P.vals32 != nullptr;
    float* vh = reinterpret_cast<float*>(vstage);
    float* vl = vh + w;
    // pull this chunk's panel rows towards L2 while the direction is staged
    // (rows of one cell are contiguous; each row starts 16-byte aligned and
    // holds a multiple of 16 bytes)
    for (int row = r0 + threadIdx.x; row < r1; row += kFlowThreads) {
        const int g = P.rowCell[row];
        const int nc = P.ncols[g];
        const int64_t off = P.valOff[g] + (int64_t)(row - P.wOff[g]) * nc;
        if (row - r0 < kFlowDenseRows) rowoff[row - r0] = off;    // kept for the dense product below
        const char* src = mixed ? (const char*)(P.vals32 + off) : (const char*)(P.vals64 + off);
        const unsigned bytes = (unsigned)nc * (mixed ? 4u : 8u);
        for (unsigned o = 0; o < bytes; o += 32768u)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + o), "r"(min(32768u, bytes - o))
                         : "memory");
    }
    // four columns per thread in flight: the staging is latency bound.  A
    // CTA that already staged this problem's epoch keeps it.  Every chunk
    // reads the same two vectors at about the same time, so each starts at
    // its own block of columns: the requests spread over the L2 slices
    // instead of queueing on the same lines.
    const int nblk = (w + 4 * kFlowThreads - 1) / (4 * kFlowThreads);
    for (int bi = staged ? nblk : 0; bi < nblk; ++bi) {
        const int j0 = ((bi + c) % nblk) * 4 * kFlowThreads + threadIdx.x;
        double zz[4], pp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * kFlowThreads;
            const bool live = j < P.n;
            zz[u] = live ? __ldcg((it == 0 ? P.p0 : P.z) + j) : 0.0;
            pp[u] = (live && it > 0) ? __ldcg(pold + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * kFlowThreads;
            if (j >= w) break;
            const double v = it == 0 ? zz[u] : zz[u] + beta * pp[u];
            if (mixed) {
                const float h = (float)v;
                vh[j] = h;
                vl[j] = (float)(v - (double)h);
            } else {
                vstage[j] = v;
            }
        }
    }
    if (it > 0)
        for (int row = r0 + threadIdx.x; row < r1; row += kFlowThreads)
            pnew[row] = __ldcg(P.z + row) + beta * __ldcg(pold + row);
    __syncthreads();
    double pq = 0.0;
    if (P.dense) {
        // every row holds all w columns in order.  Warps 0-3 and 4-7 take the
        // two column halves of the chunk's 16 rows, four rows per warp sharing
        // each staged column load, so a chunk is half as many dependent load
        // steps long; FP32 sums over blocks of kFlowSpan columns, FP64 across
        // blocks and halves (half 0 + half 1, in that order)
        const int step = mixed ? 256 : 128;
        const int mid = min(w, (w / 2 + step - 1) / step * step);
        const int half = warp >> 2;
        const int cb = half ? mid : 0, ce = half ? w : mid;
        const int rg = r0 + 4 * (warp & 3);
        const void* rowp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t off = rowoff[min(rg + q, r1 - 1) - r0];
            rowp[q] = mixed ? (const void*)(P.vals32 + off) : (const void*)(P.vals64 + off);
        }
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        if (rg < r1) {
            for (int jb = cb; jb < ce; jb += kFlowSpan) {
                const int je = min(ce, jb + kFlowSpan);
                if (mixed) {
                    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int j0 = jb + 4 * lane; j0 < je; j0 += 256) {
                        const int j1 = j0 + 128;
                        const bool ok1 = j1 < je;
                        float4 a0[4], a1[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float* rp = reinterpret_cast<const float*>(rowp[q]);
                            a0[q] = __ldg(reinterpret_cast<const float4*>(rp + j0));
                            a1[q] = ok1 ? __ldg(reinterpret_cast<const float4*>(rp + j1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        const float4 h0 = *reinterpret_cast<const float4*>(vh + j0);
                        const float4 l0 = *reinterpret_cast<const float4*>(vl + j0);
                        const float4 h1 = ok1 ? *reinterpret_cast<const float4*>(vh + j1) : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 l1 = ok1 ? *reinterpret_cast<const float4*>(vl + j1) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float t = sh[q];
                            t = fmaf(a0[q].x, h0.x, t); t = fmaf(a0[q].y, h0.y, t); t = fmaf(a0[q].z, h0.z, t); t = fmaf(a0[q].w, h0.w, t);
                            t = fmaf(a1[q].x, h1.x, t); t = fmaf(a1[q].y, h1.y, t); t = fmaf(a1[q].z, h1.z, t); t = fmaf(a1[q].w, h1.w, t);
                            sh[q] = t;
                            float u = sl[q];
                            u = fmaf(a0[q].x, l0.x, u); u = fmaf(a0[q].y, l0.y, u); u = fmaf(a0[q].z, l0.z, u); u = fmaf(a0[q].w, l0.w, u);
                            u = fmaf(a1[q].x, l1.x, u); u = fmaf(a1[q].y, l1.y, u); u = fmaf(a1[q].z, l1.z, u); u = fmaf(a1[q].w, l1.w, u);
                            sl[q] = u;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += (double)sh[q] + (double)sl[q];
                } else {
                    for (int j0 = jb + 4 * lane; j0 < je; j0 += 128) {
                        double2 a0[4], a1[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const double* rp = reinterpret_cast<const double*>(rowp[q]);
                            a0[q] = __ldg(reinterpret_cast<const double2*>(rp + j0));
                            a1[q] = __ldg(reinterpret_cast<const double2*>(rp + j0 + 2));
                        }
                        const double2 v0 = *reinterpret_cast<const double2*>(vstage + j0);
                        const double2 v1 = *reinterpret_cast<const double2*>(vstage + j0 + 2);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[q] += a0[q].x * v0.x + a0[q].y * v0.y + a1[q].x * v1.x + a1[q].y * v1.y;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (half == 1 && lane == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) hsum[4 * (warp & 3) + q] = acc[q];
        __syncthreads();
        if (half == 0 && lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = rg + q;
                if (row < r1) {
                    const double a = acc[q] + hsum[4 * (warp & 3) + q];
                    P.q[row] = a;
                    const double prow = it == 0 ? __ldcg(P.p0 + row) : __ldcg(P.z + row) + beta * __ldcg(pold + row);
                    pq += prow * a;
                }
            }
        }
    } else {
    for (int row = r0 + warp; row < r1; row += kFlowWarps) {
        const int g = P.rowCell[row];
        const int nc = P.ncols[g];
        const int64_t off = P.valOff[g] + (int64_t)(row - P.wOff[g]) * nc;
        const int* ci = P.colidx + P.colOff[g];
        double acc = 0.0;
        if (mixed) {
            const float* a = P.vals32 + off;
            for (int j0 = 4 * lane; j0 < nc; j0 += 512) {
                float4 v[4];
                int4 cc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + 128 * u;
                    v[u] = j < nc ? __ldg(reinterpret_cast<const float4*>(a + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    cc[u] = (P.dense || j >= nc) ? make_int4(j, j + 1, j + 2, j + 3)
                                                 : __ldg(reinterpret_cast<const int4*>(ci + j));
                }
                float sh = 0.0f, sl = 0.0f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + 128 * u >= nc) break;
                    sh = fmaf(v[u].x, vh[cc[u].x], sh);
                    sh = fmaf(v[u].y, vh[cc[u].y], sh);
                    sh = fmaf(v[u].z, vh[cc[u].z], sh);
                    sh = fmaf(v[u].w, vh[cc[u].w], sh);
                    sl = fmaf(v[u].x, vl[cc[u].x], sl);
                    sl = fmaf(v[u].y, vl[cc[u].y], sl);
                    sl = fmaf(v[u].z, vl[cc[u].z], sl);
                    sl = fmaf(v[u].w, vl[cc[u].w], sl);
                }
                acc += (double)sh + (double)sl;
            }
        } else {
            const double* a = P.vals64 + off;
            for (int j = 4 * lane; j < nc; j += 128) {
                const double2 a0 = __ldg(reinterpret_cast<const double2*>(a + j));
                const double2 a1 = __ldg(reinterpret_cast<const double2*>(a + j + 2));
                const int4 cc = P.dense ? make_int4(j, j + 1, j + 2, j + 3) : __ldg(reinterpret_cast<const int4*>(ci + j));
                acc += a0.x * vstage[cc.x] + a0.y * vstage[cc.y] + a1.x * vstage[cc.z] + a1.y * vstage[cc.w];
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            P.q[row] = acc;
            const double prow = it == 0 ? __ldcg(P.p0 + row) : __ldcg(P.z + row) + beta * __ldcg(pold + row);
            pq += prow * acc;
        }
    }
    }
    const double2 s = flow_sum2(pq, 0.0, red);
    if (threadIdx.x == 0) P.part[c] = s.x;
}

// Epoch 2i + 1 on the symmetric FP32 storage: chunk c is block b's 128 rows
// against its column segment s (kFlowSymSeg columns of its stored width,
// which starts at its own diagonal square).  Every stored value is read once
// and used twice: A[r][j] p_j goes to row r (FP32 over the segment, into
// rowpart[s][r]) and, for columns j right of the diagonal square, A[r][j] p_r
// to column j (FP32 over the block's rows, into colpart[b][j]); the update
// epoch adds the pieces of each q_r in a fixed order.  Only the block's rows
// and the segment's columns of p_i = z + beta p_(i-1) are staged (FP32 high
// and low parts, and FP64 for the partial p_i.q).  Warp w takes rows w, w +
// 8, ..., four at a time; a lane takes columns 4 lane and 128 + 4 lane of
// each 256-column step (tiles lane / 16 and 2 + lane / 16).
__device__ void flow_product_sym(const FlowProblem& P, int it, double beta, int c, double* red, double* smd) {
    const int2 item = P.symItem[c];
    const int b = item.x, sg = item.y;
    const int n = P.n;
    const int row0 = b * kSymRows, rows = min(kSymRows, n - row0);
    const int W = (int)sym_width(n, b);
    const int cs = row0 + sg * kFlowSymSeg, ce = min(row0 + W, cs + kFlowSymSeg);   // columns, multiples of 64
    const int diagEnd = row0 + kSymRows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* pnew = flow_dir(P, it);
    const double* pold = flow_dir(P, it + 1);
    // shared scratch: row and column parts of p (FP64, FP32 high, FP32 low),
    // then the eight warps' column sums of one step
    double* vrd = smd;                                   // kSymRows
    double* vcd = vrd + kSymRows;                        // kFlowSymSeg
    float* vrh = reinterpret_cast<float*>(vcd + kFlowSymSeg);
    float* vrl = vrh + kSymRows;
    float* vch = vrl + kSymRows;
    float* vcl = vch + kFlowSymSeg;
    float* cred = vcl + kFlowSymSeg;                     // 8 x 256
    const float* vb = P.symVals + P.symOff[b];
    const int64_t tstride = (int64_t)rows * kSymTile;     // values per tile
    // the segment's tiles towards L2 (each tile one contiguous block)
    if (threadIdx.x < (ce - cs) / kSymTile)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vb + ((cs - row0) / kSymTile + threadIdx.x) * tstride),
                     "r"((unsigned)(tstride * 4))
                     : "memory");
    for (int t = threadIdx.x; t < kSymRows + kFlowSymSeg; t += kFlowThreads) {
        const int j = t < kSymRows ? row0 + t : cs + (t - kSymRows);
        const bool live = t < kSymRows ? t < rows : (j < ce && j < n);
        double v = 0.0;
        if (live) v = it == 0 ? __ldcg(P.p0 + j) : __ldcg(P.z + j) + beta * __ldcg(pold + j);
        const float h = (float)v, l = (float)(v - (double)h);
        if (t < kSymRows) {
            vrd[t] = v;
            vrh[t] = h;
            vrl[t] = l;
            if (it > 0 && sg == 0 && live) pnew[j] = v;     // each row's block has one segment 0
        } else {
            vcd[t - kSymRows] = v;
            vch[t - kSymRows] = h;
            vcl[t - kSymRows] = l;
        }
    }
    __syncthreads();
    constexpr int RW = kSymRows / kFlowWarps;   // rows per warp (16)
    float racc[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) racc[k] = 0.0f;
    double pq = 0.0;
    const int j0 = 4 * lane, j1 = 128 + 4 * lane;
    for (int c0 = cs; c0 < ce; c0 += 256) {
        const int m = min(256, ce - c0);            // a multiple of 64
        const bool ok0 = j0 < m, ok1 = j1 < m;
        const int cb = c0 - cs;                     // first column of the step within the segment
        const float4 h0 = ok0 ? *reinterpret_cast<const float4*>(vch + cb + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l0 = ok0 ? *reinterpret_cast<const float4*>(vcl + cb + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 h1 = ok1 ? *reinterpret_cast<const float4*>(vch + cb + j1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l1 = ok1 ? *reinterpret_cast<const float4*>(vcl + cb + j1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float* vc0 = vb + ((c0 - row0) / kSymTile + (lane >> 4)) * tstride + 4 * (lane & 15);
        const float* vc1 = vc0 + 2 * tstride;
        float ca[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ca[k] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < RW; k0 += 4) {
            float4 a[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = min(warp + kFlowWarps * (k0 + q), rows - 1);
                a[q][0] = ok0 ? __ldg(reinterpret_cast<const float4*>(vc0 + r * kSymTile)) : make_float4(0.f, 0.f, 0.f, 0.f);
                a[q][1] = ok1 ? __ldg(reinterpret_cast<const float4*>(vc1 + r * kSymTile)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = warp + kFlowWarps * (k0 + q);
                const float4 x = a[q][0], y = a[q][1];
                float t = 0.0f;
                t = fmaf(x.x, h0.x, t); t = fmaf(x.y, h0.y, t); t = fmaf(x.z, h0.z, t); t = fmaf(x.w, h0.w, t);
                t = fmaf(y.x, h1.x, t); t = fmaf(y.y, h1.y, t); t = fmaf(y.z, h1.z, t); t = fmaf(y.w, h1.w, t);
                t = fmaf(x.x, l0.x, t); t = fmaf(x.y, l0.y, t); t = fmaf(x.z, l0.z, t); t = fmaf(x.w, l0.w, t);
                t = fmaf(y.x, l1.x, t); t = fmaf(y.y, l1.y, t); t = fmaf(y.z, l1.z, t); t = fmaf(y.w, l1.w, t);
                racc[k0 + q] += t;
                const float wh = vrh[r], wl = vrl[r];    // zero past the block's last row
                ca[0] = fmaf(x.x, wh, fmaf(x.x, wl, ca[0]));
                ca[1] = fmaf(x.y, wh, fmaf(x.y, wl, ca[1]));
                ca[2] = fmaf(x.z, wh, fmaf(x.z, wl, ca[2]));
                ca[3] = fmaf(x.w, wh, fmaf(x.w, wl, ca[3]));
                ca[4] = fmaf(y.x, wh, fmaf(y.x, wl, ca[4]));
                ca[5] = fmaf(y.y, wh, fmaf(y.y, wl, ca[5]));
                ca[6] = fmaf(y.z, wh, fmaf(y.z, wl, ca[6]));
                ca[7] = fmaf(y.w, wh, fmaf(y.w, wl, ca[7]));
            }
        }
        *reinterpret_cast<float4*>(cred + warp * 256 + j0) = make_float4(ca[0], ca[1], ca[2], ca[3]);
        *reinterpret_cast<float4*>(cred + warp * 256 + j1) = make_float4(ca[4], ca[5], ca[6], ca[7]);
        __syncthreads();
        // one thread per column right of the diagonal square: the eight warps' sums in order
        {
            const int t = threadIdx.x;
            const int col = c0 + t;
            if (t < m && col >= diagEnd && col < n) {
                float sum = 0.0f;
#pragma unroll
                for (int w8 = 0; w8 < kFlowWarps; ++w8) sum += cred[w8 * 256 + t];
                P.colpart[(int64_t)b * n + col] = sum;
                pq += vcd[cb + t] * (double)sum;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        float a = racc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const int r = warp + kFlowWarps * k;
        if (lane == 0 && r < rows) {
            P.rowpart[(int64_t)sg * n + row0 + r] = a;
            pq += vrd[r] * (double)a;
        }
    }
    const double2 s2 = flow_sum2(pq, 0.0, red);
    if (threadIdx.x == 0) P.part[c] = s2.x;
}

// Epoch 2i + 2, rows [r0, r1): x += alpha p_i, r -= alpha q, z = D^-1 r;
// partials r.r and r.z.
__device__ void flow_update(const FlowProblem& P, int it, double alpha, int c, double* red) {
    const int r0 = c * kUpdRows, r1 = min(P.n, r0 + kUpdRows);
    const double* p = flow_dir(P, it);
    double rr = 0.0, rz = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += kFlowThreads) {
        P.x[i] = __ldcg(P.x + i) + alpha * __ldcg(p + i);
        double qi;
        if (P.symVals) {
            // q_i: the row sums of its block's segments, then the column sums
            // of the blocks above it, in that order
            const int bi = i / kSymRows;
            const int ns = (int)((sym_width(P.n, bi) + kFlowSymSeg - 1) / kFlowSymSeg);
            qi = 0.0;
            for (int sgi = 0; sgi < ns; ++sgi) qi += (double)__ldcg(P.rowpart + (int64_t)sgi * P.n + i);
            for (int bb = 0; bb < bi; ++bb) qi += (double)__ldcg(P.colpart + (int64_t)bb * P.n + i);
        } else {
            qi = __ldcg(P.q + i);
        }
        const double ri = __ldcg(P.r + i) - alpha * qi;
        P.r[i] = ri;
        const double zi = P.diag ? ri / P.diag[i] : ri;
        P.z[i] = zi;
        rr += ri * ri;
        rz += ri * zi;
    }
    const double2 s = flow_sum2(rr, rz, red);
    if (threadIdx.x == 0) {
        P.part[2 * c] = s.x;
        P.part[2 * c + 1] = s.y;
    }
}

// Warp 0: the chunks' partial sums in chunk order (pairs when `pairs`).
__device__ __forceinline__ double2 flow_gather(const double* part, int nchunk, bool pairs) {
    const int lane = threadIdx.x & 31;
    double a = 0.0, b = 0.0;
    // four slots per lane loaded before any is added (the sum order stays
    // lane, lane + 32, lane + 64, ...)
    for (int c0 = lane; c0 < nchunk; c0 += 128) {
        double va[4], vb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + 32 * u;
            va[u] = c < nchunk ? __ldcg(part + (pairs ? 2 * c : c)) : 0.0;
            vb[u] = (pairs && c < nchunk) ? __ldcg(part + 2 * c + 1) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c0 + 32 * u >= nchunk) break;
            a += va[u];
            b += vb[u];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    return make_double2(a, b);
}

__device__ void flow_open(FlowCtl& C, FlowGlobal* g, unsigned e) {
    atomicExch(&C.done, 0u);
    __threadfence();
    atomicExch(&C.ticket, (unsigned long long)e << 32);
    atomicAdd(&g->progress, 1u);
}

__device__ void flow_finish(const FlowProblem& P, FlowCtl& C, FlowGlobal* g, int it, double rr, int status) {
    P.st->it = it;
    P.st->rr = rr;
    P.st->bb = C.bb;
    P.st->status = status;
    __threadfence();
    P.st->done = 1;
    atomicExch(&C.finished, 1);
    atomicSub(&g->remaining, 1);
    atomicAdd(&g->progress, 1u);
}

// The last finisher of epoch e: reduce, test, set the scalars, open e + 1.
// Run by warp 0; lane 0 writes.  Matches pcg_run: x0 = 0, stop when
// ||r_k||^2 <= tol^2 ||b||^2 on the recursive unpreconditioned residual.
__device__ void flow_transition(const FlowProblem& P, FlowCtl& C, FlowGlobal* g, unsigned e, int k) {
    const int lane = threadIdx.x & 31;
    if (e == 0) {
        const double2 s = flow_gather(P.part, P.nupd, true);
        if (lane == 0) {
            C.rz = s.x;
            C.bb = s.y;
            C.rr = s.y;
            C.it = 0;
            C.beta = 0.0;
            if (!(s.y > 0.0)) flow_finish(P, C, g, 0, s.y, ST_OK);
            else flow_open(C, g, 1u);
        }
    } else if (e & 1u) {
        const double2 s = flow_gather(P.part, P.nprod, false);
        if (lane == 0) {
            const int it = (int)((e - 1u) >> 1);
            if (!(s.x > 0.0)) {
                flow_finish(P, C, g, it, C.rr, ST_BREAKDOWN);
            } else {
                C.alpha = C.rz / s.x;
                flow_open(C, g, e + 1u);
            }
        }
    } else {
        const double2 s = flow_gather(P.part, P.nupd, true);
        if (lane == 0) {
            const int it = (int)(e >> 1);           // iterations completed
            C.rr = s.x;
            C.it = it;
            if (s.x <= P.tol2 * C.bb) {
                flow_finish(P, C, g, it, s.x, ST_OK);
            } else if (it >= P.maxit) {
                flow_finish(P, C, g, it, s.x, ST_NOCONV);
            } else {
                C.beta = s.y / C.rz;
                C.rz = s.y;
                // the problem with most iterations so far is offered first:
                // a long solve is the batch's critical path
                atomicMax(&g->hot, ((unsigned long long)it << 32) | (unsigned)k);
                flow_open(C, g, e + 1u);
            }
        }
    }
}

// Lane 0 of a searching warp: takes chunks of problem P's open epoch, if it
// has any.  A grab is about one CTA's share when the live problems split the
// grid evenly: whole epochs while hundreds of problems run (the direction is
// then staged once per CTA and epoch), single chunks once one problem is
// left, so that it spreads over the whole GPU.  Returns the number taken.
__device__ __forceinline__ unsigned flow_take(const FlowProblem& P, FlowCtl& C, unsigned live, unsigned& epoch,
                                              unsigned& chunk) {
    const unsigned long long t = *(volatile unsigned long long*)&C.ticket;
    const unsigned n0 = flow_chunks(P, (unsigned)(t >> 32));
    if ((unsigned)t >= n0) return 0;
    const unsigned long long share = (unsigned long long)n0 * live / gridDim.x;
    const unsigned m = (unsigned)min((unsigned long long)n0, max(1ull, share));
    const unsigned long long t2 = atomicAdd(&C.ticket, (unsigned long long)m);
    epoch = (unsigned)(t2 >> 32);
    chunk = (unsigned)t2;
    const unsigned n = flow_chunks(P, epoch);
    return chunk < n ? min(m, n - chunk) : 0u;
}

// All problems' PCGs in one launch.  Each CTA starts at its home problem
// (CTAs spread over the problems in proportion to their panel sizes), takes
// chunks of whatever epoch is open there, and moves on to other problems
// when none is left.  Waiting happens only while no chunk is open anywhere;
// if nothing moves for kWaitCycles the CTA sets g->err and leaves.
__global__ void __launch_bounds__(kFlowThreads, 3) batch_flow_pcg_kernel(const FlowProblem* __restrict__ probs,
                                                                      FlowCtl* ctl, int count,
                                                                      const int* __restrict__ home, FlowGlobal* g) {
    extern __shared__ __align__(16) double vstage[];
    __shared__ double red[2 * kFlowWarps];
    __shared__ int s_k, s_exit, s_last;
    __shared__ int s_stk;                  // problem and epoch whose direction is staged
    __shared__ unsigned s_ste;
    __shared__ double hsum[kFlowDenseRows];
    __shared__ int64_t rowoff[kFlowDenseRows];   // panel offsets of a dense chunk's rows
    __shared__ unsigned s_chunk, s_count, s_epoch;
    __shared__ double s_scalar;
    const int lane = threadIdx.x & 31;
    int cur = home[blockIdx.x];
    if (threadIdx.x == 0) {
        s_stk = -1;
        s_ste = 0;
    }
    bool idle = false;
    unsigned seen = 0;
    long long idle0 = 0;
    while (true) {
        if (threadIdx.x < 32) {
            int k = -1;
            unsigned chunk = 0, epoch = 0, taken = 0;
            const unsigned live = (unsigned)max(1, *(volatile int*)&g->remaining);
            {
                // the longest-running problem first
                int hk = -1;
                if (lane == 0) {
                    const unsigned long long h = *(volatile unsigned long long*)&g->hot;
                    const int kh = (int)(unsigned)(h & 0xffffffffull);
                    if (kh < count) {
                        taken = flow_take(probs[kh], ctl[kh], live, epoch, chunk);
                        if (taken) hk = kh;
                    }
                }
                k = __shfl_sync(0xffffffffu, hk, 0);
            }
            for (int base = 0; base < count && k < 0; base += 32) {
                const int j = base + lane;
                bool cand = false;
                if (j < count) {
                    // a finished problem shows no open chunk: its last epoch's
                    // chunks were all handed out
                    const int kk = (cur + j) % count;
                    const unsigned long long t = *(volatile unsigned long long*)&ctl[kk].ticket;
                    cand = (unsigned)t < flow_chunks(probs[kk], (unsigned)(t >> 32));
                }
                unsigned m = __ballot_sync(0xffffffffu, cand);
                while (m && k < 0) {
                    const int l = __ffs(m) - 1;
                    m &= m - 1;
                    const int kk = (cur + base + l) % count;
                    int got = 0;
                    if (lane == 0) {
                        taken = flow_take(probs[kk], ctl[kk], live, epoch, chunk);
                        got = taken > 0;
                    }
                    if (__shfl_sync(0xffffffffu, got, 0)) k = kk;
                }
            }
            if (k >= 0) cur = k;      // k is the same in every lane, so cur stays warp-uniform
            if (lane == 0) {
                int ex = 0;
                if (k >= 0) {
                    idle = false;
                } else if (*(volatile int*)&g->remaining <= 0 || *(volatile int*)&g->err) {
                    ex = 1;
                } else {
                    const unsigned pr = *(volatile unsigned*)&g->progress;
                    const long long now = clock64();
                    if (!idle || pr != seen) {
                        idle = true;
                        seen = pr;
                        idle0 = now;
                    } else if (now - idle0 > kWaitCycles) {
                        atomicExch(&g->err, 1);
                        ex = 1;
                    }
                    __nanosleep(256);
                }
                s_k = k;
                s_chunk = chunk;
                s_count = taken;
                s_epoch = epoch;
                s_exit = ex;
                if (k >= 0) {
                    __threadfence();
                    const FlowCtl& C = ctl[k];
                    s_scalar = (epoch & 1u) ? __ldcg(&C.beta) : __ldcg(&C.alpha);
                }
            }
        }
        __syncthreads();
        if (s_exit) break;
        const int k = s_k;
        if (k < 0) {
            __syncthreads();      // every thread has read s_k before warp 0 writes it again
            continue;
        }
        const unsigned e = s_epoch;
        const unsigned c0 = s_chunk, cnt = s_count;
        const FlowProblem& P = probs[k];
        for (unsigned c = c0; c < c0 + cnt; ++c) {
            if (e == 0) flow_init(P, (int)c, red);
            else if ((e & 1u) && P.symVals) {
                flow_product_sym(P, (int)((e - 1u) >> 1), s_scalar, (int)c, red, vstage);
            }
            else if (e & 1u) {
                const bool staged = s_stk == k && s_ste == e;
                flow_product(P, (int)((e - 1u) >> 1), s_scalar, (int)c, red, vstage, staged, hsum, rowoff);
                if (threadIdx.x == 0) {
                    s_stk = k;
                    s_ste = e;
                }
            }
            else flow_update(P, (int)((e >> 1) - 1u), s_scalar, (int)c, red);
            __syncthreads();      // s_stk, s_ste and the reduction scratch, before the next chunk
        }
        __threadfence();          // these chunks' writes, visible before they count as done
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned d = atomicAdd(&ctl[k].done, cnt);
            s_last = d + cnt == flow_chunks(P, e);
        }
        __syncthreads();
        if (s_last && threadIdx.x < 32) {
            __threadfence();
            flow_transition(P, ctl[k], g, e, k);
        }
        __syncthreads();
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
    bool flow = false;        // solved by the persistent launch
};

mlb_status setup_one(Job& j, const mlb_opts& o, cudaStream_t st) {
    mlb_batch_problem& P = *j.prob;
    mlb_status s = mlb_create(&o, &j.ctx);
    if (s != MLB_OK) return s;
    mlb_set_stream(j.ctx, st);
    s = mlb_build_basis(j.ctx, P.points, P.n, P.d, P.w);
    if (s != MLB_OK) return s;
    // the persistent launch reads the row panels of the systems it solves
    // complete patterns of the mixed path get the symmetric FP32 storage
    // (both the persistent launch and the single-problem PCG use it)
    j.ctx->allow_sym = true;
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
    if (j.flow && !hs.done) return fail(c, MLB_ETIMEOUT, "the persistent PCG stopped before this problem finished");
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
    // phase 2: every system of at most kFlowCols unknowns in one persistent
    // launch (largest first), larger ones on the stream pool meanwhile
    std::vector<int> order, big;
    for (int i = 0; i < count; ++i)
        if (jobs[i].status == MLB_OK) (jobs[i].ctx->nwav > kFlowCols ? big : order).push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].ctx->nwav > jobs[b].ctx->nwav; });
    std::vector<FlowProblem> hp;
    std::vector<double> weight;
    int64_t partTotal = 0, rowpartTotal = 0, colpartTotal = 0;
    std::vector<int2> symItems;
    std::vector<int64_t> symItemOff, rowpartOff, colpartOff;
    int maxWidth = 4;
    for (int i : order) {
        mlb_ctx* c = jobs[i].ctx;
        jobs[i].flow = true;
        FlowProblem f{};
        f.vals32 = c->pan.vals32;
        f.vals64 = c->pan.vals32 ? nullptr : c->pan.vals;
        f.colidx = c->pan.colidx;
        f.ncols = c->pan.ncols;
        f.valOff = c->pan.valOff;
        f.colOff = c->pan.colOff;
        f.rowCell = c->pan.rowCell;
        f.wOff = c->cells.wOff;
        f.diag = o.precond ? c->diag : nullptr;
        const int n = (int)c->nwav;
        f.n = n;
        f.width = (n + 3) & ~3;
        f.dense = c->pan.nnz == (int64_t)n * n ? 1 : 0;
        f.prodRows = f.dense ? kFlowDenseRows
                             : (int)std::max<int64_t>(8, std::min<int64_t>(n, kProdValues / f.width));
        f.nprod = (n + f.prodRows - 1) / f.prodRows;
        f.nupd = (n + kUpdRows - 1) / kUpdRows;
        f.b = c->vec;
        f.x = c->gW;
        f.r = c->vec + n;
        f.z = c->vec + 2 * n;
        f.p0 = c->vec + 3 * n;
        f.q = c->vec + 4 * n;
        f.p1 = c->vec + 5 * n;
        f.tol2 = o.pcg_rtol * o.pcg_rtol;
        f.maxit = o.pcg_maxit;
        f.st = c->pcg;
        if (c->sym.vals) {
            // symmetric storage: (block, segment) chunks, block by block
            f.symVals = c->sym.vals;
            f.symOff = c->sym.off;
            const int nblk = c->sym.nblk;
            symItemOff.push_back((int64_t)symItems.size());
            for (int bk = 0; bk < nblk; ++bk) {
                const int ns = (int)((sym_width(n, bk) + kFlowSymSeg - 1) / kFlowSymSeg);
                for (int sg = 0; sg < ns; ++sg) symItems.push_back(make_int2(bk, sg));
            }
            f.nprod = (int)(symItems.size() - symItemOff.back());
            rowpartOff.push_back(rowpartTotal);
            rowpartTotal += (int64_t)((sym_width(n, 0) + kFlowSymSeg - 1) / kFlowSymSeg) * n;
            colpartOff.push_back(colpartTotal);
            colpartTotal += (int64_t)nblk * n;
            maxWidth = std::max(maxWidth, kFlowSymSmem);
        } else {
            symItemOff.push_back(-1);
            rowpartOff.push_back(-1);
            colpartOff.push_back(-1);
        }
        partTotal += 2 * std::max(f.nprod, f.nupd);
        maxWidth = std::max(maxWidth, f.width);
        weight.push_back((double)(c->sym.vals ? c->sym.stored : c->pan.stored) + 1.0);
        hp.push_back(f);
    }
    mlb_status first = MLB_OK;
    FlowProblem* dp = nullptr;
    FlowCtl* dctl = nullptr;
    FlowGlobal* dg = nullptr;
    double* dpart = nullptr;
    int2* dsymItem = nullptr;
    float* drowpart = nullptr;
    float* dcolpart = nullptr;
    int* dhome = nullptr;
    cudaStream_t ps = nullptr;
    auto flow_err = [&](mlb_status st, const std::string& what) {
        if (first == MLB_OK) {
            first = st;
            g_batch_err = what;
        }
    };
    if (!hp.empty()) {
        int dev = o.device, nsm = 0, perSm = 0, optin = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t smem = sizeof(double) * (size_t)maxWidth;
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)batch_flow_pcg_kernel);
        // the process-wide opt-in is always the device maximum, so concurrent
        // calls on other host threads cannot lower it under each other
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)batch_flow_pcg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSm, batch_flow_pcg_kernel, kFlowThreads, smem);
        if (e != cudaSuccess || perSm < 1) {
            cudaGetLastError();
            flow_err(MLB_ECUDA, std::string("batch_flow_pcg_kernel setup: ") + cudaGetErrorString(e));
        }
        const int grid = std::max(1, nsm * std::max(perSm, 1));
        // CTAs start spread over the problems in proportion to their panel sizes
        std::vector<int> home(grid);
        {
            double total = 0.0;
            for (double w : weight) total += w;
            double acc = 0.0;
            int k = 0;
            for (int b = 0; b < grid; ++b) {
                const double target = (b + 0.5) / grid * total;
                while (k + 1 < (int)weight.size() && acc + weight[k] <= target) acc += weight[k++];
                home[b] = k;
            }
        }
        int64_t partOff = 0;
        if (first == MLB_OK &&
            (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess ||
             cudaMalloc(&dp, sizeof(FlowProblem) * hp.size()) != cudaSuccess ||
             cudaMalloc(&dctl, sizeof(FlowCtl) * hp.size()) != cudaSuccess ||
             cudaMalloc(&dg, sizeof(FlowGlobal)) != cudaSuccess ||
             cudaMalloc(&dpart, sizeof(double) * std::max<int64_t>(partTotal, 1)) != cudaSuccess ||
             cudaMalloc(&dsymItem, sizeof(int2) * std::max<size_t>(symItems.size(), 1)) != cudaSuccess ||
             cudaMalloc(&drowpart, sizeof(float) * std::max<int64_t>(rowpartTotal, 1)) != cudaSuccess ||
             cudaMalloc(&dcolpart, sizeof(float) * std::max<int64_t>(colpartTotal, 1)) != cudaSuccess ||
             cudaMalloc(&dhome, sizeof(int) * grid) != cudaSuccess)) {
            cudaGetLastError();
            flow_err(MLB_ENOMEM, "stream or tables for the persistent PCG");
        }
        if (first == MLB_OK) {
            for (size_t q = 0; q < hp.size(); ++q) {
                FlowProblem& f = hp[q];
                f.part = dpart + partOff;
                partOff += 2 * std::max(f.nprod, f.nupd);
                if (f.symVals) {
                    f.symItem = dsymItem + symItemOff[q];
                    f.rowpart = drowpart + rowpartOff[q];
                    f.colpart = dcolpart + colpartOff[q];
                }
            }
            FlowGlobal hg{};
            hg.remaining = (int)hp.size();
            e = cudaMemcpyAsync(dp, hp.data(), sizeof(FlowProblem) * hp.size(), cudaMemcpyHostToDevice, ps);
            if (e == cudaSuccess && !symItems.empty())
                e = cudaMemcpyAsync(dsymItem, symItems.data(), sizeof(int2) * symItems.size(), cudaMemcpyHostToDevice, ps);
            if (e == cudaSuccess) e = cudaMemsetAsync(dctl, 0, sizeof(FlowCtl) * hp.size(), ps);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dg, &hg, sizeof(FlowGlobal), cudaMemcpyHostToDevice, ps);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dhome, home.data(), sizeof(int) * grid, cudaMemcpyHostToDevice, ps);
            if (e == cudaSuccess) {
                batch_flow_pcg_kernel<<<(unsigned)grid, kFlowThreads, smem, ps>>>(dp, dctl, (int)hp.size(), dhome, dg);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) flow_err(MLB_ECUDA, std::string("batch_flow_pcg_kernel: ") + cudaGetErrorString(e));
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
        FlowGlobal hg{};
        cudaError_t e = cudaSuccess;
        if (dg) e = cudaMemcpyAsync(&hg, dg, sizeof(FlowGlobal), cudaMemcpyDeviceToHost, ps);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
        if (e != cudaSuccess) flow_err(MLB_ECUDA, std::string("batch_flow_pcg_kernel: ") + cudaGetErrorString(e));
        else if (hg.err) flow_err(MLB_ETIMEOUT, "batch_flow_pcg_kernel: no problem made progress within the wait limit");
        cudaStreamDestroy(ps);
    }
    for (void* q : {(void*)dp, (void*)dctl, (void*)dg, (void*)dpart, (void*)dsymItem, (void*)drowpart, (void*)dcolpart,
                    (void*)dhome})
        if (q) cudaFree(q);
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
