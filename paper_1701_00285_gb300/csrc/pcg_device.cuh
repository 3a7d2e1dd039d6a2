// Device helpers shared by the PCG kernels of solve.cu and symv.cu:
// deterministic block reductions and the last-CTA ("ticket") scheme that lets
// the CTA finishing a launch complete a reduction without any CTA waiting.
#pragma once

#include "internal.h"

namespace mlb {

constexpr int kVecBlocks = 512;

enum { ST_OK = 0, ST_BREAKDOWN = 1, ST_NOCONV = 2, ST_TIMEOUT = 3 };

static __device__ double block_reduce(double v) {
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

// Last-CTA reduction: every CTA taking part (`count` of them; the whole grid
// by default) has written its partial sums; each then draws a ticket, and the
// CTA that draws the last one (after a fence, so it sees every partial)
// finishes the reduction in a fixed order.  No CTA waits for another.  The
// ticket is reset for the next launch.
static __device__ bool draw_last_ticket(PcgState* st, unsigned count = 0) {
    __shared__ bool last;
    if (count == 0) count = gridDim.x;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(&st->ticket, 1u) == count - 1;
        if (last) st->ticket = 0;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// alpha = (r.z) / (p.q) from the per-CTA partials of p.q
static __device__ void pcg_alpha_finish(const double* part, int nparts, PcgState* st) {
    double a = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += __ldcg(part + i);
    const double pq = block_reduce(a);
    if (threadIdx.x) return;
    st->pq = pq;
    if (!(pq > 0.0)) {
        st->status = ST_BREAKDOWN;
        st->done = 1;
        return;
    }
    st->alpha = st->rz / pq;
}

// Part of q_i (right-hand side rhs) of the symmetric packed product: the
// slots k = first, first + step, ... of the list (row sums of the segments of
// row i's block, then column sums of the blocks above it), added in order.
static __device__ __forceinline__ double sym_q_slots(const SymPanels& S, int64_t n, int64_t i, int rhs, int first,
                                                     int step) {
    const int b = (int)(i / kSymRows);
    const int ns = sym_nseg(n, b, S.seg);
    const float* rp = S.rowpart + (int64_t)rhs * S.nsegCap * n + i;
    const float* cp = S.colpart + (int64_t)rhs * S.nblk * n + i;
    double q = 0.0;
    for (int k = first; k < ns + b; k += step) q += (double)(k < ns ? rp[(int64_t)k * n] : cp[(int64_t)(k - ns) * n]);
    return q;
}

// q_i (right-hand side rhs) of the symmetric packed product: the row sums of
// the segments of row i's block, then the column sums of the blocks above it,
// always in this order, so the result does not depend on scheduling.
static __device__ __forceinline__ double sym_q(const SymPanels& S, int64_t n, int64_t i, int rhs) {
    const int b = (int)(i / kSymRows);
    const int ns = sym_nseg(n, b, S.seg);
    const float* rp = S.rowpart + (int64_t)rhs * S.nsegCap * n + i;
    double q = 0.0;
    for (int s = 0; s < ns; ++s) q += (double)rp[(int64_t)s * n];
    const float* cp = S.colpart + (int64_t)rhs * S.nblk * n + i;
    for (int c = 0; c < b; ++c) q += (double)cp[(int64_t)c * n];
    return q;
}

}  // namespace mlb
