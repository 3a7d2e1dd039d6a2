// Sparse multilevel covariance C~_W (Sec. 4, Algorithms 4-7) on the GPU.
//
// Alg. 7 evaluates every stored entry psi^T C psi directly, which costs a
// kernel block of n_m x n_q evaluations for each admissible pair of cells at
// every level pair -- about N^2 evaluations per coarse level pair.  Here the
// same entries come from the two-scale relations of the basis (Sec. 3.1: a
// cell's scaling and wavelet vectors are [phi_L 0; 0 phi_R] V):
//
//  1. leaf pass: for every pair of leaves (f <= e), G = V_f^T C(S_f, S_e) V_e with
//     C evaluated on the fly (nugget on coinciding points).  Its
//     wavelet-wavelet part is the (t, t) block of C_W; its scaling-scaling
//     part SS and scaling-wavelet part SW feed the coarser levels;
//  2. level pass, l = t-1 .. 0: for every pair of cells (c <= d) of level l,
//     G = V_c^T H V_d where H is the 2x2 arrangement of the children's SS
//     blocks; again WW -> block (l, l) of C_W, SS and SW -> next level;
//  3. cross-level pass: for j = t .. 1 the rows of SW_j (scaling functions of
//     level j against wavelets of level j) are carried up the tree with the
//     factors V of levels j-1 .. 0; the wavelet rows that appear at level l are
//     the blocks (l, j) of C_W.
//
// The result equals psi^T C psi for every entry (same definition, different
// association order); only admissible blocks (distance criterion of Sec. 4.1,
// see the pattern kernels) are stored.  The kernel is evaluated once per pair
// of points, N^2 / 2 times in all, instead of once per pair per level pair.
//
// Storage: one dense row panel per cell (k_c rows, the admissible blocks side
// by side in global column order) plus one column-index list per panel.
#include <algorithm>
#include <cmath>
#include <utility>

#include "internal.h"
#include "ff.cuh"
#include "matern.cuh"

namespace mlb {

struct PatArgs {
    const double* lo;
    const double* hi;
    const double* diam;
    int d;
    int inf;
    double c;
};

// Distance criterion (Sec. 4.1): the box of q's points meets the box of m's
// points grown by tau_{i,j} = c sqrt(Dbar_i Dbar_j) on every axis, Dbar_l the
// mean box diagonal of level l (the cell tables carry it per cell).  The test
// is symmetric in m and q.
__device__ __forceinline__ bool admissible(const PatArgs& P, int gm, int gq) {
    if (P.inf) return true;
    const double tau = __dmul_rn(P.c, sqrt(__dmul_rn(P.diam[gm], P.diam[gq])));
    for (int k = 0; k < P.d; ++k) {
        if (__dsub_rn(P.lo[gq * P.d + k], P.hi[gm * P.d + k]) > tau) return false;
        if (__dsub_rn(P.lo[gm * P.d + k], P.hi[gq * P.d + k]) > tau) return false;
    }
    return true;
}

__global__ void count_kernel(PatArgs P, CellTables C, int ncell, int* ncols, int* nblk) {
    const int gm = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gm >= ncell) return;
    int cols = 0, nb = 0;
    if (C.k[gm] > 0) {
        for (int gq = lane; gq < ncell; gq += 32) {
            const int kq = C.k[gq];
            if (kq > 0 && admissible(P, gm, gq)) {
                cols += kq;
                nb += 1;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cols += __shfl_xor_sync(0xffffffffu, cols, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if (lane == 0) {
        ncols[gm] = cols;
        nblk[gm] = nb;
    }
}

// Column lists and the block-column table, columns in global wavelet order.
__global__ void fill_kernel(PatArgs P, CellTables C, int ncell, const int* __restrict__ colOrder,
                            Panels pan) {
    const int gm = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gm >= ncell) return;
    const bool rowOk = C.k[gm] > 0;
    int base = 0;
    int* brow = pan.bcol + (int64_t)gm * ncell;
    int* cols = pan.colidx + (rowOk ? pan.colOff[gm] : 0);
    for (int q0 = 0; q0 < ncell; q0 += 32) {
        const int q = q0 + lane;
        int gq = -1, kk = 0;
        bool ok = false;
        if (q < ncell) {
            gq = colOrder[q];
            const int kq = C.k[gq];
            ok = rowOk && kq > 0 && admissible(P, gm, gq);
            kk = ok ? kq : 0;
        }
        int incl = kk;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = base + incl - kk;
        if (q < ncell) {
            brow[gq] = ok ? excl : -1;
            if (ok) {
                const int64_t w0 = C.wOff[gq];
                for (int i = 0; i < kk; ++i) cols[excl + i] = (int)(w0 + i);
            }
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

struct TileOut {
    double* SS;          // this level's SS matrix (sumA x sumA, row-major)
    double* SW;          // this level's SW matrix (sumA x sumK, row-major)
    int64_t ldSS, ldSW;
    Panels pan;
    int ncell;
};

struct TileIn {
    const double* V;     // pool of the cells' orthogonal factors
    // leaf pass: kernel block on the fly
    const double* xs;
    const float* xl32;   // mixed: offsets of the points from their leaf's centre, FP32 high part
    const float* xl32lo; //        and low part (offset = high + low to about 1e-14)
    const double* ctr;   // mixed: leaf centres (ncell x d)
    int d;
    KernelFn K;          // the covariance function
    double nugget;
    double sc[kMaxDim];  // per-axis distance scales (FP64 coordinates are scaled as loaded)
    // level pass: children's SS matrix
    const double* SSc;
    int64_t ldSSc;
};

__device__ __forceinline__ void unrank_pair(int64_t pi, int& f, int& e) {
    int64_t ee = (int64_t)((sqrt(8.0 * (double)pi + 1.0) - 1.0) * 0.5);
    while ((ee + 1) * (ee + 2) / 2 <= pi) ++ee;
    while (ee * (ee + 1) / 2 > pi) --ee;
    e = (int)ee;
    f = (int)(pi - ee * (ee + 1) / 2);
}

// Writes one entry G[r][c] of the pair (f, e) of one level to SS, SW and the
// panels, with the mirrored copies for f != e.
__device__ __forceinline__ void put_entry(const CellTables& C, const TileOut& o, int gf, int ge,
                                          bool diagPair, int af, int ae, int r, int c, double v) {
    if (r < af) {
        if (c < ae) {
            o.SS[(C.sOff[gf] + r) * o.ldSS + C.sOff[ge] + c] = v;
            if (!diagPair) o.SS[(C.sOff[ge] + c) * o.ldSS + C.sOff[gf] + r] = v;
        } else {
            o.SW[(C.sOff[gf] + r) * o.ldSW + C.wLoc[ge] + (c - ae)] = v;
        }
    } else if (c < ae) {
        if (!diagPair) o.SW[(C.sOff[ge] + c) * o.ldSW + C.wLoc[gf] + (r - af)] = v;
    } else {
        const int bc = o.pan.bcol[(int64_t)gf * o.ncell + ge];
        if (bc >= 0) {
            o.pan.vals[o.pan.valOff[gf] + (int64_t)(r - af) * o.pan.ncols[gf] + bc + (c - ae)] = v;
            if (!diagPair) {
                const int bt = o.pan.bcol[(int64_t)ge * o.ncell + gf];
                o.pan.vals[o.pan.valOff[ge] + (int64_t)(c - ae) * o.pan.ncols[ge] + bt + (r - af)] = v;
            }
        }
    }
}

// G = V_f^T H V_e for every pair f <= e of one level (tiles up to 64 x 64,
// 256 threads, 4 x 4 register micro-tiles), FP64.  H is the covariance block
// of the two leaves (LEAF) or the children's SS blocks (coarser levels).
template <bool LEAF>
__global__ void __launch_bounds__(256) galerkin_tile_kernel(CellTables C, int level, int64_t npairs,
                                                            TileIn in, TileOut out) {
    constexpr int S = kTile;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* Vf = reinterpret_cast<double*>(smraw);
    double* Ve = Vf + S * S;
    double* P = Ve + S * S;
    double* xf = P + S * S;
    double* xe = xf + S * kMaxDim;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int r0 = ty * 4, c0 = tx * 4;
    const int first = (1 << level) - 1;
    for (int64_t pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
        int f, e;
        unrank_pair(pi, f, e);
        const int gf = first + f, ge = first + e;
        const int sf = C.s[gf], se = C.s[ge], af = C.a[gf], ae = C.a[ge];
        const double* gVf = in.V + C.vOff[gf];
        const double* gVe = in.V + C.vOff[ge];
        for (int idx = tid; idx < S * S; idx += 256) {
            const int r = idx / S, c = idx % S;
            Vf[idx] = (r < sf && c < sf) ? gVf[r * sf + c] : 0.0;
            Ve[idx] = (r < se && c < se) ? gVe[r * se + c] : 0.0;
        }
        if (LEAF) {
            const int d = in.d;
            const int64_t bf = C.beg[gf], be = C.beg[ge];
            for (int idx = tid; idx < sf * d; idx += 256) xf[idx] = in.xs[bf * d + idx] * in.sc[idx % d];
            for (int idx = tid; idx < se * d; idx += 256) xe[idx] = in.xs[be * d + idx] * in.sc[idx % d];
        }
        __syncthreads();
        if (LEAF) {
            const int d = in.d;
            for (int idx = tid; idx < S * S; idx += 256) {
                const int r = idx / S, c = idx % S;
                double v = 0.0;
                if (r < sf && c < se) {
                    double r2 = 0.0;
                    for (int k = 0; k < d; ++k) {
                        const double df = xf[r * d + k] - xe[c * d + k];
                        r2 += df * df;
                    }
                    v = kern_f64<false>(sqrt(r2), in.K);
                    if (gf == ge && r == c) v += in.nugget;
                }
                P[idx] = v;
            }
        } else {
            const int64_t row0 = C.sOff[2 * gf + 1], col0 = C.sOff[2 * ge + 1];
            for (int idx = tid; idx < S * S; idx += 256) {
                const int r = idx / S, c = idx % S;
                P[idx] = (r < sf && c < se) ? in.SSc[(row0 + r) * in.ldSSc + col0 + c] : 0.0;
            }
        }
        __syncthreads();
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k = 0; k < S; ++k) {
            double a4[4], b4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a4[i] = P[(r0 + i) * S + k];
#pragma unroll
            for (int j = 0; j < 4; ++j) b4[j] = Ve[k * S + c0 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a4[i] * b4[j];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) P[(r0 + i) * S + c0 + j] = acc[i][j];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k = 0; k < S; ++k) {
            double a4[4], b4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a4[i] = Vf[k * S + r0 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b4[j] = P[k * S + c0 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a4[i] * b4[j];
        }
        const bool diagPair = (gf == ge);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = r0 + i, c = c0 + j;
                if (r < sf && c < se) put_entry(C, out, gf, ge, diagPair, af, ae, r, c, acc[i][j]);
            }
        __syncthreads();
    }
}

// Coarse levels: G = V_f^T H V_e with H the children's SS block, for cells
// of at most SM <= 32 basis vectors (s = a_left + a_right <= 2p).  A group of
// SM*SM/8 threads owns one pair and each thread a 2 x 4 micro-tile, so one
// 256-thread CTA works on 256 / (SM*SM/8) pairs at once (8 at SM = 16, 2 at
// SM = 32) instead of padding every pair to a 64 x 64 tile.  The sums run
// over the pair's own sizes, in the same order as the padded kernel.
template <int SM>
__global__ void __launch_bounds__(256) galerkin_level_kernel(CellTables C, int level, int64_t npairs,
                                                             TileIn in, TileOut out) {
    constexpr int G = SM * SM / 8;        // threads per pair
    constexpr int PPC = 256 / G;          // pairs per CTA
    constexpr int CG = SM / 4;            // column groups of a micro-tile row
    extern __shared__ __align__(16) unsigned char smraw[];
    const int grp = threadIdx.x / G, t = threadIdx.x % G;
    double* Vf = reinterpret_cast<double*>(smraw) + grp * 3 * SM * SM;
    double* Ve = Vf + SM * SM;
    double* P = Ve + SM * SM;
    const int r0 = 2 * (t / CG), c0 = 4 * (t % CG);
    const int first = (1 << level) - 1;
    for (int64_t base = (int64_t)blockIdx.x * PPC; base < npairs; base += (int64_t)gridDim.x * PPC) {
        const int64_t pi = base + grp;
        const bool live = pi < npairs;
        int gf = first, ge = first, sf = 0, se = 0, af = 0, ae = 0;
        if (live) {
            int f, e;
            unrank_pair(pi, f, e);
            gf = first + f;
            ge = first + e;
            sf = C.s[gf];
            se = C.s[ge];
            af = C.a[gf];
            ae = C.a[ge];
            const double* gVf = in.V + C.vOff[gf];
            const double* gVe = in.V + C.vOff[ge];
            const int64_t row0 = C.sOff[2 * gf + 1], col0 = C.sOff[2 * ge + 1];
            for (int idx = t; idx < SM * SM; idx += G) {
                const int r = idx / SM, c = idx % SM;
                Vf[idx] = (r < sf && c < sf) ? gVf[r * sf + c] : 0.0;
                Ve[idx] = (r < se && c < se) ? gVe[r * se + c] : 0.0;
                P[idx] = (r < sf && c < se) ? in.SSc[(row0 + r) * in.ldSSc + col0 + c] : 0.0;
            }
        }
        __syncthreads();
        double acc[2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k = 0; k < se; ++k) {      // T = H V_e
            const double a0 = P[r0 * SM + k], a1 = P[(r0 + 1) * SM + k];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double b = Ve[k * SM + c0 + j];
                acc[0][j] += a0 * b;
                acc[1][j] += a1 * b;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                P[(r0 + i) * SM + c0 + j] = acc[i][j];
                acc[i][j] = 0.0;
            }
        __syncthreads();
        for (int k = 0; k < sf; ++k) {      // G = V_f^T T
            const double a0 = Vf[k * SM + r0], a1 = Vf[k * SM + r0 + 1];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double b = P[k * SM + c0 + j];
                acc[0][j] += a0 * b;
                acc[1][j] += a1 * b;
            }
        }
        if (live) {
            const bool diagPair = (gf == ge);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = r0 + i, c = c0 + j;
                    if (r < sf && c < se) put_entry(C, out, gf, ge, diagPair, af, ae, r, c, acc[i][j]);
                }
        }
        __syncthreads();
    }
}

// Mixed leaf pass: G = V_f^T Phi V_e on the FP32 pipes.  Phi is evaluated in
// double-float (ff.cuh): coordinates as double-float offsets from the leaf
// centres plus the double-float difference of the two centres, distance,
// square root, exponential and polynomial in double-float.  Both contractions
// run on split operands (Phi = Phi_hi + Phi_lo, V = V_hi + V_lo, T = T_hi +
// T_lo): the leading products in a cascaded FP32 sum (Sum2), their rounding
// errors (Dekker's TwoProduct, one FMA each) and the cross terms in plain FP32
// sums.  Rounding V or Phi to one FP32 number would perturb the
// wavelet entries at the 1e-7 level of the smooth part of Phi, which the
// vanishing moments otherwise cancel.  The nugget is added in FP64 to G's
// diagonal (V is orthogonal).
__global__ void __launch_bounds__(256) galerkin_leaf_f32_kernel(CellTables C, int level, int64_t npairs,
                                                                TileIn in, TileOut out) {
    constexpr int S = kTile;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* Vfh = reinterpret_cast<float*>(smraw);
    float* Vfl = Vfh + S * S;
    float* Veh = Vfl + S * S;
    float* Vel = Veh + S * S;
    float* P = Vel + S * S;       // Phi_hi, then T_hi
    float* Pl = P + S * S;        // Phi_lo, then T_lo
    // the coordinates live in the V buffers until Phi is formed
    float* xfh = Vfh;
    float* xfl = Vfh + S * kMaxDim;
    float* xeh = Veh;
    float* xel = Veh + S * kMaxDim;
    __shared__ float dch[kMaxDim], dcl[kMaxDim];
    __shared__ float2 tab[64];
    ff_fill_exp2_table(tab);
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int r0 = ty * 4, c0 = tx * 4;
    const int first = (1 << level) - 1;
    const ff scale = ff_from_double(in.K.scale);
    for (int64_t pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
        int f, e;
        unrank_pair(pi, f, e);
        const int gf = first + f, ge = first + e;
        const int sf = C.s[gf], se = C.s[ge], af = C.a[gf], ae = C.a[ge];
        const int d = in.d;
        const int64_t bf = C.beg[gf], be = C.beg[ge];
        for (int idx = tid; idx < sf * d; idx += 256) {
            xfh[idx] = in.xl32[bf * d + idx];
            xfl[idx] = in.xl32lo[bf * d + idx];
        }
        for (int idx = tid; idx < se * d; idx += 256) {
            xeh[idx] = in.xl32[be * d + idx];
            xel[idx] = in.xl32lo[be * d + idx];
        }
        if (tid < d) {
            const ff dc = ff_from_double(in.ctr[gf * d + tid] - in.ctr[ge * d + tid]);
            dch[tid] = dc.h;
            dcl[tid] = dc.l;
        }
        __syncthreads();
        for (int idx = tid; idx < S * S; idx += 256) {
            const int r = idx / S, c = idx % S;
            ff v = {0.0f, 0.0f};
            if (r < sf && c < se) {
                ff r2 = {0.0f, 0.0f};
                for (int k = 0; k < d; ++k) {
                    ff df = ff_two_sum(xfh[r * d + k], -xeh[c * d + k]);
                    df = ff_add(df, {__fsub_rn(xfl[r * d + k], xel[c * d + k]), 0.0f});
                    df = ff_add(df, {dch[k], dcl[k]});
                    r2 = ff_add(r2, ff_mul(df, df));
                }
                v = ff_kern<false>(ff_sqrt(r2), in.K, scale, tab);
            }
            P[idx] = v.h;
            Pl[idx] = v.l;
        }
        __syncthreads();
        const double* gVf = in.V + C.vOff[gf];
        const double* gVe = in.V + C.vOff[ge];
        for (int idx = tid; idx < S * S; idx += 256) {
            const int r = idx / S, c = idx % S;
            const double vf = (r < sf && c < sf) ? gVf[r * sf + c] : 0.0;
            const double ve = (r < se && c < se) ? gVe[r * se + c] : 0.0;
            const float vfh = (float)vf, veh = (float)ve;
            Vfh[idx] = vfh;
            Vfl[idx] = (float)(vf - (double)vfh);
            Veh[idx] = veh;
            Vel[idx] = (float)(ve - (double)veh);
        }
        __syncthreads();
        // T = (Phi_hi + Phi_lo)(V_hi + V_lo)
        float ah[4][4], ac[4][4], al[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ah[i][j] = ac[i][j] = al[i][j] = 0.0f;
        for (int k = 0; k < S; ++k) {
            float a4[4], a4l[4], bh[4], bl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a4[i] = P[(r0 + i) * S + k];
                a4l[i] = Pl[(r0 + i) * S + k];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bh[j] = Veh[k * S + c0 + j];
                bl[j] = Vel[k * S + c0 + j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float pr = __fmul_rn(a4[i], bh[j]);
                    sum2_add(ah[i][j], ac[i][j], pr);
                    // rounding error of the product (TwoProduct) and the cross terms
                    al[i][j] = fmaf(a4[i], bl[j], fmaf(a4l[i], bh[j], __fadd_rn(al[i][j], fmaf(a4[i], bh[j], -pr))));
                }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                P[(r0 + i) * S + c0 + j] = ah[i][j];
                Pl[(r0 + i) * S + c0 + j] = __fadd_rn(al[i][j], ac[i][j]);
            }
        __syncthreads();
        // G = (V_hi + V_lo)^T (T_hi + T_lo)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ah[i][j] = ac[i][j] = al[i][j] = 0.0f;
        for (int k = 0; k < S; ++k) {
            float uh[4], ul[4], th[4], tl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uh[i] = Vfh[k * S + r0 + i];
                ul[i] = Vfl[k * S + r0 + i];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                th[j] = P[k * S + c0 + j];
                tl[j] = Pl[k * S + c0 + j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float pr = __fmul_rn(uh[i], th[j]);
                    sum2_add(ah[i][j], ac[i][j], pr);
                    al[i][j] = fmaf(uh[i], tl[j], fmaf(ul[i], th[j], __fadd_rn(al[i][j], fmaf(uh[i], th[j], -pr))));
                }
        }
        const bool diagPair = (gf == ge);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = r0 + i, c = c0 + j;
                if (r < sf && c < se) {
                    double v = (double)ah[i][j] + ((double)al[i][j] + (double)ac[i][j]);
                    if (diagPair && r == c) v += in.nugget;
                    put_entry(C, out, gf, ge, diagPair, af, ae, r, c, v);
                }
            }
        __syncthreads();
    }
}

__global__ void to_f32_kernel(const double* __restrict__ src, int64_t n, float* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// One step of the cross-level pass: rows of X_{l+1} (scaling functions of
// level l+1 against the wavelets of level j) -> V_c^T per cell c of level l.
// Scaling rows go to X_l, wavelet rows are the blocks (c, e) of C_W.
__global__ void __launch_bounds__(128) cross_kernel(CellTables C, const double* __restrict__ Vpool,
                                                    int level, int jlevel, const double* __restrict__ Xin,
                                                    double* __restrict__ Xout, int64_t ldX,
                                                    int64_t levelBaseJ, Panels pan, int ncell) {
    extern __shared__ double sm[];
    const int g = (1 << level) - 1 + blockIdx.x;
    const int s = C.s[g], a = C.a[g];
    double* Vc = sm;
    double* inb = Vc + s * s;
    const int tid = threadIdx.x;
    const int64_t col = (int64_t)blockIdx.y * 128 + tid;
    const double* gV = Vpool + C.vOff[g];
    for (int idx = tid; idx < s * s; idx += 128) Vc[idx] = gV[idx];
    const int64_t row0 = C.sOff[2 * g + 1];
    if (col < ldX)
        for (int i = 0; i < s; ++i) inb[i * 128 + tid] = Xin[(row0 + i) * ldX + col];
    __syncthreads();
    if (col >= ldX) return;
    const int ge = pan.rowCell[levelBaseJ + col];
    const int cl = (int)(levelBaseJ + col - C.wOff[ge]);
    const int bc = pan.bcol[(int64_t)g * ncell + ge];
    const int bt = bc >= 0 ? pan.bcol[(int64_t)ge * ncell + g] : -1;
    for (int j = 0; j < s; ++j) {
        if (j >= a && bc < 0) break;
        double acc = 0.0;
        for (int i = 0; i < s; ++i) acc += Vc[i * s + j] * inb[i * 128 + tid];
        if (j < a) {
            if (level > 0) Xout[(C.sOff[g] + j) * ldX + col] = acc;
        } else {
            pan.vals[pan.valOff[g] + (int64_t)(j - a) * pan.ncols[g] + bc + cl] = acc;
            pan.vals[pan.valOff[ge] + (int64_t)cl * pan.ncols[ge] + bt + (j - a)] = acc;
        }
    }
}

__global__ void diag_kernel(CellTables C, Panels pan, int ncell, int64_t nwav, double* diag) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nwav) return;
    const int g = pan.rowCell[r];
    const int i = (int)(r - C.wOff[g]);
    const int bc = pan.bcol[(int64_t)g * ncell + g];
    diag[r] = pan.vals[pan.valOff[g] + (int64_t)i * pan.ncols[g] + bc + i];
}

mlb_status assemble_dev(mlb_ctx* ctx) {
    cudaStream_t st = ctx->stream;
    const int ncell = ctx->ncell, t = ctx->t;
    PatArgs P;
    P.lo = ctx->cells.lo;
    P.hi = ctx->cells.hi;
    P.diam = ctx->cells.diam;
    P.d = ctx->d;
    P.inf = std::isinf(ctx->tau_factor) ? 1 : 0;
    P.c = P.inf ? 0.0 : ctx->tau_factor;
    Panels& pan = ctx->pan;
    mlb::Arena& A = ctx->arena_asm;
    pan.ncols = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    int* nblk = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    pan.valOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    pan.colOff = (int64_t*)dalloc(ctx, A, sizeof(int64_t) * ncell);
    pan.bcol = (int*)dalloc(ctx, A, sizeof(int) * (size_t)ncell * ncell);
    int* colOrder = (int*)dalloc(ctx, A, sizeof(int) * ncell);
    if (!pan.ncols || !nblk || !pan.valOff || !pan.colOff || !pan.bcol || !colOrder) return MLB_ENOMEM;
    const unsigned wb = (unsigned)((ncell * 32 + 255) / 256);
    count_kernel<<<wb, 256, 0, st>>>(P, ctx->cells, ncell, pan.ncols, nblk);
    MLB_CHECK_LAUNCH(ctx, "count_kernel");
    std::vector<int> hn(ncell), hb(ncell), order;
    MLB_CUDA(ctx, cudaMemcpyAsync(hn.data(), pan.ncols, sizeof(int) * ncell, cudaMemcpyDeviceToHost, st));
    MLB_CUDA(ctx, cudaMemcpyAsync(hb.data(), nblk, sizeof(int) * ncell, cudaMemcpyDeviceToHost, st));
    MLB_CUDA(ctx, cudaStreamSynchronize(st));
    // panels padded to a width that is a multiple of 4 (zero values, column 0)
    // so that every row starts 16-byte aligned for the vector loads of the SpMV
    std::vector<int64_t> vo(ncell), co(ncell);
    std::vector<int> padded(ncell);
    int64_t nnz = 0, stored = 0, ctot = 0, blocks = 0;
    for (int g = 0; g < ncell; ++g) {
        padded[g] = ctx->hcells[g].k > 0 ? (hn[g] + 3) & ~3 : 0;
        vo[g] = stored;
        co[g] = ctot;
        nnz += (int64_t)ctx->hcells[g].k * hn[g];
        stored += (int64_t)ctx->hcells[g].k * padded[g];
        ctot += padded[g];
        blocks += hb[g];
    }
    for (int l = t; l >= 0; --l)
        for (int k = 0; k < (1 << l); ++k) order.push_back((1 << l) - 1 + k);
    pan.nnz = nnz;
    int64_t selfEntries = 0;
    for (int g = 0; g < ncell; ++g) selfEntries += (int64_t)ctx->hcells[g].k * ctx->hcells[g].k;
    pan.nnzUnique = (nnz + selfEntries) / 2;
    pan.colTotal = ctot;
    pan.blocks = blocks;
    pan.stored = stored;
    pan.colidx = (int*)dalloc(ctx, A, sizeof(int) * (ctot > 0 ? ctot : 1));
    pan.vals = (double*)dalloc(ctx, A, sizeof(double) * (stored > 0 ? stored : 1));
    ctx->diag = (double*)dalloc(ctx, A, sizeof(double) * ctx->nwav);
    if (!pan.colidx || !pan.vals || !ctx->diag) return MLB_ENOMEM;
    MLB_CUDA(ctx, cudaMemsetAsync(pan.colidx, 0, sizeof(int) * (ctot > 0 ? ctot : 1), st));
    MLB_CUDA(ctx, cudaMemsetAsync(pan.vals, 0, sizeof(double) * (stored > 0 ? stored : 1), st));
    MLB_CUDA(ctx, cudaMemcpyAsync(pan.ncols, padded.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, st));
    MLB_CUDA(ctx, cudaMemcpyAsync(pan.valOff, vo.data(), sizeof(int64_t) * ncell, cudaMemcpyHostToDevice, st));
    MLB_CUDA(ctx, cudaMemcpyAsync(pan.colOff, co.data(), sizeof(int64_t) * ncell, cudaMemcpyHostToDevice, st));
    MLB_CUDA(ctx, cudaMemcpyAsync(colOrder, order.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, st));
    fill_kernel<<<wb, 256, 0, st>>>(P, ctx->cells, ncell, colOrder, pan);
    MLB_CHECK_LAUNCH(ctx, "fill_kernel");

    // per-level SS / SW matrices
    std::vector<double*> SS(t + 1), SW(t + 1);
    for (int l = 0; l <= t; ++l) {
        SS[l] = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(1, ctx->sumA[l] * ctx->sumA[l]));
        SW[l] = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(1, ctx->sumA[l] * ctx->sumK[l]));
        if (!SS[l] || !SW[l]) return MLB_ENOMEM;
    }
    const bool mixed = ctx->opts.precision == MLB_MIXED;
    const size_t shm = sizeof(double) * (3 * kTile * kTile + 2 * kTile * kMaxDim);
    const size_t shm32 = sizeof(float) * (6 * kTile * kTile);
    MLB_CUDA(ctx, cudaFuncSetAttribute(galerkin_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    MLB_CUDA(ctx, cudaFuncSetAttribute(galerkin_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    MLB_CUDA(ctx, cudaFuncSetAttribute(galerkin_leaf_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm32));
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TileIn in{};
    in.V = ctx->V;
    in.xs = ctx->xs;
    in.xl32 = ctx->kxl32;
    in.xl32lo = ctx->kxl32lo;
    in.ctr = ctx->kctr;
    in.d = ctx->d;
    in.K = ctx->kfn;
    for (int c = 0; c < kMaxDim; ++c) in.sc[c] = ctx->kgeo.sc[c];
    in.nugget = ctx->theta.nugget;
    for (int l = t; l >= 0; --l) {
        TileOut o;
        o.SS = SS[l];
        o.SW = SW[l];
        o.ldSS = ctx->sumA[l];
        o.ldSW = ctx->sumK[l];
        o.pan = pan;
        o.ncell = ncell;
        const int64_t L = 1LL << l;
        const int64_t npairs = L * (L + 1) / 2;
        const unsigned grid = (unsigned)std::min<int64_t>(npairs, (int64_t)nsm * 16);
        if (l == t) {
            if (mixed) {
                const unsigned g32 = (unsigned)std::min<int64_t>(npairs, (int64_t)nsm * 32);
                galerkin_leaf_f32_kernel<<<g32, 256, shm32, st>>>(ctx->cells, l, npairs, in, o);
            } else {
                galerkin_tile_kernel<true><<<grid, 256, shm, st>>>(ctx->cells, l, npairs, in, o);
            }
        } else {
            in.SSc = SS[l + 1];
            in.ldSSc = ctx->sumA[l + 1];
            int smax = 0;
            for (int64_t k = 0; k < L; ++k) smax = std::max(smax, ctx->hcells[L - 1 + k].s);
            // small coarse cells: several pairs per CTA at their own size
            const size_t lshm = sizeof(double) * 3 * 256 * 8;    // 3 SM^2 doubles per pair, 256/(SM^2/8) pairs
            if (smax <= 16) {
                const unsigned lg = (unsigned)std::min<int64_t>((npairs + 7) / 8, (int64_t)nsm * 16);
                galerkin_level_kernel<16><<<lg, 256, lshm, st>>>(ctx->cells, l, npairs, in, o);
            } else if (smax <= 32) {
                const unsigned lg = (unsigned)std::min<int64_t>((npairs + 1) / 2, (int64_t)nsm * 16);
                galerkin_level_kernel<32><<<lg, 256, lshm, st>>>(ctx->cells, l, npairs, in, o);
            } else {
                galerkin_tile_kernel<false><<<grid, 256, shm, st>>>(ctx->cells, l, npairs, in, o);
            }
        }
        MLB_CHECK_LAUNCH(ctx, "galerkin_tile_kernel");
    }
    // cross-level pass
    int smax = 0;
    for (auto& c : ctx->hcells) smax = std::max(smax, c.s);
    const size_t cshm = sizeof(double) * ((size_t)smax * smax + (size_t)smax * 128);
    // the opt-in limit is a process-wide property of the kernel: contexts on
    // other host threads would race on a per-context value, so every context
    // requests the device maximum
    {
        mlb_status ss = allow_max_dynamic_smem(ctx, (const void*)cross_kernel, "cross_kernel smem");
        if (ss != MLB_OK) return ss;
    }
    int64_t maxX = 0;
    for (int j = t; j >= 1; --j) maxX = std::max(maxX, ctx->sumA[j - 1] * ctx->sumK[j]);
    double* X0 = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(1, maxX));
    double* X1 = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(1, maxX));
    if (!X0 || !X1) return MLB_ENOMEM;
    for (int j = t; j >= 1; --j) {
        const int64_t ldX = ctx->sumK[j];
        if (ldX == 0) continue;
        const double* xin = SW[j];
        double* bufs[2] = {X0, X1};
        int which = 0;
        for (int l = j - 1; l >= 0; --l) {
            dim3 grid(1u << l, (unsigned)((ldX + 127) / 128));
            cross_kernel<<<grid, 128, cshm, st>>>(ctx->cells, ctx->V, l, j, xin, bufs[which], ldX,
                                                  ctx->levelBase[j], pan, ncell);
            MLB_CHECK_LAUNCH(ctx, "cross_kernel");
            xin = bufs[which];
            which ^= 1;
        }
    }
    diag_kernel<<<(unsigned)((ctx->nwav + 255) / 256), 256, 0, st>>>(ctx->cells, pan, ncell, ctx->nwav, ctx->diag);
    MLB_CHECK_LAUNCH(ctx, "diag_kernel");
    // the SS / SW work matrices are no longer needed
    for (int l = 0; l <= t; ++l) {
        dfree(ctx, A, SS[l]);
        dfree(ctx, A, SW[l]);
    }
    dfree(ctx, A, X0);
    dfree(ctx, A, X1);
    if (mixed) {
        // complete pattern: each symmetric pair stored once in FP32 (symv.cu)
        bool complete = ctx->allow_sym && ctx->nwav > 0;
        for (int g = 0; g < ncell && complete; ++g)
            if (ctx->hcells[g].k > 0 && hn[g] != ctx->nwav) complete = false;
        if (complete) {
            mlb_status ss = build_sym(ctx);
            if (ss != MLB_OK) return ss;
            dfree(ctx, A, pan.vals);
            pan.vals = nullptr;
            return MLB_OK;
        }
        // otherwise the mixed path keeps the row panels in FP32: half the
        // bytes of the FP64 panels per product.  Its
        // product runs one CTA per kItemRows rows x kSegCols columns of a
        // panel, heaviest items first, so the last wave of CTAs is short.
        std::vector<std::pair<int64_t, int4>> items;
        std::vector<int> nseg(ncell, 0);
        int nsegMax = 1;
        for (int g = 0; g < ncell; ++g) {
            if (ctx->hcells[g].k == 0) continue;
            nseg[g] = (padded[g] + kSegCols - 1) / kSegCols;
            nsegMax = std::max(nsegMax, nseg[g]);
            for (int r = 0; r < ctx->hcells[g].k; r += kItemRows)
                for (int sg = 0; sg < nseg[g]; ++sg) {
                    const int cb = sg * kSegCols;
                    const int64_t w = (int64_t)std::min(kItemRows, ctx->hcells[g].k - r) *
                                      std::min(kSegCols, padded[g] - cb);
                    items.push_back({-w, make_int4(g, r, cb, sg)});
                }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, int4>& x, const std::pair<int64_t, int4>& y) {
                             return x.first < y.first;
                         });
        std::vector<int4> work;
        for (auto& it : items) work.push_back(it.second);
        if (work.size() > max_work_items(ncell, ctx->N)) return fail(ctx, MLB_EINVAL, "work table bound");
        pan.nwork = (int)work.size();
        pan.nsegMax = nsegMax;
        pan.work = (int4*)dalloc(ctx, A, sizeof(int4) * std::max<size_t>(1, work.size()));
        pan.nseg = (int*)dalloc(ctx, A, sizeof(int) * ncell);
        pan.ypart = (double*)dalloc(ctx, A, sizeof(double) * std::max<int64_t>(1, (int64_t)nsegMax * ctx->nwav));
        if (!pan.work || !pan.nseg || !pan.ypart) return MLB_ENOMEM;
        MLB_CUDA(ctx, cudaMemcpyAsync(pan.work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice, st));
        MLB_CUDA(ctx, cudaMemcpyAsync(pan.nseg, nseg.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, st));
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        pan.vals32 = (float*)dalloc(ctx, A, sizeof(float) * std::max<int64_t>(1, stored));
        if (!pan.vals32) return MLB_ENOMEM;
        to_f32_kernel<<<1216, 256, 0, st>>>(pan.vals, std::max<int64_t>(1, stored), pan.vals32);
        MLB_CHECK_LAUNCH(ctx, "to_f32_kernel");
        MLB_CUDA(ctx, cudaStreamSynchronize(st));
        dfree(ctx, A, pan.vals);
        pan.vals = nullptr;
    }
    return MLB_OK;
}

}  // namespace mlb
