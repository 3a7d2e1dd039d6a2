// Kernel sum of the matrix-free product on the tensor cores (Sec. 6.2: the
// middle step C (W^T g) of the three-step product; targets and sources are
// both the data points), for the closed-form Matern kinds.
//
// For a block of 128 targets x and a tile of 256 sources y the squared
// distances form one dense contraction:
//
//   r^2 = |x' - y'' + D|^2 = |x'|^2 + |y''|^2 + (2 x'.D + |D|^2) - 2 y''.D - 2 x'.y''
//
// with x' = x - c_T and y'' = y - c_S offsets from a point of the target
// block and of the source tile, and D = c_T - c_S.  Every coordinate is split
// into three BF16 numbers (h + m + l = the FP32 value; the split is exact),
// and the products h.h + h.m + m.h + h.l + l.h + m.m (the terms above 2^-24
// relative) are six BF16 dot products of length d.  Those, the norms and the
// two correction terms (each again split in three) are laid out along K, so
// one 128 x 256 x K tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation
// in tensor memory; K = 6d + 12 padded to a multiple of 16) leaves r^2 of all
// 32,768 pairs in TMEM.  Offsets from nearby points keep the terms that must
// cancel for near pairs small, so r^2 of near pairs keeps about FP32
// accuracy; the pair of a point with itself is set to r^2 = 0 exactly.
//
// Per tile: all threads write the source operand (and the correction terms of
// the target operand) to shared memory, one thread issues the MMAs and
// commits them to an mbarrier, and eight warps read r^2 back with tcgen05.ld
// (warp w: TMEM lanes 32 (w mod 4) .. +31, columns 128 (w div 4) .. +127),
// evaluate phi and accumulate phi(r) a_j (FP32 sums per 32 columns, cascaded
// with Sum2, FP64 across tiles).  phi is evaluated in t = s log2(e): one
// approximate square root of sc^2 r^2 and one 2^-t, both on the MUFU, and
// the Matern polynomial in t on the FMA pipe.  Two CTAs per SM, each holding 256 TMEM
// columns (the 512 of an SM); the dynamic shared memory requested keeps a
// third CTA off the SM, so the allocation never waits.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>

#include "bulk.cuh"
#include "internal.h"

namespace mlb {

namespace {

constexpr int kTcM = 128;        // targets per CTA: TMEM lanes of the accumulator
constexpr int kTcN = 256;        // sources per tile: TMEM columns
constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 256;
constexpr int kTcSmem = 96 * 1024;   // dynamic shared memory: at most two CTAs per SM

template <int D>
struct TcShape {
    static constexpr int KP = ((6 * D + 12) + 15) / 16 * 16;   // K padded to the MMA's 16
    static constexpr int KG = KP / 8;                          // 16-byte core-matrix columns along K
    static constexpr int ABytes = kTcM * KP * 2;
    static constexpr int BBytes = kTcN * KP * 2;
};

// Byte offset of element (row, k) of a K-major operand without swizzling:
// core matrices of 8 rows x 16 bytes, K-adjacent core matrices 128 bytes
// apart (the descriptor's leading-dimension offset), 8-row groups KG * 128
// bytes apart (its stride-dimension offset).
template <int KG>
__device__ __forceinline__ int op_off(int row, int k) {
    return (row >> 3) * (KG * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride dimension byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 D, both operands
// K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4)                 // D format F32
                            | (1u << 7)               // A format BF16
                            | (1u << 10)              // B format BF16
                            | ((uint32_t)(kTcN >> 3) << 17)
                            | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane, waited for
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// v = h + m + l exactly, each part BF16 (the remainders are exact in FP32)
__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(v);
    const float r1 = __fsub_rn(v, __bfloat162float(h));
    m = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(m));
    l = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// One operand row: the six split coordinate vectors, then four groups of
// three (target: |x'|^2, ones, R, ones; source: ones, |y''|^2, ones, Q).
template <int D>
__device__ void write_row(unsigned char* base, int row, const float* c, bool target, float norm, float corr) {
    constexpr int KP = TcShape<D>::KP, KG = TcShape<D>::KG;
    __nv_bfloat16 v[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) v[k] = bf(0.0f);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        __nv_bfloat16 h, m, l;
        split3(c[k], h, m, l);
        if (target) {   // -2 (h | h | m | h | l | m)
            const __nv_bfloat16 h2 = bf(-2.0f * __bfloat162float(h)), m2 = bf(-2.0f * __bfloat162float(m)),
                                l2 = bf(-2.0f * __bfloat162float(l));
            v[k] = h2;
            v[D + k] = h2;
            v[2 * D + k] = m2;
            v[3 * D + k] = h2;
            v[4 * D + k] = l2;
            v[5 * D + k] = m2;
        } else {        // h | m | h | l | h | m
            v[k] = h;
            v[D + k] = m;
            v[2 * D + k] = h;
            v[3 * D + k] = l;
            v[4 * D + k] = h;
            v[5 * D + k] = m;
        }
    }
    __nv_bfloat16 nh, nm, nl, ch, cm, cl;
    split3(norm, nh, nm, nl);
    split3(corr, ch, cm, cl);
    const __nv_bfloat16 one = bf(1.0f);
    const int e = 6 * D;
    if (target) {
        v[e + 0] = nh; v[e + 1] = nm; v[e + 2] = nl;
        v[e + 3] = one; v[e + 4] = one; v[e + 5] = one;
        v[e + 6] = ch; v[e + 7] = cm; v[e + 8] = cl;
        v[e + 9] = one; v[e + 10] = one; v[e + 11] = one;
    } else {
        v[e + 0] = one; v[e + 1] = one; v[e + 2] = one;
        v[e + 3] = nh; v[e + 4] = nm; v[e + 5] = nl;
        v[e + 6] = one; v[e + 7] = one; v[e + 8] = one;
        v[e + 9] = ch; v[e + 10] = cm; v[e + 11] = cl;
    }
#pragma unroll
    for (int g = 0; g < KG; ++g) {
        uint4 q;
        q.x = (uint32_t)__bfloat16_as_ushort(v[8 * g + 0]) | ((uint32_t)__bfloat16_as_ushort(v[8 * g + 1]) << 16);
        q.y = (uint32_t)__bfloat16_as_ushort(v[8 * g + 2]) | ((uint32_t)__bfloat16_as_ushort(v[8 * g + 3]) << 16);
        q.z = (uint32_t)__bfloat16_as_ushort(v[8 * g + 4]) | ((uint32_t)__bfloat16_as_ushort(v[8 * g + 5]) << 16);
        q.w = (uint32_t)__bfloat16_as_ushort(v[8 * g + 6]) | ((uint32_t)__bfloat16_as_ushort(v[8 * g + 7]) << 16);
        *reinterpret_cast<uint4*>(base + op_off<KG>(row, 8 * g)) = q;
    }
}

// the target operand's correction R = 2 x'.D + |D|^2 (three BF16 slots)
template <int D>
__device__ void write_corr(unsigned char* base, int row, float corr) {
    constexpr int KG = TcShape<D>::KG;
    __nv_bfloat16 h, m, l;
    split3(corr, h, m, l);
    const int e = 6 * D + 6;
    *reinterpret_cast<__nv_bfloat16*>(base + op_off<KG>(row, e)) = h;
    *reinterpret_cast<__nv_bfloat16*>(base + op_off<KG>(row, e + 1)) = m;
    *reinterpret_cast<__nv_bfloat16*>(base + op_off<KG>(row, e + 2)) = l;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// phi at s = t ln 2, given t = s log2(e): e^-s = 2^-t (one MUFU operation),
// the Matern polynomial rewritten in t
template <int KIND>
__device__ __forceinline__ float matern_t(float t) {
    constexpr float kLn2 = 0.693147180559945309f;
    const float e = ex2_approx(-t);
    if (KIND == 0) return e;
    if (KIND == 1) return fmaf(kLn2, t, 1.0f) * e;
    return fmaf(t, fmaf(t, kLn2 * kLn2 / 3.0f, kLn2), 1.0f) * e;
}

// 32 accumulator columns of one target row: t = sqrt(sc2 r^2), phi, and the
// weighted sums.  DIAG: the chunk may hold the row's own point (column
// selfc), whose distance is set to zero exactly.
template <int KIND, bool DIAG>
__device__ __forceinline__ void tc_row_chunk(const float (&r2)[32], const float* __restrict__ wh,
                                             const float* __restrict__ wl, float sc2, int selfc, float& ch,
                                             float& suml) {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        float q2 = fmaxf(r2[c], 0.0f) * sc2;
        if (DIAG && c == selfc) q2 = 0.0f;
        const float kv = matern_t<KIND>(sqrt_approx(q2));
        ch = fmaf(kv, wh[c], ch);
        suml = fmaf(kv, wl[c], suml);
    }
}

template <int D, int KIND>
__global__ void __launch_bounds__(kTcThreads, 2)
    ksum_tc_kernel(const float* __restrict__ x32, const double* __restrict__ a, int64_t N, float sc2,
                   int64_t jchunk, double* __restrict__ out, double* __restrict__ part, int* err) {
    using S = TcShape<D>;
    extern __shared__ __align__(1024) unsigned char sm_tc[];
    unsigned char* sa = sm_tc;                       // target operand (S::ABytes)
    unsigned char* sb = sm_tc + ((S::ABytes + 1023) / 1024) * 1024;   // source operand (S::BBytes)
    float* wh = reinterpret_cast<float*>(sb + ((S::BBytes + 1023) / 1024) * 1024);   // weights, high parts
    float* wl = wh + kTcN;                                                             // and low parts
    double* red = reinterpret_cast<double*>(wl + kTcN);                               // halves of the sums
    uint64_t* mbar = reinterpret_cast<uint64_t*>(red + kTcM);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kTcM;
    const int64_t jb = (int64_t)blockIdx.y * jchunk, je = min(N, jb + jchunk);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_fence_init();
        bad = 0;
    }
    // the target block's reference point (its middle point) and this thread's target
    float cT[D], xp[D];
    {
        const int64_t ic = min(i0 + kTcM / 2, N - 1);
#pragma unroll
        for (int k = 0; k < D; ++k) cT[k] = x32[ic * D + k];
    }
    if (tid < kTcM) {
        const int64_t i = i0 + tid;
        float n2 = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            xp[k] = i < N ? __fsub_rn(x32[i * D + k], cT[k]) : 0.0f;
            n2 = fmaf(xp[k], xp[k], n2);
        }
        write_row<D>(sa, tid, xp, true, n2, 0.0f);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t aaddr = smem_u32(sa), baddr = smem_u32(sb);

    const int quarter = warp & 3, half = warp >> 2;
    const int64_t my_i = i0 + quarter * 32 + lane;      // this thread's target (TMEM lane)
    float sumh = 0.0f, sume = 0.0f, suml = 0.0f;
    double acc = 0.0;
    int it = 0;
    for (int64_t jt = jb; jt < je; jt += kTcN, ++it) {
        // the tile's reference point, D = c_T - c_S, and the two operand rows
        float dl[D], d2 = 0.0f;
        {
            const int64_t jc = min(jt + kTcN / 2, N - 1);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                dl[k] = __fsub_rn(cT[k], x32[jc * D + k]);
                d2 = fmaf(dl[k], dl[k], d2);
            }
        }
        {
            const int64_t j = jt + tid;
            float yp[D], n2 = 0.0f, q = 0.0f;
            const bool live = j < je;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                yp[k] = live ? __fsub_rn(x32[j * D + k], x32[min(jt + kTcN / 2, N - 1) * D + k]) : 0.0f;
                n2 = fmaf(yp[k], yp[k], n2);
                q = fmaf(yp[k], dl[k], q);
            }
            write_row<D>(sb, tid, yp, false, n2, -2.0f * q);
            const double w = live ? a[j] : 0.0;
            const float h = (float)w;
            wh[tid] = h;
            wl[tid] = (float)(w - (double)h);
        }
        if (tid < kTcM) {
            float rc = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) rc = fmaf(xp[k], dl[k], rc);
            write_corr<D>(sa, tid, fmaf(2.0f, rc, d2));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < S::KP / 16; ++ks)
                umma(tmem, smem_desc(aaddr + ks * 256, 128, S::KG * 128), smem_desc(baddr + ks * 256, 128, S::KG * 128),
                     ks > 0 ? 1u : 0u);
            umma_commit(mbar);
        }
        if (!mbar_wait(mbar, (unsigned)(it & 1))) bad = 1;
        tc_fence_after();
        __syncthreads();
        if (bad) break;
        // the self pairs: target i against source i of this tile; a chunk of
        // 32 columns can hold them only where it meets the warp's 32 rows
        const int64_t rowBase = i0 + quarter * 32;
#pragma unroll 1
        for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
            float r2[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r2);
            float ch = 0.0f;
            const int64_t colBase = jt + c0;
            if (rowBase < colBase + 32 && colBase < rowBase + 32)
                tc_row_chunk<KIND, true>(r2, wh + c0, wl + c0, sc2, (int)(my_i - colBase), ch, suml);
            else
                tc_row_chunk<KIND, false>(r2, wh + c0, wl + c0, sc2, 0, ch, suml);
            sum2_add(sumh, sume, ch);
        }
        acc += (double)sumh + ((double)sume + (double)suml);
        sumh = sume = suml = 0.0f;
        tc_fence_before();
        __syncthreads();
    }
    // the two column halves of every target, then the output
    if (half == 1) red[quarter * 32 + lane] = acc;
    __syncthreads();
    if (half == 0 && my_i < N) {
        const double v = acc + red[quarter * 32 + lane];
        if (part) part[blockIdx.y * N + my_i] = v;
        else out[my_i] = v;
    }
    if (bad && tid == 0) {
        atomicOr(err, 1);
        // the MMAs in flight finish before the tensor memory is released
        mbar_wait(mbar, (unsigned)(it & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// out_k = sum over the source chunks of part[chunk][k], in chunk order
__global__ void tc_reduce_kernel(const double* __restrict__ part, int splits, int64_t N, double* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int c = 0; c < splits; ++c) v += part[c * N + k];
        out[k] = v;
    }
}

template <int D, int KIND>
bool launch_d(mlb_ctx* ctx, const double* a, double* out) {
    static_assert(TcShape<D>::ABytes + TcShape<D>::BBytes + 4096 + 1024 <= kTcSmem, "shared memory");
    const int64_t N = ctx->N;
    const int64_t ctasM = (N + kTcM - 1) / kTcM;
    // sources split so that about two waves of CTAs fill the GPU
    int64_t want = (2LL * 2 * std::max(ctx->nsm, 1) + ctasM - 1) / ctasM;
    want = std::min<int64_t>(want, std::max<int64_t>(1, N / (4LL * kTcN)));
    want = std::min<int64_t>(want, ctx->ksum_part_cap / std::max<int64_t>(N, 1));
    int64_t chunk = N, splits = 1;
    if (want > 1 && ctx->ksum_part) {
        chunk = (N + want - 1) / want;
        chunk = (chunk + kTcN - 1) / kTcN * kTcN;
        splits = (N + chunk - 1) / chunk;
    }
    // t = s log2(e) = sc r: the epilogue's exponential is then one 2^-t
    const double sc = ctx->kfn.scale * 1.4426950408889634;
    if (cudaFuncSetAttribute(ksum_tc_kernel<D, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ksum_tc_kernel<D, KIND><<<dim3((unsigned)ctasM, (unsigned)splits), kTcThreads, kTcSmem, ctx->stream>>>(
        ctx->kxs32, a, N, (float)(sc * sc), chunk, out, splits > 1 ? ctx->ksum_part : nullptr, ctx->flag + 3);
    ctx->launches += 1;
    if (splits > 1) {
        tc_reduce_kernel<<<(unsigned)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, ctx->stream>>>(
            ctx->ksum_part, (int)splits, N, out);
        ctx->launches += 1;
    }
    return true;
}

template <int D>
bool launch_kind(mlb_ctx* ctx, const double* a, double* out) {
    switch (ctx->kfn.kind) {
        case KIND_NU_HALF: return launch_d<D, 0>(ctx, a, out);
        case KIND_NU_3HALF: return launch_d<D, 1>(ctx, a, out);
        case KIND_NU_5HALF: return launch_d<D, 2>(ctx, a, out);
        default: return false;
    }
}

}  // namespace

bool ksum_tc_supported(const mlb_ctx* ctx) {
    return ctx->kfn.kind <= KIND_NU_5HALF && (ctx->d == 5 || ctx->d == 8 || ctx->d == 10);
}

bool ksum_tc_self(mlb_ctx* ctx, const double* a, double* out) {
    if (!ksum_tc_supported(ctx)) return false;
    switch (ctx->d) {
        case 5: return launch_kind<5>(ctx, a, out);
        case 8: return launch_kind<8>(ctx, a, out);
        case 10: return launch_kind<10>(ctx, a, out);
        default: return false;
    }
}

}  // namespace mlb
