// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32
// numbers (about 48 significant bits).  Built from the error-free
// transformations of Knuth (TwoSum) and Dekker (TwoProduct, here with a fused
// multiply-add), "A floating-point technique for extending the available
// precision" (Dekker 1971).  On GB300 the FP32 pipes run about 64 times
// faster than FP64, so kernel values needed to better than FP32 accuracy are
// evaluated this way instead of in FP64.
//
// ff_exp follows Tang's table-driven method ("Table-driven implementation of
// the exponential function in IEEE floating-point arithmetic", ACM TOMS 15,
// 1989): x = k ln2/64 + r with a
// Cody-Waite three-part ln2/64 (the high part has 11 significant bits, so k
// times it is exact for |k| < 2^13), e^x = 2^(k div 64) * 2^((k mod 64)/64) * e^r,
// the 64 table values 2^(j/64) as double-float (each CTA fills its shared
// table from FP64 exp2 once), and e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24 + r^3/120)
// for |r| <= ln2/128 (truncation below 1e-16 relative).  Relative error about
// 1e-13 for -87 < x <= 0.
#pragma once

#include <cuda_runtime.h>

#include "matern.cuh"

namespace mlb {

struct ff {
    float h, l;
};

// Every operation below is written with the _rn intrinsics: the compiler must
// not fuse a product into a following addition here, or the error terms would
// describe a rounding that never happened.
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_quick(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = ff_two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return ff_quick(s.h, s.l);
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, {-y.h, -y.l}); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = ff_two_prod(x.h, y.h);
    p.l = fmaf(x.h, y.l, fmaf(x.l, y.h, p.l));
    return ff_quick(p.h, p.l);
}

__device__ __forceinline__ ff ff_mul_f(ff x, float b) {
    ff p = ff_two_prod(x.h, b);
    p.l = fmaf(x.l, b, p.l);
    return ff_quick(p.h, p.l);
}

// sqrt with one Newton correction: r = sqrt(x_h), t = (x - r^2) / (2 r)
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.h > 0.0f)) return {0.0f, 0.0f};
    const float r = sqrtf(x.h);
    const ff rr = ff_two_prod(r, r);
    const float t = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.h, rr.h), rr.l), x.l), __fmul_rn(2.0f, r));
    return ff_quick(r, t);
}

// Fills a shared table of 2^(j/64), j = 0..63, as double-float (call with all
// threads of the block, then __syncthreads()).
__device__ __forceinline__ void ff_fill_exp2_table(float2* tab) {
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        const double v = exp2((double)j / 64.0);
        const float h = (float)v;
        tab[j] = make_float2(h, (float)(v - (double)h));
    }
}

// e^x for x <= 0 (x = x_h + x_l); returns 0 below -87
__device__ __forceinline__ ff ff_exp(ff x, const float2* tab) {
    if (x.h < -87.0f) return {0.0f, 0.0f};
    constexpr float kInvL = 92.33248138427734f;          // 64 / ln 2 (only selects k)
    constexpr float kL1 = 0.010833740234375f;             // ln2/64, 11 significant bits
    constexpr float kL2 = -3.3155381515825866e-06f;       // next FP32 part of ln2/64
    constexpr float kL3 = 2.572804640231345e-14f;         // remainder
    const float kf = rintf(x.h * kInvL);
    const int k = (int)kf;
    ff r = ff_two_sum(fmaf(-kf, kL1, x.h), x.l);         // x_h - k kL1 is exact
    r = ff_add(r, ff_two_prod(-kf, kL2));
    r.l = fmaf(-kf, kL3, r.l);
    r = ff_quick(r.h, r.l);
    const float q = 0.5f + r.h * (1.0f / 6.0f + r.h * (1.0f / 24.0f + r.h * (1.0f / 120.0f)));
    const ff r2 = ff_mul(r, r);
    const ff em1 = ff_add(r, ff_mul_f(r2, q));           // e^r - 1
    const ff er = ff_add({1.0f, 0.0f}, em1);             // e^r
    const int j = k & 63;
    const int m = (k - j) / 64;
    const float2 t = tab[j];
    const ff v = ff_mul(er, {t.x, t.y});
    const float sc = __int_as_float((m + 127) << 23);    // 2^m, m >= -126 here
    return {__fmul_rn(v.h, sc), __fmul_rn(v.l, sc)};
}

// Matern kernel value in double-float: s = scale * r, kind 0/1/2 = nu 1/2, 3/2, 5/2
__device__ __forceinline__ ff ff_matern(ff r, int kind, ff scale, const float2* tab) {
    const ff s = ff_mul(scale, r);
    const ff e = ff_exp({-s.h, -s.l}, tab);
    if (kind == 0) return e;
    ff poly = ff_add({1.0f, 0.0f}, s);
    if (kind == 2) {
        constexpr float kThirdH = 0.3333333432674408f;
        constexpr float kThirdL = -9.934107758624577e-09f;
        poly = ff_add(poly, ff_mul(ff_mul(s, s), {kThirdH, kThirdL}));
    }
    return ff_mul(poly, e);
}

// d phi / d log(rho) = -s phi'(s) in double-float: s e^-s, s^2 e^-s, (s^2/3)(1 + s) e^-s
__device__ __forceinline__ ff ff_dmatern(ff r, int kind, ff scale, const float2* tab) {
    const ff s = ff_mul(scale, r);
    const ff e = ff_exp({-s.h, -s.l}, tab);
    if (kind == 0) return ff_mul(s, e);
    const ff s2 = ff_mul(s, s);
    if (kind == 1) return ff_mul(s2, e);
    constexpr float kThirdH = 0.3333333432674408f;
    constexpr float kThirdL = -9.934107758624577e-09f;
    return ff_mul(ff_mul(ff_mul(s2, {kThirdH, kThirdL}), ff_add({1.0f, 0.0f}, s)), e);
}

// split a double into double-float
__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(__dsub_rn(v, (double)h))};
}

// Any covariance function in double-float (DERIV: d phi / d log(rho)):
// closed-form Matern kinds and the Gaussian on the FP32 pipes; tabulated
// smoothness through the FP64 table (matern.cuh), split into double-float.
template <bool DERIV>
__device__ __forceinline__ ff ff_kern(ff r, const KernelFn& K, ff scale, const float2* tab) {
    if (K.kind <= KIND_NU_5HALF) return DERIV ? ff_dmatern(r, K.kind, scale, tab) : ff_matern(r, K.kind, scale, tab);
    if (K.kind == KIND_GAUSS) {
        const ff s = ff_mul(scale, r);
        const ff h2 = ff_mul_f(ff_mul(s, s), 0.5f);
        const ff g = ff_exp({-h2.h, -h2.l}, tab);
        return DERIV ? ff_mul(ff_mul(s, s), g) : g;
    }
    const double s = ((double)r.h + (double)r.l) * K.scale;
    return ff_from_double(table_f64(K.tab, K.noct, K.nhi, s, DERIV ? 1 : 0));
}

}  // namespace mlb
