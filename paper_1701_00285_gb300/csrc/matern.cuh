// Matern covariance for half-integer smoothness (Def. "Matern covariance
// function", Sec. 3.1), written from the definition with the textbook
// half-integer Bessel functions: with s = sqrt(2 nu) r / rho,
//   nu = 1/2: e^-s,  nu = 3/2: (1 + s) e^-s,  nu = 5/2: (1 + s + s^2/3) e^-s.
// kind = 0, 1, 2 selects nu = 1/2, 3/2, 5/2; scale = sqrt(2 nu) / rho.
#pragma once

#include <cuda_runtime.h>

namespace mlb {

__device__ __forceinline__ double matern_f64(double r, int kind, double scale) {
    const double s = scale * r;
    const double e = exp(-s);
    if (kind == 0) return e;
    if (kind == 1) return (1.0 + s) * e;
    return (1.0 + s + s * s * (1.0 / 3.0)) * e;
}

// d phi / d log(rho) = -s phi'(s): s e^-s, s^2 e^-s, (s^2/3)(1 + s) e^-s.
__device__ __forceinline__ double dmatern_dlogrho_f64(double r, int kind, double scale) {
    const double s = scale * r;
    const double e = exp(-s);
    if (kind == 0) return s * e;
    if (kind == 1) return s * s * e;
    return (s * s * (1.0 / 3.0)) * (1.0 + s) * e;
}

__device__ __forceinline__ float matern_f32(float r, int kind, float scale) {
    const float s = scale * r;
    const float e = expf(-s);
    if (kind == 0) return e;
    if (kind == 1) return (1.0f + s) * e;
    return (1.0f + s + s * s * (1.0f / 3.0f)) * e;
}

__device__ __forceinline__ float dmatern_dlogrho_f32(float r, int kind, float scale) {
    const float s = scale * r;
    const float e = expf(-s);
    if (kind == 0) return s * e;
    if (kind == 1) return s * s * e;
    return (s * s * (1.0f / 3.0f)) * (1.0f + s) * e;
}

// Cascaded FP32 accumulation (Sum2 of Ogita, Rump and Oishi, "Accurate sum and
// dot product", 2005): every addition is an error-free TwoSum and the rounding
// errors are summed separately, so s + e carries the sum to about twice FP32
// precision even when the terms cancel (plain Kahan compensation does not).
// The _rn intrinsics keep the compiler from fusing a product into the sums.
__device__ __forceinline__ void sum2_add(float& s, float& e, float v) {
    const float t = __fadd_rn(s, v);
    const float bb = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(v, bb)));
    s = t;
}

inline int nu_kind(double nu) {
    if (nu == 0.5) return 0;
    if (nu == 1.5) return 1;
    if (nu == 2.5) return 2;
    return -1;
}

}  // namespace mlb
