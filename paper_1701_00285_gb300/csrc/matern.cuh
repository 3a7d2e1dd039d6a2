// Covariance functions on the device.
//
// Matern (Def. "Matern covariance function", Sec. 3.1), unit variance, with
// s = sqrt(2 nu) r / rho:
//   phi(s) = s^nu K_nu(s) / (Gamma(nu) 2^(nu-1)),  phi(0) = 1.
// For half-integer smoothness the textbook half-integer Bessel functions give
// closed forms (kind 0, 1, 2):
//   nu = 1/2: e^-s,  nu = 3/2: (1 + s) e^-s,  nu = 5/2: (1 + s + s^2/3) e^-s.
// Any other nu (kind 3) is evaluated from a table of Chebyshev pieces of phi
// and of -s phi'(s) that the host builds for the assembly's nu (kernelfn.cu):
// pieces on [2^-k-1, 1.5 2^-k-1) and [1.5 2^-k-1, 2^-k) for k = 0 .. noct-1
// (graded towards s = 0, where phi carries the non-smooth term s^(2 nu)) and
// pieces of width kTabWidth from s = 1 on; below the finest octave phi = 1
// and past the last piece phi = 0 to working accuracy.
// Gaussian (kind 4, the kernel of the accuracy study of Sec. 8.2):
//   phi(r) = exp(-r^2 / (2 theta^2)), s = r / theta, phi = exp(-s^2 / 2).
// Derivatives are taken in log(rho) (log(theta)): since s is proportional to
// 1 / rho, d phi / d log(rho) = -s phi'(s).
#pragma once

#include <cuda_runtime.h>

namespace mlb {

constexpr int kTabCoef = 16;         // Chebyshev coefficients per piece and function
constexpr double kTabWidth = 0.25;   // width of the pieces from s = 1 on

enum { KIND_NU_HALF = 0, KIND_NU_3HALF = 1, KIND_NU_5HALF = 2, KIND_TABLE = 3, KIND_GAUSS = 4 };

// The covariance function of one assembly, passed by value to the kernels.
struct KernelFn {
    int kind;              // see above
    double scale;          // s = scale r: sqrt(2 nu) / rho (Matern), 1 / theta (Gaussian)
    float scale32;
    const double* tab;     // kind 3: per piece, kTabCoef coefficients of phi then of -s phi'
    const float* tab32;    // the same in FP32
    int noct;              // kind 3: octaves of graded pieces below s = 1
    int nhi;               // kind 3: pieces of width kTabWidth from s = 1
};

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

// Table evaluation (kind 3): the piece holding s, then Clenshaw's recurrence
// for sum_k c_k T_k(z) on the piece mapped to [-1, 1] (c_0 stored halved).
// The FP64 form also runs on the host (mlb_covariance).
static __host__ __device__ __noinline__ double table_f64(const double* __restrict__ tab, int noct, int nhi, double s, int deriv) {
    double a, w;
    int piece;
    if (s >= 1.0) {
        const double t = (s - 1.0) * (1.0 / kTabWidth);
        if (t >= (double)nhi) return 0.0;
        const int j = (int)t;
        piece = 2 * noct + j;
        a = 1.0 + j * kTabWidth;
        w = kTabWidth;
    } else {
        if (!(s > 0.0)) return deriv ? 0.0 : 1.0;
        int e;
        const double m = frexp(s, &e);            // s = m 2^e, m in [0.5, 1), e <= 0
        if (-e >= noct) return deriv ? 0.0 : 1.0;
        const double lo = ldexp(0.5, e);          // 2^(e-1): the octave [lo, 2 lo)
        const int hiHalf = m >= 0.75;
        piece = 2 * (-e) + hiHalf;
        a = hiHalf ? 1.5 * lo : lo;
        w = 0.5 * lo;
    }
    const double* c = tab + (size_t)(2 * piece + deriv) * kTabCoef;
    const double z = (2.0 * (s - a) - w) / w;
    double b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int i = kTabCoef - 1; i >= 1; --i) {
        const double t = fma(2.0 * z, b1, c[i] - b2);
        b2 = b1;
        b1 = t;
    }
    return fma(z, b1, c[0] - b2);
}

static __device__ __noinline__ float table_f32(const float* __restrict__ tab, int noct, int nhi, float s, int deriv) {
    float a, w;
    int piece;
    if (s >= 1.0f) {
        const float t = (s - 1.0f) * (float)(1.0 / kTabWidth);
        if (t >= (float)nhi) return 0.0f;
        const int j = (int)t;
        piece = 2 * noct + j;
        a = 1.0f + j * (float)kTabWidth;
        w = (float)kTabWidth;
    } else {
        if (!(s > 0.0f)) return deriv ? 0.0f : 1.0f;
        int e;
        const float m = frexpf(s, &e);
        if (-e >= noct) return deriv ? 0.0f : 1.0f;
        const float lo = ldexpf(0.5f, e);
        const int hiHalf = m >= 0.75f;
        piece = 2 * (-e) + hiHalf;
        a = hiHalf ? 1.5f * lo : lo;
        w = 0.5f * lo;
    }
    const float* c = tab + (size_t)(2 * piece + deriv) * kTabCoef;
    const float z = (2.0f * (s - a) - w) / w;
    float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int i = kTabCoef - 1; i >= 1; --i) {
        const float t = fmaf(2.0f * z, b1, c[i] - b2);
        b2 = b1;
        b1 = t;
    }
    return fmaf(z, b1, c[0] - b2);
}

// phi(r) (DERIV: d phi / d log(rho)) for any kind
template <bool DERIV>
__device__ __forceinline__ double kern_f64(double r, const KernelFn& K) {
    if (K.kind <= KIND_NU_5HALF)
        return DERIV ? dmatern_dlogrho_f64(r, K.kind, K.scale) : matern_f64(r, K.kind, K.scale);
    const double s = K.scale * r;
    if (K.kind == KIND_GAUSS) {
        const double g = exp(-0.5 * s * s);
        return DERIV ? s * s * g : g;
    }
    return table_f64(K.tab, K.noct, K.nhi, s, DERIV ? 1 : 0);
}

template <bool DERIV>
__device__ __forceinline__ float kern_f32(float r, const KernelFn& K) {
    if (K.kind <= KIND_NU_5HALF)
        return DERIV ? dmatern_dlogrho_f32(r, K.kind, K.scale32) : matern_f32(r, K.kind, K.scale32);
    const float s = K.scale32 * r;
    if (K.kind == KIND_GAUSS) {
        const float g = expf(-0.5f * s * s);
        return DERIV ? s * s * g : g;
    }
    return table_f32(K.tab32, K.noct, K.nhi, s, DERIV ? 1 : 0);
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
