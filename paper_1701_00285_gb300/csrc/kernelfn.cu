// Covariance function of an assembly: the kind and scale the kernels
// evaluate, the table of Chebyshev pieces for Matern smoothness without a
// closed form, and the coordinates of the anisotropic distance.
//
// Table (kind 3).  phi(s) = s^nu K_nu(s) / (Gamma(nu) 2^(nu-1)) and
// -s phi'(s) = s^(nu+1) K_{nu-1}(s) / (Gamma(nu) 2^(nu-1)) (from
// d/ds [s^nu K_nu(s)] = -s^nu K_{nu-1}(s), A&S 9.6.28) are sampled at the
// Chebyshev points of every piece (see matern.cuh for the pieces) and turned
// into 16 Chebyshev coefficients each.  The samples come from the integral
// representation K_nu(s) = int_0^inf exp(-s cosh t) cosh(nu t) dt (A&S 9.6.24)
// by the trapezoidal rule with step 1/16: the integrand is analytic and
// decaying in the strip |Im t| < pi/2, so the rule converges geometrically
// (error about exp(-2 pi (pi/4) / h) 2^(nu/2), far below 1e-16; Trefethen and
// Weideman, "The exponentially convergent trapezoidal rule", SIAM Review
// 2014).  Every term is formed in logarithms, so s^nu K_nu(s) stays in range
// for small s and large nu.  On each piece the functions are analytic with
// their only singularity at s = 0, at least as far from the piece as its own
// width; 16 coefficients then carry them to about 1e-16.  The graded pieces
// reach down to where |phi - 1| < 1e-17 (s^(2 min(nu, 1)) < 1e-17), the
// uniform ones up to where phi and -s phi' fall below 1e-18.
//
// Anisotropy (Sec. 3): r(theta)^2 = (x - y)^T diag(theta) (x - y) is the
// Euclidean distance of the coordinates scaled by sqrt(theta_k), so the
// kernels read scaled coordinates: precomputed copies of the FP32 offsets,
// and scale factors applied where FP64 coordinates are loaded.  The tree,
// the basis and the distance criterion keep the caller's coordinates.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "matern.cuh"

namespace mlb {

namespace {

constexpr double kStep = 0.0625;

// log(s^a K_nu(s) / (Gamma(nu) 2^(nu-1))) for s > 0, by the trapezoidal rule.
// The integrand's logarithm a ln s + ln cosh(mu t) - s cosh t (mu = |nu|) is
// formed as (a - mu) ln s + mu ln(s e^t) + ln((1 + e^(-2 mu t)) / 2) - s cosh t:
// near the peak s e^t is of order mu, so the large terms mu ln s and mu t of
// small s never meet as two rounded numbers (their difference would carry an
// error of mu |ln s| ulps into phi = 1 - O(s^2)).
double log_scaled_knu(double s, double nu, double a, double lognorm) {
    const double mu = std::fabs(nu);
    const double tstar = mu > 0.0 ? std::asinh(mu / s) : 0.0;   // the integrand's peak
    const double base = (a - mu) * std::log(s) - std::log(2.0) - lognorm;
    std::vector<double> ex;
    double emax = -INFINITY;
    for (int j = 0;; ++j) {
        const double t = j * kStep;
        const double e = base + mu * std::log(s * std::exp(t)) + std::log1p(std::exp(-2.0 * mu * t)) -
                         s * std::cosh(t) + (j == 0 ? std::log(0.5) : 0.0);
        ex.push_back(e);
        emax = std::max(emax, e);
        if (e < emax - 60.0 && t > tstar) break;
        if (j > 200000) break;
    }
    double acc = 0.0;
    for (double e : ex) acc += std::exp(e - emax);
    return emax + std::log(kStep * acc);
}

double phi_general(double s, double nu, double lognorm) {
    return std::exp(log_scaled_knu(s, nu, nu, lognorm));
}

double dphi_general(double s, double nu, double lognorm) {
    return std::exp(log_scaled_knu(s, nu - 1.0, nu + 1.0, lognorm));
}

// Chebyshev coefficients (c_0 halved) of f on [a, a + w] from kTabCoef samples
template <typename F>
void cheb_fit(F f, double a, double w, double* c) {
    const int n = kTabCoef;
    double fv[kTabCoef];
    for (int j = 0; j < n; ++j) {
        const double z = std::cos(M_PI * (j + 0.5) / n);
        fv[j] = f(a + 0.5 * w * (z + 1.0));
    }
    for (int k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += fv[j] * std::cos(M_PI * k * (j + 0.5) / n);
        c[k] = (2.0 / n) * acc;
    }
    c[0] *= 0.5;
}

struct Table {
    std::vector<double> c;
    int noct = 0, nhi = 0;
};

Table build_table(double nu) {
    Table T;
    const double lognorm = std::lgamma(nu) + (nu - 1.0) * std::log(2.0);
    const double lead = 2.0 * std::min(nu, 1.0);
    T.noct = (int)std::ceil(17.0 * std::log2(10.0) / lead) + 2;
    double smax = 1.0;
    while (smax < 2000.0 && (phi_general(smax, nu, lognorm) > 1e-18 || dphi_general(smax, nu, lognorm) > 1e-18))
        smax += 1.0;
    T.nhi = (int)std::ceil((smax - 1.0) / kTabWidth);
    const int npieces = 2 * T.noct + T.nhi;
    T.c.assign((size_t)npieces * 2 * kTabCoef, 0.0);
    auto fit = [&](int piece, double a, double w) {
        cheb_fit([&](double s) { return phi_general(s, nu, lognorm); }, a, w, &T.c[(size_t)(2 * piece) * kTabCoef]);
        cheb_fit([&](double s) { return dphi_general(s, nu, lognorm); }, a, w,
                 &T.c[(size_t)(2 * piece + 1) * kTabCoef]);
    };
    for (int k = 0; k < T.noct; ++k) {
        const double lo = std::ldexp(0.5, -k);   // the octave [2^-k-1, 2^-k)
        fit(2 * k, lo, 0.5 * lo);
        fit(2 * k + 1, 1.5 * lo, 0.5 * lo);
    }
    for (int j = 0; j < T.nhi; ++j) fit(2 * T.noct + j, 1.0 + j * kTabWidth, kTabWidth);
    return T;
}

std::mutex g_table_mutex;
std::map<double, Table> g_tables;   // per smoothness, for the rest of the process

// scaled FP32 coordinates of the mixed path: offsets from the data box centre
// and from the point's leaf centre, each as FP32 high and low parts
__global__ void scale_coords_kernel(int64_t N, int d, const double* __restrict__ xs, const int* __restrict__ leafOf,
                                    const double* __restrict__ leafctr, KGeo g, float* x32, float* x32lo,
                                    float* xl32, float* xl32lo, double* ctrA, int ncell) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = tid; k < N * d; k += stride) {
        const int64_t i = k / d;
        const int c = (int)(k - i * d);
        const double v = xs[k];
        const double og = (v - g.c[c]) * g.sc[c];
        const double ol = (v - leafctr[(int64_t)leafOf[i] * d + c]) * g.sc[c];
        const float oh = (float)og, lh = (float)ol;
        x32[k] = oh;
        x32lo[k] = (float)(og - (double)oh);
        xl32[k] = lh;
        xl32lo[k] = (float)(ol - (double)lh);
    }
    for (int64_t k = tid; k < (int64_t)ncell * d; k += stride) ctrA[k] = leafctr[k] * g.sc[k % d];
}

}  // namespace

mlb_status setup_kernel_fn(mlb_ctx* ctx) {
    const mlb_theta& th = ctx->theta;
    KernelFn K{};
    if (th.family == MLB_GAUSSIAN) {
        K.kind = KIND_GAUSS;
        K.scale = 1.0 / th.rho;
    } else {
        const int hk = nu_kind(th.nu);
        K.kind = hk >= 0 ? hk : KIND_TABLE;
        K.scale = std::sqrt(2.0 * th.nu) / th.rho;
    }
    K.scale32 = (float)K.scale;
    Arena& A = ctx->arena_asm;
    if (K.kind == KIND_TABLE) {
        const Table* T = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_table_mutex);
            auto it = g_tables.find(th.nu);
            if (it == g_tables.end()) it = g_tables.emplace(th.nu, build_table(th.nu)).first;
            T = &it->second;
        }
        std::vector<float> c32(T->c.begin(), T->c.end());
        double* tab = (double*)dalloc(ctx, A, sizeof(double) * T->c.size());
        float* tab32 = (float*)dalloc(ctx, A, sizeof(float) * c32.size());
        if (!tab || !tab32) return fail(ctx, MLB_ENOMEM, "covariance table");
        // on the context's stream: a plain cudaMemcpy from pageable memory may
        // return before its DMA lands, and the legacy stream it runs on is not
        // ordered with the context's non-blocking stream
        MLB_CUDA(ctx, cudaMemcpyAsync(tab, T->c.data(), sizeof(double) * T->c.size(), cudaMemcpyHostToDevice,
                                      ctx->stream));
        MLB_CUDA(ctx, cudaMemcpyAsync(tab32, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice,
                                      ctx->stream));
        MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        K.tab = tab;
        K.tab32 = tab32;
        K.noct = T->noct;
        K.nhi = T->nhi;
    }
    ctx->kfn = K;
    // the anisotropic distance: scale factors and scaled coordinates
    for (int c = 0; c < kMaxDim; ++c) {
        ctx->kgeo.c[c] = c < ctx->d ? 0.5 * (ctx->box_lo[c] + ctx->box_hi[c]) : 0.0;
        ctx->kgeo.sc[c] = (th.naxis > 0 && c < ctx->d) ? std::sqrt(th.axis[c]) : 1.0;
    }
    ctx->kxs32 = ctx->xs32;
    ctx->kxs32lo = ctx->xs32lo;
    ctx->kxl32 = ctx->xl32;
    ctx->kxl32lo = ctx->xl32lo;
    ctx->kctr = ctx->leafctr;
    if (th.naxis > 0) {
        const int64_t N = ctx->N;
        const int d = ctx->d;
        std::vector<int> leafOf(N);
        for (int k = 0; k < (1 << ctx->t); ++k) {
            const HostCell& c = ctx->hcells[(1 << ctx->t) - 1 + k];
            for (int i = c.beg; i < c.end; ++i) leafOf[i] = (1 << ctx->t) - 1 + k;
        }
        int* dleaf = (int*)dalloc(ctx, A, sizeof(int) * N);
        float* b[4];
        for (auto& q : b) q = (float*)dalloc(ctx, A, sizeof(float) * N * d);
        double* ctrA = (double*)dalloc(ctx, A, sizeof(double) * ctx->ncell * d);
        if (!dleaf || !b[0] || !b[1] || !b[2] || !b[3] || !ctrA) return fail(ctx, MLB_ENOMEM, "scaled coordinates");
        MLB_CUDA(ctx, cudaMemcpyAsync(dleaf, leafOf.data(), sizeof(int) * N, cudaMemcpyHostToDevice, ctx->stream));
        scale_coords_kernel<<<(unsigned)std::min<int64_t>((N * d + 255) / 256, 4096), 256, 0, ctx->stream>>>(
            N, d, ctx->xs, dleaf, ctx->leafctr, ctx->kgeo, b[0], b[1], b[2], b[3], ctrA, ctx->ncell);
        MLB_CHECK_LAUNCH(ctx, "scale_coords_kernel");
        MLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // leafOf goes out of scope
        ctx->kxs32 = b[0];
        ctx->kxs32lo = b[1];
        ctx->kxl32 = b[2];
        ctx->kxl32lo = b[3];
        ctx->kctr = ctrA;
    }
    return MLB_OK;
}

}  // namespace mlb

using namespace mlb;

extern "C" mlb_status mlb_covariance(const mlb_theta* th, const double* r, int64_t n, int deriv, double* out) {
    if (!th || (n > 0 && (!r || !out)) || n < 0) return MLB_EINVAL;
    if (th->family != MLB_MATERN && th->family != MLB_GAUSSIAN) return MLB_EINVAL;
    if (th->family == MLB_MATERN && !(th->nu >= 0.2 && th->nu <= 30.0)) return MLB_EINVAL;
    if (!(th->rho > 0) || !std::isfinite(th->rho)) return MLB_EINVAL;
    const bool dv = deriv != 0;
    if (th->family == MLB_GAUSSIAN) {
        for (int64_t i = 0; i < n; ++i) {
            const double s = r[i] / th->rho, g = std::exp(-0.5 * s * s);
            out[i] = dv ? s * s * g : g;
        }
        return MLB_OK;
    }
    const double scale = std::sqrt(2.0 * th->nu) / th->rho;
    const int hk = nu_kind(th->nu);
    if (hk >= 0) {
        for (int64_t i = 0; i < n; ++i) {
            const double s = scale * r[i], e = std::exp(-s);
            const double poly = hk == 0 ? 1.0 : (hk == 1 ? 1.0 + s : 1.0 + s + s * s / 3.0);
            const double dpoly = hk == 0 ? s : (hk == 1 ? s * s : s * s / 3.0 * (1.0 + s));
            out[i] = (dv ? dpoly : poly) * e;
        }
        return MLB_OK;
    }
    const Table* T = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_table_mutex);
        auto it = g_tables.find(th->nu);
        if (it == g_tables.end()) it = g_tables.emplace(th->nu, build_table(th->nu)).first;
        T = &it->second;
    }
    for (int64_t i = 0; i < n; ++i) out[i] = table_f64(T->c.data(), T->noct, T->nhi, scale * r[i], dv ? 1 : 0);
    return MLB_OK;
}
