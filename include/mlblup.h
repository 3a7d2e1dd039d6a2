/*
 * mlblup.h -- C ABI of the GB300 multilevel BLUP library (libmlblup.so).
 *
 * The library computes the multilevel best linear unbiased predictor of
 * Castrillon-Candas, "Spatial best linear unbiased prediction: a computational
 * mathematics approach for high dimensional massive datasets" (arXiv:1701.00285):
 *
 *   model       Z = X beta + eps, eps ~ N(0, C(theta))          (Sec. 2, eq. vectormodel)
 *   basis       kd-tree + multilevel basis W, with W X = 0      (Sec. 3.1, Algs. 1-3, steps 1-5)
 *   assembly    C~_W = entries psi^T C psi within distance tau  (Sec. 4, Algs. 4-7)
 *   solve       C~_W gamma_W = W Z by diagonal PCG, gamma = W^T gamma_W,
 *               beta = (X^T X)^{-1} X^T (Z - C gamma)            (Sec. 5.2, eqs. Spatial:eqn1-3; Sec. 6.2)
 *   predict     Z(x0) = k(x0)^T beta + c(x0)^T gamma            (Sec. 5.2, eq. Spatial)
 *   also        the gradient of a held-out loss in log(rho), log(nugget) (adjoint),
 *               the kriging MSE at targets (formula after eq. Spatial), the
 *               multilevel log-likelihood (Sec. 5.1) and many problems per call.
 *
 * Conventions (all entry points):
 *  - Every call returns an mlb_status; no exception crosses the ABI.  On error
 *    mlb_last_error(ctx) returns a message that stays valid until the next call.
 *  - Points are row-major double arrays (N x d), in the caller's order; every
 *    vector in or out (Z, gamma, predictions) is in the caller's order.  The
 *    kd-tree permutation is internal.
 *  - The caller owns every buffer it passes; the library copies inputs and
 *    writes outputs before returning (host variants) or in stream order on
 *    the context's stream (_dev variants, which take device pointers and do
 *    not synchronise).  The context owns all device memory it allocates.
 *  - Call order: mlb_build_basis -> mlb_assemble -> mlb_solve -> mlb_predict
 *    or mlb_grad (mlb_mse and mlb_loglik need only mlb_assemble).  A call
 *    made before its prerequisite returns MLB_ESTATE.
 *    A new mlb_build_basis invalidates the assembly and the solution; a new
 *    mlb_assemble invalidates the solution.
 *  - Covariance: Matern of any smoothness 0.2 <= nu <= 30 (Sec. 3.1) or the
 *    Gaussian kernel (Sec. 8.2), unit variance, Euclidean or anisotropic
 *    distance (Sec. 3); the nugget is added on the data diagonal only.
 *  - beta is reported on the library's monomial basis: total degree <= w,
 *    graded order, lexicographically decreasing exponents within a degree
 *    (1, x1, .., xd, x1^2, x1 x2, ..), evaluated on coordinates mapped onto
 *    [-1, 1]^d by the bounding box of the data points.
 */
#ifndef MLBLUP_H
#define MLBLUP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLB_ABI_VERSION 2

typedef struct mlb_ctx mlb_ctx;

typedef enum {
    MLB_OK = 0,
    MLB_EINVAL = 1,      /* bad argument (sizes, nu, NULL pointer, unsupported option) */
    MLB_ERANK = 2,       /* a local moment matrix or X is rank deficient (Sec. 2: X full column rank) */
    MLB_ENOCONV = 3,     /* PCG reached pcg_maxit before the tolerance */
    MLB_EBREAKDOWN = 4,  /* PCG found p^T A p <= 0 (truncated C~_W not positive definite) */
    MLB_ENOMEM = 5,      /* device allocation failed */
    MLB_ECUDA = 6,       /* a CUDA call failed (message has the CUDA error string) */
    MLB_ETIMEOUT = 7,    /* a bounded device wait gave up */
    MLB_ESTATE = 8       /* call made out of order */
} mlb_status;

enum { MLB_FP64 = 0, MLB_MIXED = 1 };

typedef struct {
    int precision;     /* MLB_FP64: every step in FP64.  MLB_MIXED: kernel tiles and
                          kernel sums in FP32 (FP64 accumulation across tiles), basis,
                          PCG vectors, inner products and the p x p trend solve in FP64 */
    int leaf_size;     /* kd-tree leaf size n0 (cells split while they hold more than n0 points) */
    double pcg_rtol;   /* stop when ||Z_W - C~_W g||_2 <= pcg_rtol ||Z_W||_2 (Sec. 6.2, remark) */
    int pcg_maxit;     /* iteration cap */
    int precond;       /* 1: P_W = diag(C~_W) (Sec. 5.2 remark); 0: P_W = I */
    int matrix_free;   /* 0: assembled C~_W; 1: three-step product W (C (W^T g)) (Sec. 6.2),
                          which needs tau = inf and keeps no matrix */
    int device;        /* CUDA device ordinal */
} mlb_opts;

enum { MLB_MATERN = 0, MLB_GAUSSIAN = 1 };

typedef struct {
    double nu;         /* Matern smoothness, 0.2 <= nu <= 30 (closed forms at 0.5, 1.5, 2.5;
                          any other value from the definition with K_nu, Sec. 3.1) */
    double rho;        /* Matern range, or the width theta of the Gaussian kernel (> 0) */
    double nugget;     /* eta >= 0, added to the covariance of the observations */
    int family;        /* MLB_MATERN, or MLB_GAUSSIAN: phi(r) = exp(-r^2 / (2 rho^2)) (Sec. 8.2);
                          nu is ignored for the Gaussian */
    int naxis;         /* 0: Euclidean distance; d: the anisotropic distance of Sec. 3,
                          r^2 = sum_k axis[k] (x_k - y_k)^2 */
    double axis[16];   /* axis weights theta_k > 0 (first naxis entries) */
} mlb_theta;

typedef struct {
    int iterations;            /* PCG iterations */
    int converged;             /* 1 if the tolerance was met */
    double rel_residual;       /* ||r_k|| / ||Z_W|| of the recursive PCG residual */
    int64_t nnz;               /* stored entries of C~_W (both triangles) */
    int64_t blocks;            /* stored cell-pair blocks (both triangles) */
    double ms_assemble;        /* device time of the last mlb_assemble */
    double ms_pcg;             /* device time of the PCG loop */
    double ms_beta;            /* device time of gamma = W^T g and the beta step */
    int64_t nnz_unique;        /* entries of the blocks j >= i (each symmetric pair once) */
    int64_t launches;          /* kernels this context has launched since mlb_create */
    int64_t col_total;         /* column indices stored (one list per row panel) */
    int64_t product_values;    /* matrix values one product C~_W u streams (FP32 on the
                                  mixed path, FP64 otherwise; 0 when matrix-free) */
    int symmetric;             /* 1: the product streams each symmetric pair of entries once
                                  (mixed path, every cell pair admissible); 0: both triangles */
    int product_variant;       /* form of the product chosen by timing at assembly: symmetric
                                  storage 0 plain loads, 1 bulk-copy pipeline; matrix-free
                                  kernel sum 0..5 launch shapes, 6 tensor cores */
} mlb_info;

/* Fills *opts with defaults: FP64, n0 = 64, rtol 1e-10, maxit 20000, diagonal
 * preconditioner, assembled matrix, device 0. */
void mlb_default_opts(mlb_opts* opts);

/* Creates a context on opts->device with its own CUDA stream.
 * Errors: MLB_EINVAL (bad options), MLB_ECUDA. */
mlb_status mlb_create(const mlb_opts* opts, mlb_ctx** out);

/* Frees every device buffer of the context.  NULL is accepted. */
void mlb_destroy(mlb_ctx* ctx);

const char* mlb_last_error(const mlb_ctx* ctx);
const char* mlb_status_string(mlb_status s);

/* Replaces the context's stream by a caller-owned cudaStream_t (NULL: back
 * to the context's own stream).  Later calls enqueue their kernels there. */
mlb_status mlb_set_stream(mlb_ctx* ctx, void* cuda_stream);

/* Kd-tree (Algs. 1-3) and multilevel basis (Sec. 3.1, steps 1-5) of N points
 * in d dimensions with the total-degree-w trend space, p = binom(d+w, w).
 * points: host, N x d row-major.  Needs N > p.  The basis is built in FP64:
 * each cell's orthonormal split of its moment matrix X^T B into scaling and
 * wavelet vectors comes from a Householder QR.  MLB_ERANK if some local
 * moment matrix is not of full rank min(p, s) (points not in general position). */
mlb_status mlb_build_basis(mlb_ctx* ctx, const double* points, int64_t N, int d, int w);
/* Same with points in device memory. */
mlb_status mlb_build_basis_dev(mlb_ctx* ctx, const double* points_dev, int64_t N, int d, int w);

/* Sparse multilevel covariance C~_W (Sec. 4, Algs. 4-7) for theta.  A pair of
 * cells (m of level i, q of level j) is kept when the bounding box of q's
 * points meets the box of m's points grown on every axis by
 * tau_ij = tau_factor * sqrt(Dbar_i Dbar_j), Dbar_l the mean box diagonal of
 * the cells of level l; tau_factor = INFINITY keeps every pair.  Also forms
 * P_W = diag(C~_W).  With opts.matrix_free = 1 only theta is recorded (tau_factor
 * must be INFINITY).  MLB_EINVAL: bad theta, leaf_size or 2p above 64 on the
 * assembled path. */
mlb_status mlb_assemble(mlb_ctx* ctx, const mlb_theta* theta, double tau_factor);

/* Solves for gamma and beta (eqs. Spatial:eqn2-3).  Z: host, N.  beta_out:
 * host, p entries, may be NULL.  info may be NULL.  MLB_ENOCONV / MLB_EBREAKDOWN
 * leave the last iterate in place (predict still works). */
mlb_status mlb_solve(mlb_ctx* ctx, const double* Z, double* beta_out, mlb_info* info);
/* Same with Z and beta_out in device memory (beta_out may be NULL). */
mlb_status mlb_solve_dev(mlb_ctx* ctx, const double* Z_dev, double* beta_dev, mlb_info* info);

/* Predictions at M targets (eq. Spatial).  targets: host M x d; yhat_out: host M. */
mlb_status mlb_predict(mlb_ctx* ctx, const double* targets, int64_t M, double* yhat_out);
mlb_status mlb_predict_dev(mlb_ctx* ctx, const double* targets_dev, int64_t M, double* yhat_dev);

/* Held-out loss L = mean_k (yhat_k - y_k)^2 and its derivatives in log(rho) and
 * log(nugget) by the adjoint of the saddle-point system (eq. Spatial:problem);
 * the adjoint is solved with the same multilevel PCG and the derivative blocks
 * dC/dlog(rho) are contracted on the fly, never stored.  Requires a solve.
 * Host pointers; any of the three outputs may be NULL. */
mlb_status mlb_grad(mlb_ctx* ctx, const double* targets, int64_t M, const double* y_obs,
                    double* loss_out, double* dlogrho_out, double* dlognugget_out);

/* Kriging mean squared error at M targets (the formula after eq. Spatial,
 * unit variance): MSE(x0) = 1 + u^T (X^T C^{-1} X)^{-1} u - c^T C^{-1} c with
 * u = X^T C^{-1} c - k(x0), c = c(x0), evaluated as 1 - c^T lambda - k^T mu
 * from the saddle-point system [[C, X], [X^T, 0]] [lambda; mu] = [c; k]; one
 * multilevel PCG solve on C~_W per target.  Requires mlb_assemble (not a
 * solve).  targets: host M x d row-major; mse_out: host M.  The _dev form
 * takes device buffers.  MLB_EBREAKDOWN / MLB_ENOCONV as for mlb_solve. */
mlb_status mlb_mse(mlb_ctx* ctx, const double* targets, int64_t M, double* mse_out);

/* Multilevel log-likelihood (Sec. 5.1, the reduced likelihood of the full
 * transform): l_W = -(N~/2) log(2 pi) - (1/2) log det C~_W - (1/2) Z_W^T
 * C~_W^{-1} Z_W, with Z_W = W Z and N~ = N - p.  The quadratic form comes from
 * the PCG solve; log det C~_W is estimated by stochastic Lanczos quadrature
 * (steps Lanczos steps, 1..100, fully reorthogonalised) over nprobe probe
 * vectors z_i that the caller draws in the data space (host, nprobe x N, caller
 * order; W z_i enters the Lanczos recurrence), e.g. Rademacher entries.  With
 * nprobe = 0 the log-determinant is not estimated and reported as 0.  Z: host,
 * N, caller order.  out3 = {l_W, log det estimate, quadratic form} (host).
 * Requires mlb_assemble.  The paper has no stochastic estimator: it uses a
 * sparse Cholesky factorisation. */
mlb_status mlb_loglik(mlb_ctx* ctx, const double* Z, const double* probes, int nprobe, int steps, double* out3);
mlb_status mlb_mse_dev(mlb_ctx* ctx, const double* targets_dev, int64_t M, double* out_dev);

/* ---- many independent problems -------------------------------------------- */

typedef struct {
    const double* points;   /* host, n x d row-major, caller order */
    int64_t n;
    int d;
    int w;                  /* trend degree */
    mlb_theta theta;
    double tau_factor;      /* INFINITY: all pairs */
    const double* Z;        /* host, n observations */
    const double* targets;  /* host, m x d */
    int64_t m;
    double* yhat;           /* host, m predictions (output) */
    double* beta;           /* host, p trend coefficients (output, may be NULL) */
    int status;             /* output: this problem's mlb_status */
    int iterations;         /* output: its PCG iterations */
} mlb_batch_problem;

/* Solves `count` independent multilevel BLUP problems (each: basis, assembly,
 * diagonal PCG, trend step, predictions, as for a single context with
 * `opts`).  Problems may differ in n, d, w, theta and tau.  The setup and
 * closing phases run on `host_threads` streams in parallel.  The PCG solves
 * of all problems of at most 12,288 unknowns run in one persistent launch,
 * their iterations cut into chunks that any CTA may take; wider systems run
 * the single-problem PCG on the stream pool meanwhile.  Results do not depend
 * on the scheduling: every reduction has a fixed order.  Returns
 * MLB_OK if every problem succeeded, else the first failing status (each
 * problem's own status is in probs[i].status).  ms_out (may be NULL): wall
 * time of the call.  opts->matrix_free must be 0. */
mlb_status mlb_batch_solve(const mlb_opts* opts, mlb_batch_problem* probs, int count, int host_threads,
                           double* ms_out);
/* Message of the last failing mlb_batch_solve on the calling thread ("" if none). */
const char* mlb_batch_last_error(void);
/* Wall-clock milliseconds of the last mlb_batch_solve on the calling thread,
 * by phase: [0] setup (basis, assembly, Z_W), [1] PCG, [2] closing (gamma,
 * trend, predictions, context release).  out: 3 doubles (host). */
void mlb_batch_last_phase_ms(double* out);
/* Kernels launched by the last mlb_batch_solve on the calling thread (all
 * problems' kernels plus the one persistent PCG launch). */
int64_t mlb_batch_last_launches(void);

/* ---- inspection (tests and tools) ---------------------------------------- */

/* The covariance function phi(r) of theta (deriv != 0: d phi / d log(rho)) at
 * n distances r (host arrays; the distance is passed in, so naxis is not
 * used), evaluated on the host exactly as the kernels evaluate it in FP64: the
 * closed forms, the Gaussian, or the table of Chebyshev pieces that
 * mlb_assemble builds for any other smoothness.  Needs no GPU and no context.
 * MLB_EINVAL for an invalid theta. */
mlb_status mlb_covariance(const mlb_theta* theta, const double* r, int64_t n, int deriv, double* out);

/* Sizes of the current basis.  Any pointer may be NULL. */
mlb_status mlb_get_sizes(const mlb_ctx* ctx, int64_t* N, int* d, int* p, int* t, int64_t* nwav);

/* perm[i] = caller index of the point at kd-tree position i (host, N entries). */
mlb_status mlb_get_perm(mlb_ctx* ctx, int32_t* perm);

/* gamma-hat of the last solve, caller order (host, N). */
mlb_status mlb_get_gamma(mlb_ctx* ctx, double* gamma);

/* out = W v (host, N -> N-p) and out = W^T u (host, N-p -> N). */
mlb_status mlb_apply_W(mlb_ctx* ctx, const double* v, double* out);
mlb_status mlb_apply_Wt(mlb_ctx* ctx, const double* u, double* out);

/* out = C~_W u with the assembled matrix (or the three-step product). Host, N-p. */
mlb_status mlb_cw_matvec(mlb_ctx* ctx, const double* u, double* out);
/* Same on device buffers (N-p doubles each), enqueued on the context's stream:
 * the very product one PCG iteration performs. */
mlb_status mlb_cw_matvec_dev(mlb_ctx* ctx, const double* u_dev, double* out_dev);

/* W v like mlb_apply_W, for callers that cannot allocate device memory at the
 * moment they need it (loops that must not block on the allocator, processes
 * held to a fixed device-memory budget, hosts whose device memory belongs to
 * another framework's pool).  The paper has no
 * counterpart: it only changes where the work space lives.  v_dev (N doubles,
 * caller order) and out_dev (N - p doubles) are device buffers owned by the
 * caller; the work space is one fixed 4 MiB array in device memory that every
 * GPU loading this library keeps until the process exits, so the call accepts
 * only N + (the scaling coefficients of all levels, about 2^(t+1) p) <= 524,288
 * and returns MLB_EINVAL beyond that.  Nothing is allocated or freed.  The
 * first call on a device looks up the array's device address on that device;
 * make that first call before any stream capture.  The kernels are enqueued on
 * the context's stream without synchronising.  All calls on one device share
 * the array: calls whose kernels overlap in time race. */
mlb_status mlb_apply_W_noalloc(mlb_ctx* ctx, const double* v_dev, double* out_dev);

/* Figures of the current assembly (nnz, nnz_unique, blocks, col_total,
 * product_values, symmetric, ms_assemble) and of the last solve (iterations,
 * converged, rel_residual, ms_pcg, ms_beta; zero before one), plus launches.
 * info: host.  MLB_ESTATE before mlb_assemble. */
mlb_status mlb_get_info(const mlb_ctx* ctx, mlb_info* info);

/* Forces the form of the product that mlb_assemble otherwise picks by timing
 * the candidates; for tests and measurements.  Symmetric FP32 storage: 0 plain
 * loads with L2 prefetch, 1 bulk-copy pipeline through shared memory (the two
 * add the FP32 products of a row in different orders, so they agree to FP32
 * rounding, not bit for bit).  Mixed matrix-free product: the FP32 kernel
 * sum's launch shape 0..5, or 6 for its tensor-core form (squared distances
 * as one BF16x3 contraction on the tensor cores; d = 5, 8 or 10 and a
 * closed-form Matern kind).  MLB_ESTATE for other assemblies; MLB_EINVAL for
 * values outside these. */
mlb_status mlb_set_product_variant(mlb_ctx* ctx, int variant);

/* Number of kernels the context has launched since mlb_create. */
mlb_status mlb_get_launch_count(const mlb_ctx* ctx, int64_t* count);

/* Pattern of the assembled matrix: flags[m * n_j + q] = 1 if cell m of level i
 * and cell q of level j form a stored block (host buffer of 2^i * 2^j bytes). */
mlb_status mlb_get_pattern(mlb_ctx* ctx, int i, int j, uint8_t* flags);

/* Kernel sum out_k = sum_j phi(|x0_k - x_j|) a_j over the data points (no
 * nugget): the primitive behind C gamma and c(x0)^T gamma.  Host pointers;
 * a in caller order. */
mlb_status mlb_kernel_sum(mlb_ctx* ctx, const double* targets, int64_t M, const double* a,
                          double* out);

#ifdef __cplusplus
}
#endif

#endif /* MLBLUP_H */
