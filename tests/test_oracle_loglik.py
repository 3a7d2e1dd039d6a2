"""Pins of the oracle's multilevel log-likelihood and its stochastic Lanczos
quadrature (CPU), each against something other than the oracle's own code."""
import math

import numpy as np

import workloads as wl
from oracle import design, loglik, matern, mlblup


def test_slq_with_all_unit_probes_is_exact():
    """Lanczos run to the full dimension from e_i reproduces (log A)_ii exactly,
    so the estimator over all n unit vectors is tr log A = log det A."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Q @ np.diag(np.logspace(-2, 2, 12)) @ Q.T
    est = loglik.slq_logdet(A, np.eye(12), 12)
    assert abs(est - np.linalg.slogdet(A)[1]) < 1e-10


def test_slq_statistical_accuracy_with_rademacher_probes():
    """Many Rademacher probes, few Lanczos steps: the estimate is unbiased and
    concentrates around log det (a loose bound for a seeded draw)."""
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((200, 200)))
    A = Q @ np.diag(np.logspace(-1, 1, 200)) @ Q.T
    probes = rng.choice([-1.0, 1.0], size=(400, 200))
    est = loglik.slq_logdet(A, probes, 25)
    exact = np.linalg.slogdet(A)[1]
    # Hutchinson's estimator with Rademacher probes has variance
    # 2 sum_{i != j} (log A)_ij^2 per probe; allow four standard deviations
    lam, U = np.linalg.eigh(A)
    L = (U * np.log(lam)) @ U.T
    sd = math.sqrt(2.0 * (np.sum(L ** 2) - np.sum(np.diag(L) ** 2)) / probes.shape[0])
    assert abs(est - exact) < 4.0 * sd


def test_log_det_of_cw_matches_the_dense_identity():
    """With [W; L] orthonormal and L spanning the trend, det C = det C_W /
    det(L C^{-1} L^T); in terms of X = L^T R: log det C_W = log det C +
    log det(X^T C^{-1} X) - log det(X^T X).  Independent of the multilevel
    assembly and of any Lanczos estimate."""
    P = wl.small_problem(31, 140, 2, 1, nu=1.5, rho=0.3, nugget=1e-3, leaf_size=12)
    B = mlblup.setup(P.points, P.w, P.leaf_size)
    l, logdet, quad = loglik.multilevel_loglik(B, P.points, P.Z, P.nu, P.rho, P.nugget)
    C = matern.covariance(P.points, P.nu, P.rho, P.nugget)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, P.w, lo, hi)
    Ci_X = np.linalg.solve(C, X)
    ref = np.linalg.slogdet(C)[1] + np.linalg.slogdet(X.T @ Ci_X)[1] - np.linalg.slogdet(X.T @ X)[1]
    assert abs(logdet - ref) < 1e-9 * max(1.0, abs(ref))
    # the quadratic form is the REML one: Z^T (C^-1 - C^-1 X (X^T C^-1 X)^-1 X^T C^-1) Z
    Ci_Z = np.linalg.solve(C, P.Z)
    q_ref = P.Z @ Ci_Z - (X.T @ Ci_Z) @ np.linalg.solve(X.T @ Ci_X, X.T @ Ci_Z)
    assert abs(quad - q_ref) < 1e-9 * abs(q_ref)
    n = P.N - B.p
    assert abs(l + 0.5 * (n * math.log(2 * math.pi) + logdet + quad)) < 1e-12 * abs(l)
