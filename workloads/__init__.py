"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws random inputs: point clouds, observation vectors,
target points and covariance parameters.  It holds none of the method's
arithmetic (no design matrix, no covariance, no tree, no basis) and is the
one module shared by the CPU oracle and the GPU path.

The paper's own data sets (nested random n-sphere and hypercube point sets,
and Gaussian-random-field "normal test data", Sec. "Experimental setup") were
generated on a cluster and are not available, so these recipes stand in for
them.  Every array comes from its own PCG64 stream spawned from
``SeedSequence(BASE_SEED + config_id)``.

Observation recipe (all configs): ``Z = trend(x) + sum_k sin(w_k . x) +
noise``.  The trend is a polynomial of total degree <= w in the fixed affine
map ``u = 2x - 1`` of the unit cube, with standard-normal coefficients on the
monomials ``u^alpha`` (|alpha| <= w); being a polynomial of degree <= w it
lies in the span of the method's design matrix for any affine rescaling of
the coordinates.  Frequencies ``w_k = r_k * v_k`` with ``v_k`` uniform on the
unit sphere and ``r_k ~ U[0, 8]`` (so ``|w_k| <= 8``); noise is Gaussian with
the stated variance.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 170100285

__all__ = [
    "BASE_SEED", "Problem", "dense_2d", "clustered_3d", "uniform_10d", "batched_problems",
    "heldout_5d", "small_problem", "subsample", "unit_disk_gaussian", "TABLE5_ROWS",
]


@dataclass
class Problem:
    """One BLUP problem: inputs only (no derived quantities)."""
    name: str
    points: np.ndarray          # (N, d) float64, user order
    Z: np.ndarray               # (N,) float64 observations
    targets: np.ndarray         # (M, d) float64 prediction locations
    nu: float                   # Matern smoothness
    rho: float                  # Matern range (Gaussian kernel: its width theta)
    nugget: float               # variance added on the data diagonal
    w: int                      # total degree of the polynomial trend space
    leaf_size: int              # kd-tree leaf size n0
    tau_factor: float           # distance threshold in cell diameters (inf = all pairs)
    pcg_rtol: float = 1e-10
    y_targets: np.ndarray | None = None   # held-out observations (differentiation config)
    meta: dict = field(default_factory=dict)
    family: str = "matern"      # or "gaussian"

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])


def _streams(config_id: int, n: int):
    ss = np.random.SeedSequence(BASE_SEED + config_id)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


def _exponents(d: int, w: int):
    out = []
    for alpha in itertools.product(range(w + 1), repeat=d):
        if sum(alpha) <= w:
            out.append(alpha)
    return out


def _trend(x: np.ndarray, w: int, coef: np.ndarray) -> np.ndarray:
    u = 2.0 * x - 1.0
    val = np.zeros(x.shape[0])
    for c, alpha in zip(coef, _exponents(x.shape[1], w)):
        term = np.ones(x.shape[0])
        for k, a in enumerate(alpha):
            if a:
                term = term * u[:, k] ** a
        val += c * term
    return val


def _frequencies(rng, d: int, count: int) -> np.ndarray:
    v = rng.standard_normal((count, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = rng.uniform(0.0, 8.0, size=(count, 1))
    return v * r


def _observe(x, w, coef, omega, noise):
    z = _trend(x, w, coef)
    if omega is not None and len(omega):
        z = z + np.sin(x @ omega.T).sum(axis=1)
    if noise is not None:
        z = z + noise
    return z


def _mixture(rng, n, d, centres, sigma):
    lab = rng.integers(0, centres.shape[0], size=n)
    return centres[lab] + sigma * rng.standard_normal((n, d))


def dense_2d() -> Problem:
    """Dense BLUP check: 1,000 uniform points in [0,1]^2, exponential kernel."""
    r_pts, r_beta, r_tgt = _streams(1, 3)
    N, d, w = 1000, 2, 1
    x = r_pts.uniform(0.0, 1.0, size=(N, d))
    coef = r_beta.standard_normal(math.comb(d + w, w))
    z = _trend(x, w, coef) + np.sin(4 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    tg = r_tgt.uniform(0.0, 1.0, size=(200, d))
    return Problem("dense_2d_n1000", x, z, tg, nu=0.5, rho=0.25, nugget=0.0,
                   w=w, leaf_size=64, tau_factor=math.inf, pcg_rtol=1e-12,
                   meta={"trend_coef": coef})


def clustered_3d(N: int = 65536, M: int = 16384) -> Problem:
    """Multilevel FP64: half uniform, half 8-centre Gaussian mixture in [0,1]^3."""
    r_pts, r_mix, r_beta, r_om, r_noise, r_tgt = _streams(2, 6)
    d, w = 3, 2
    centres = r_mix.uniform(0.0, 1.0, size=(8, d))
    nu_ = N // 2
    x = np.concatenate([r_pts.uniform(0.0, 1.0, size=(nu_, d)),
                        _mixture(r_mix, N - nu_, d, centres, 0.03)])
    coef = r_beta.standard_normal(math.comb(d + w, w))
    omega = _frequencies(r_om, d, 16)
    noise = math.sqrt(1e-4) * r_noise.standard_normal(N)
    z = _observe(x, w, coef, omega, noise)
    mt = M // 2
    tg = np.concatenate([r_tgt.uniform(0.0, 1.0, size=(mt, d)),
                         _mixture(r_tgt, M - mt, d, centres, 0.03)])
    return Problem(f"clustered_3d_n{N}", x, z, tg, nu=1.5, rho=0.2, nugget=1e-6,
                   w=w, leaf_size=64, tau_factor=2.0, pcg_rtol=1e-10,
                   meta={"trend_coef": coef, "omega": omega})


def uniform_10d(N: int = 262144, M: int = 65536) -> Problem:
    """Mixed precision, high dimension: uniform points in [0,1]^10."""
    r_pts, r_beta, r_om, r_noise, r_tgt = _streams(3, 5)
    d, w = 10, 2
    x = r_pts.uniform(0.0, 1.0, size=(N, d))
    coef = r_beta.standard_normal(math.comb(d + w, w))
    omega = _frequencies(r_om, d, 32)
    noise = math.sqrt(1e-4) * r_noise.standard_normal(N)
    z = _observe(x, w, coef, omega, noise)
    tg = r_tgt.uniform(0.0, 1.0, size=(M, d))
    return Problem(f"uniform_10d_n{N}", x, z, tg, nu=2.5, rho=0.5, nugget=1e-5,
                   w=w, leaf_size=128, tau_factor=math.inf, pcg_rtol=1e-8,
                   meta={"trend_coef": coef, "omega": omega})


def batched_problems(count: int = 512, M: int = 1024, n_lo: int = 500, n_hi: int = 8000) -> list[Problem]:
    """Batched: independent problems with log-uniform sizes, mixed d, nu, rho.

    tau = infinity (the exact BLUP of every problem): with tau = 2 level-mean
    diameters the truncated C~_W of long-range problems is indefinite (the
    first problem, n = 4,678, d = 2, rho = 0.445, has 162 negative eigenvalues,
    lambda_min = -0.069), so no BLUP exists for it."""
    r_meta, r_pts, r_beta, r_om, r_noise, r_tgt = _streams(4, 6)
    probs = []
    for i in range(count):
        n = int(round(math.exp(r_meta.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(r_meta.choice([2, 3, 5]))
        nu = float(r_meta.choice([0.5, 1.5, 2.5]))
        rho = float(r_meta.uniform(0.1, 0.5))
        w = 1
        x = r_pts.uniform(0.0, 1.0, size=(n, d))
        coef = r_beta.standard_normal(math.comb(d + w, w))
        omega = _frequencies(r_om, d, 8)
        noise = 1e-2 * r_noise.standard_normal(n)
        z = _observe(x, w, coef, omega, noise)
        tg = r_tgt.uniform(0.0, 1.0, size=(M, d))
        probs.append(Problem(f"batch{i}_n{n}_d{d}", x, z, tg, nu=nu, rho=rho,
                             nugget=1e-4, w=w, leaf_size=64, tau_factor=math.inf,
                             pcg_rtol=1e-10, meta={"trend_coef": coef}))
    return probs


def heldout_5d(N: int = 32768, M: int = 4096) -> Problem:
    """Differentiation: uniform points in [0,1]^5 with held-out observations."""
    r_pts, r_beta, r_om, r_noise, r_tgt, r_tnoise = _streams(5, 6)
    d, w = 5, 1
    x = r_pts.uniform(0.0, 1.0, size=(N, d))
    coef = r_beta.standard_normal(math.comb(d + w, w))
    omega = _frequencies(r_om, d, 16)
    z = _observe(x, w, coef, omega, math.sqrt(1e-4) * r_noise.standard_normal(N))
    tg = r_tgt.uniform(0.0, 1.0, size=(M, d))
    yt = _observe(tg, w, coef, omega, math.sqrt(1e-4) * r_tnoise.standard_normal(M))
    return Problem(f"heldout_5d_n{N}", x, z, tg, nu=1.5, rho=0.3, nugget=1e-4,
                   w=w, leaf_size=64, tau_factor=math.inf, pcg_rtol=1e-10,
                   y_targets=yt, meta={"trend_coef": coef, "omega": omega})


# (alpha, theta) of the rows of the paper's accuracy table (Sec. 8.2, Table 5)
TABLE5_ROWS = ((1.0, 10.0), (0.5, 10.0), (2.0, 10.0), (2.0, 3.0), (0.5, 3.0))


def unit_disk_gaussian(alpha: float, theta: float, N: int = 200, M: int = 200) -> Problem:
    """The ill-conditioned accuracy study (Sec. 8.2, Table 5): N points drawn
    uniformly on the unit disk (radius sqrt(U), angle 2 pi V), the Gaussian
    kernel exp(-r^2 / (2 theta^2)), no nugget, trend degree w = 8 (p = 45),
    observations Z = 1 + sin(alpha x1) sin(alpha x2) without noise, M targets
    drawn the same way.  The paper does not give its points; these are one
    seeded draw, the same for every (alpha, theta)."""
    r_pts, r_tgt = _streams(6, 2)

    def disk(rng, n):
        rad = np.sqrt(rng.uniform(0.0, 1.0, size=n))
        ang = 2.0 * np.pi * rng.uniform(0.0, 1.0, size=n)
        return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)

    x = disk(r_pts, N)
    tg = disk(r_tgt, M)
    z = 1.0 + np.sin(alpha * x[:, 0]) * np.sin(alpha * x[:, 1])
    return Problem(f"unit_disk_gaussian_a{alpha:g}_t{theta:g}", x, z, tg, nu=math.inf, rho=theta,
                   nugget=0.0, w=8, leaf_size=64, tau_factor=math.inf, pcg_rtol=1e-14,
                   meta={"alpha": alpha, "theta": theta}, family="gaussian")


def small_problem(seed: int, N: int, d: int, w: int, nu: float = 1.5, rho: float = 0.3,
                  nugget: float = 1e-6, leaf_size: int = 16, tau_factor: float = math.inf,
                  M: int = 32, clustered: bool = False, with_y: bool = False) -> Problem:
    """Small seeded problem for parity tests (same recipe, any size)."""
    streams = _streams(1000 + seed, 7)
    r_pts, r_mix, r_beta, r_om, r_noise, r_tgt, r_tn = streams
    if clustered:
        centres = r_mix.uniform(0.0, 1.0, size=(4, d))
        h = N // 2
        x = np.concatenate([r_pts.uniform(0.0, 1.0, size=(h, d)),
                            _mixture(r_mix, N - h, d, centres, 0.03)])
    else:
        x = r_pts.uniform(0.0, 1.0, size=(N, d))
    coef = r_beta.standard_normal(math.comb(d + w, w))
    omega = _frequencies(r_om, d, 8)
    z = _observe(x, w, coef, omega, 1e-2 * r_noise.standard_normal(N))
    tg = r_tgt.uniform(0.0, 1.0, size=(M, d))
    yt = _observe(tg, w, coef, omega, 1e-2 * r_tn.standard_normal(M)) if with_y else None
    return Problem(f"small_s{seed}_n{N}_d{d}_w{w}", x, z, tg, nu=nu, rho=rho, nugget=nugget,
                   w=w, leaf_size=leaf_size, tau_factor=tau_factor, pcg_rtol=1e-12,
                   y_targets=yt, meta={"trend_coef": coef, "omega": omega})


def subsample(prob: Problem, n: int, seed: int = 0, m: int | None = None) -> Problem:
    """Seeded subsample of a problem's data (and optionally its targets)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 7919 * (seed + 1)))
    idx = np.sort(rng.choice(prob.N, size=n, replace=False))
    tg = prob.targets
    yt = prob.y_targets
    if m is not None and m < tg.shape[0]:
        tidx = np.sort(rng.choice(tg.shape[0], size=m, replace=False))
        tg = tg[tidx]
        yt = yt[tidx] if yt is not None else None
    return Problem(prob.name + f"_sub{n}", prob.points[idx].copy(), prob.Z[idx].copy(),
                   tg.copy(), prob.nu, prob.rho, prob.nugget, prob.w, prob.leaf_size,
                   prob.tau_factor, prob.pcg_rtol, None if yt is None else yt.copy(),
                   dict(prob.meta), prob.family)
