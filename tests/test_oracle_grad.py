"""Pins of the adjoint gradient of the held-out loss (log rho, log nugget)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import grad


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_dense_gradient_matches_central_difference(nu):
    P = wl.small_problem(30, 220, 3, 1, nu=nu, rho=0.3, nugget=1e-3, leaf_size=16, with_y=True, M=60)
    L, g_rho, g_nug = grad.grad_dense(P.points, P.Z, P.targets, P.y_targets, 1, nu, P.rho, P.nugget)
    h = 1e-4
    f = lambda rho, nug: grad.loss_dense(P.points, P.Z, P.targets, P.y_targets, 1, nu, rho, nug)
    fd_rho = (f(P.rho * math.exp(h), P.nugget) - f(P.rho * math.exp(-h), P.nugget)) / (2 * h)
    fd_nug = (f(P.rho, P.nugget * math.exp(h)) - f(P.rho, P.nugget * math.exp(-h))) / (2 * h)
    assert abs(g_rho - fd_rho) <= 1e-6 * abs(fd_rho) + 1e-12
    assert abs(g_nug - fd_nug) <= 1e-6 * abs(fd_nug) + 1e-12
    assert abs(L - f(P.rho, P.nugget)) < 1e-14


def test_multilevel_gradient_equals_dense():
    P = wl.small_problem(31, 250, 2, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=16, with_y=True, M=40)
    d = grad.grad_dense(P.points, P.Z, P.targets, P.y_targets, 1, 1.5, 0.3, 1e-4)
    m = grad.grad_multilevel(P.points, P.Z, P.targets, P.y_targets, 1, 1.5, 0.3, 1e-4, 16)
    np.testing.assert_allclose(m, d, rtol=1e-7)
