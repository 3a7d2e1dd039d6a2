"""ctypes binding of libmlblup (include/mlblup.h), argument marshalling only.

Every numerical step runs in the library's CUDA kernels; this module checks
shapes and dtypes, passes pointers and raises ``MLBError`` on a non-zero
status.  Host-array methods take numpy float64 arrays; the ``*_dev`` methods
take raw device pointers (e.g. ``torch.Tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlblup.so")

MLB_FP64, MLB_MIXED = 0, 1
STATUS = {0: "ok", 1: "EINVAL", 2: "ERANK", 3: "ENOCONV", 4: "EBREAKDOWN", 5: "ENOMEM",
          6: "ECUDA", 7: "ETIMEOUT", 8: "ESTATE"}


class MLBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("leaf_size", ctypes.c_int), ("pcg_rtol", ctypes.c_double),
                ("pcg_maxit", ctypes.c_int), ("precond", ctypes.c_int), ("matrix_free", ctypes.c_int),
                ("device", ctypes.c_int)]


MLB_MATERN, MLB_GAUSSIAN = 0, 1
FAMILIES = {"matern": MLB_MATERN, "gaussian": MLB_GAUSSIAN}


class Theta(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("rho", ctypes.c_double), ("nugget", ctypes.c_double),
                ("family", ctypes.c_int), ("naxis", ctypes.c_int), ("axis", ctypes.c_double * 16)]


def make_theta(nu: float, rho: float, nugget: float, family: str = "matern", axis=None) -> Theta:
    """mlb_theta of a Matern (any nu) or Gaussian covariance, with optional
    axis weights theta_k of the anisotropic distance (None: Euclidean)."""
    th = Theta()
    th.nu = float(nu if nu is not None else 0.0)
    th.rho, th.nugget = float(rho), float(nugget)
    th.family = FAMILIES[family]
    if axis is not None:
        ax = [float(v) for v in axis]
        if len(ax) > 16:
            raise ValueError("at most 16 axis weights")
        th.naxis = len(ax)
        for i, v in enumerate(ax):
            th.axis[i] = v
    return th


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("nnz", ctypes.c_int64), ("blocks", ctypes.c_int64), ("ms_assemble", ctypes.c_double),
                ("ms_pcg", ctypes.c_double), ("ms_beta", ctypes.c_double),
                ("nnz_unique", ctypes.c_int64), ("launches", ctypes.c_int64), ("col_total", ctypes.c_int64),
                ("product_values", ctypes.c_int64), ("symmetric", ctypes.c_int),
                ("product_variant", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchProblem(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int), ("w", ctypes.c_int),
                ("theta", Theta), ("tau_factor", ctypes.c_double), ("Z", ctypes.c_void_p),
                ("targets", ctypes.c_void_p), ("m", ctypes.c_int64), ("yhat", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("status", ctypes.c_int), ("iterations", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
_SIGS = {
    "mlb_default_opts": (None, [ctypes.POINTER(Opts)]),
    "mlb_create": (ctypes.c_int, [ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "mlb_destroy": (None, [_P]),
    "mlb_last_error": (ctypes.c_char_p, [_P]),
    "mlb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mlb_set_stream": (ctypes.c_int, [_P, _P]),
    "mlb_build_basis": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, ctypes.c_int]),
    "mlb_build_basis_dev": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, ctypes.c_int]),
    "mlb_assemble": (ctypes.c_int, [_P, ctypes.POINTER(Theta), ctypes.c_double]),
    "mlb_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Info)]),
    "mlb_solve_dev": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Info)]),
    "mlb_predict": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mlb_predict_dev": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mlb_grad": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "mlb_mse": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mlb_loglik": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "mlb_mse_dev": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mlb_batch_solve": (ctypes.c_int, [ctypes.POINTER(Opts), ctypes.POINTER(BatchProblem), ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "mlb_batch_last_error": (ctypes.c_char_p, []),
    "mlb_batch_last_phase_ms": (None, [ctypes.POINTER(ctypes.c_double)]),
    "mlb_batch_last_launches": (ctypes.c_int64, []),
    "mlb_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(_I64)]),
    "mlb_get_perm": (ctypes.c_int, [_P, _P]),
    "mlb_get_gamma": (ctypes.c_int, [_P, _P]),
    "mlb_apply_W": (ctypes.c_int, [_P, _P, _P]),
    "mlb_apply_Wt": (ctypes.c_int, [_P, _P, _P]),
    "mlb_cw_matvec": (ctypes.c_int, [_P, _P, _P]),
    "mlb_cw_matvec_dev": (ctypes.c_int, [_P, _P, _P]),
    "mlb_get_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "mlb_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "mlb_covariance": (ctypes.c_int, [ctypes.POINTER(Theta), _P, _I64, ctypes.c_int, _P]),
    "mlb_set_product_variant": (ctypes.c_int, [_P, ctypes.c_int]),
    "mlb_apply_W_noalloc": (ctypes.c_int, [_P, _P, _P]),
    "mlb_get_pattern": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "mlb_kernel_sum": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
}

_lib = None


def lib():
    """Loads libmlblup.so from the package directory (fails loudly if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1701_00285_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def batch_solve(problems, precision: str = "fp64", leaf_size: int = 64, pcg_rtol: float = 1e-10,
                pcg_maxit: int = 20000, precond: bool = True, device: int = 0, host_threads: int = 8):
    """Solves independent problems with mlb_batch_solve.  `problems` is a list of
    dicts with points, w, nu, rho, nugget, tau_factor, Z, targets.  Returns
    (list of (yhat, beta, status, iterations), wall ms)."""
    L = lib()
    o = Opts()
    L.mlb_default_opts(ctypes.byref(o))
    o.precision = MLB_MIXED if precision == "mixed" else MLB_FP64
    o.leaf_size, o.pcg_rtol, o.pcg_maxit, o.precond, o.device = leaf_size, pcg_rtol, pcg_maxit, int(precond), device
    keep, arr = [], (BatchProblem * len(problems))()
    outs = []
    for i, q in enumerate(problems):
        pts = _f64(q["points"])
        Z = _f64(q["Z"], (pts.shape[0],))
        tg = _f64(q["targets"])
        d = pts.shape[1]
        p = math.comb(d + q["w"], q["w"])
        y = np.empty(tg.shape[0])
        beta = np.empty(p)
        keep += [pts, Z, tg, y, beta]
        a = arr[i]
        a.points, a.n, a.d, a.w = pts.ctypes.data, pts.shape[0], d, q["w"]
        a.theta = make_theta(q["nu"], q["rho"], q["nugget"], q.get("family", "matern"), q.get("axis"))
        a.tau_factor = float(q.get("tau_factor", math.inf))
        a.Z, a.targets, a.m = Z.ctypes.data, tg.ctypes.data, tg.shape[0]
        a.yhat, a.beta = y.ctypes.data, beta.ctypes.data
        outs.append((y, beta))
    ms = ctypes.c_double()
    st = L.mlb_batch_solve(ctypes.byref(o), arr, len(problems), host_threads, ctypes.byref(ms))
    res = [(y, b, arr[i].status, arr[i].iterations) for i, (y, b) in enumerate(outs)]
    if st != 0:
        import warnings
        warnings.warn("mlb_batch_solve: " + L.mlb_batch_last_error().decode())
    return res, ms.value, st


def covariance(r, nu: float, rho: float, family: str = "matern", deriv: bool = False) -> np.ndarray:
    """phi(r) (or d phi / d log(rho)) as the library's kernels evaluate it in
    FP64, computed on the host (mlb_covariance; no GPU needed)."""
    r = _f64(np.atleast_1d(r))
    out = np.empty_like(r)
    th = make_theta(nu, rho, 0.0, family)
    st = lib().mlb_covariance(ctypes.byref(th), _ptr(r), r.size, int(deriv), _ptr(out))
    if st != 0:
        raise MLBError(st, "mlb_covariance: invalid covariance parameters")
    return out


def batch_last_launches() -> int:
    """Kernels launched by the calling thread's last batch_solve."""
    return int(lib().mlb_batch_last_launches())


def batch_last_phase_ms() -> dict:
    """Per-phase wall-clock ms of the calling thread's last batch_solve."""
    out = (ctypes.c_double * 3)()
    lib().mlb_batch_last_phase_ms(out)
    return {"setup": out[0], "pcg": out[1], "finish": out[2]}


class Context:
    """One multilevel BLUP problem on one GPU (wraps an mlb_ctx)."""

    def __init__(self, precision: str = "fp64", leaf_size: int = 64, pcg_rtol: float = 1e-10,
                 pcg_maxit: int = 20000, precond: bool = True, matrix_free: bool = False, device: int = 0):
        L = lib()
        o = Opts()
        L.mlb_default_opts(ctypes.byref(o))
        o.precision = MLB_MIXED if precision == "mixed" else MLB_FP64
        o.leaf_size, o.pcg_rtol, o.pcg_maxit = leaf_size, pcg_rtol, pcg_maxit
        o.precond, o.matrix_free, o.device = int(precond), int(matrix_free), device
        h = _P()
        st = L.mlb_create(ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise MLBError(st, "mlb_create failed")
        self._h = h
        self.d = self.p = self.N = None

    def _check(self, st: int):
        if st != 0:
            raise MLBError(st, lib().mlb_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().mlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int | None):
        self._check(lib().mlb_set_stream(self._h, stream_ptr or None))

    def _sizes(self):
        N, nw = _I64(), _I64()
        d, p, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().mlb_get_sizes(self._h, ctypes.byref(N), ctypes.byref(d), ctypes.byref(p),
                                        ctypes.byref(t), ctypes.byref(nw)))
        self.N, self.d, self.p, self.t, self.nwav = N.value, d.value, p.value, t.value, nw.value

    def build_basis(self, points, w: int):
        pts = _f64(points)
        if pts.ndim != 2:
            raise ValueError("points must be (N, d)")
        self._check(lib().mlb_build_basis(self._h, _ptr(pts), pts.shape[0], pts.shape[1], w))
        self._sizes()

    def build_basis_dev(self, points_ptr: int, N: int, d: int, w: int):
        self._check(lib().mlb_build_basis_dev(self._h, points_ptr, N, d, w))
        self._sizes()

    def assemble(self, nu: float, rho: float, nugget: float, tau_factor: float = math.inf,
                 family: str = "matern", axis=None):
        th = make_theta(nu, rho, nugget, family, axis)
        self._check(lib().mlb_assemble(self._h, ctypes.byref(th), float(tau_factor)))

    def solve(self, Z, check: bool = True):
        Z = _f64(Z, (self.N,))
        beta = np.empty(self.p)
        info = Info()
        st = lib().mlb_solve(self._h, _ptr(Z), _ptr(beta), ctypes.byref(info))
        if check:
            self._check(st)
        return beta, info.as_dict()

    def solve_dev(self, Z_ptr: int, beta_ptr: int | None = None, check: bool = True):
        info = Info()
        st = lib().mlb_solve_dev(self._h, Z_ptr, beta_ptr or None, ctypes.byref(info))
        if check:
            self._check(st)
        return info.as_dict()

    def predict(self, targets):
        tg = _f64(targets)
        if tg.ndim != 2 or tg.shape[1] != self.d:
            raise ValueError("targets must be (M, d)")
        out = np.empty(tg.shape[0])
        self._check(lib().mlb_predict(self._h, _ptr(tg), tg.shape[0], _ptr(out)))
        return out

    def predict_dev(self, targets_ptr: int, M: int, out_ptr: int):
        self._check(lib().mlb_predict_dev(self._h, targets_ptr, M, out_ptr))

    def loglik(self, Z, probes=None, steps: int = 30):
        """(l_W, log det C~_W, Z_W^T C~_W^{-1} Z_W): the multilevel log-likelihood
        with the log-determinant estimated by stochastic Lanczos quadrature over
        the probe rows (data space, N entries each; None: no estimate)."""
        Z = _f64(Z, (self.N,))
        if probes is None:
            pr, m = None, 0
        else:
            pr = _f64(probes)
            if pr.ndim != 2 or pr.shape[1] != self.N:
                raise ValueError("probes must be (m, N)")
            m = pr.shape[0]
        out = np.empty(3)
        self._check(lib().mlb_loglik(self._h, _ptr(Z), _ptr(pr) if pr is not None else None, m, steps, _ptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def mse(self, targets) -> np.ndarray:
        """Kriging mean squared error at the targets (one PCG solve each)."""
        tg = _f64(targets)
        if tg.ndim != 2 or tg.shape[1] != self.d:
            raise ValueError("targets must be (M, d)")
        out = np.empty(tg.shape[0])
        self._check(lib().mlb_mse(self._h, _ptr(tg), tg.shape[0], _ptr(out)))
        return out

    def mse_dev(self, targets_ptr: int, M: int, out_ptr: int):
        self._check(lib().mlb_mse_dev(self._h, targets_ptr, M, out_ptr))

    def grad(self, targets, y_obs):
        tg = _f64(targets)
        y = _f64(y_obs, (tg.shape[0],))
        loss, g1, g2 = (ctypes.c_double() for _ in range(3))
        self._check(lib().mlb_grad(self._h, _ptr(tg), tg.shape[0], _ptr(y), ctypes.byref(loss),
                                   ctypes.byref(g1), ctypes.byref(g2)))
        return loss.value, g1.value, g2.value

    # --- inspection ---------------------------------------------------------
    def perm(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int32)
        self._check(lib().mlb_get_perm(self._h, out.ctypes.data_as(_P)))
        return out

    def gamma(self) -> np.ndarray:
        out = np.empty(self.N)
        self._check(lib().mlb_get_gamma(self._h, _ptr(out)))
        return out

    def apply_W(self, v) -> np.ndarray:
        v = _f64(v, (self.N,))
        out = np.empty(self.nwav)
        self._check(lib().mlb_apply_W(self._h, _ptr(v), _ptr(out)))
        return out

    def apply_Wt(self, u) -> np.ndarray:
        u = _f64(u, (self.nwav,))
        out = np.empty(self.N)
        self._check(lib().mlb_apply_Wt(self._h, _ptr(u), _ptr(out)))
        return out

    def cw_matvec(self, u) -> np.ndarray:
        u = _f64(u, (self.nwav,))
        out = np.empty(self.nwav)
        self._check(lib().mlb_cw_matvec(self._h, _ptr(u), _ptr(out)))
        return out

    def cw_matvec_dev(self, u_ptr: int, out_ptr: int):
        self._check(lib().mlb_cw_matvec_dev(self._h, u_ptr, out_ptr))

    def apply_W_noalloc(self, v_ptr: int, out_ptr: int):
        """W v on caller-owned device buffers, with no device allocation."""
        self._check(lib().mlb_apply_W_noalloc(self._h, v_ptr, out_ptr))

    def info(self) -> dict:
        """Figures of the current assembly and of the last solve (mlb_get_info)."""
        info = Info()
        self._check(lib().mlb_get_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def set_product_variant(self, variant: int):
        """Forces the form of the symmetric FP32 product (0 loads, 1 bulk copies)."""
        self._check(lib().mlb_set_product_variant(self._h, variant))

    def launch_count(self) -> int:
        c = _I64()
        self._check(lib().mlb_get_launch_count(self._h, ctypes.byref(c)))
        return c.value

    def pattern(self, i: int, j: int) -> np.ndarray:
        out = np.zeros((1 << i) * (1 << j), dtype=np.uint8)
        self._check(lib().mlb_get_pattern(self._h, i, j, out.ctypes.data_as(_P)))
        return out.reshape(1 << i, 1 << j).astype(bool)

    def kernel_sum(self, targets, a) -> np.ndarray:
        tg = _f64(targets)
        a = _f64(a, (self.N,))
        out = np.empty(tg.shape[0])
        self._check(lib().mlb_kernel_sum(self._h, _ptr(tg), tg.shape[0], _ptr(a), _ptr(out)))
        return out
