"""CPU FP64 oracle for metric magnitude (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
it shares no code with the CUDA path.  The arithmetic lives in ``oracle.c``
(plain C, IEEE double, libm ``sqrt``/``exp``); this module only marshals numpy
arrays.  Each wrapper names the passage of the paper it follows.

Parity status: every function below is pinned by a CPU test
(``tests/test_oracle_pins.py``) against closed forms, invariants, values the
paper prints, or library routines; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status codes of oracle.c
OK, EINVAL, EDUPLICATE, ENOTPD, ENOBRACKET, ENOMEM = 0, 1, 2, 3, 5, 6


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no fast-math,
    no FMA contraction so x86 and Arm give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            sig = {
                "orc_num_threads": (i32, []),
                "orc_sum": (d, [P, i64]),
                "orc_distance": (d, [P, i64, i64, i64]),
                "orc_distance_matrix": (None, [P, i64, i64, P]),
                "orc_similarity_matrix": (None, [P, i64, i64, d, P]),
                "orc_min_distance": (d, [P, i64, i64]),
                "orc_tplus_bound": (d, [P, i64, i64]),
                "orc_cholesky": (i32, [P, i64]),
                "orc_forward": (None, [P, i64, P, P]),
                "orc_backward": (None, [P, i64, P, P]),
                "orc_residual_rows": (None, [P, i64, i64, d, P, P, P, i64, P, P]),
                "orc_relative_residual": (d, [P, i64, i64, d, P, P]),
                "orc_solve": (i32, [P, i64, i64, d, P, i32, P, P]),
                "orc_weighting": (i32, [P, i64, i64, d, i32, P, P]),
                "orc_tplus": (i32, [P, i64, i64, d, d, d, i32, P, P, P, P, P]),
                "orc_tplus_ridders": (i32, [P, i64, i64, d, d, d, i32, P, P, P, P, P]),
                "orc_scale_zero": (i32, [P, i64, i64, i32, P, P]),
                "orc_grad": (None, [P, i64, i64, d, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def num_threads() -> int:
    return int(_load().orc_num_threads())


def kahan_sum(v) -> float:
    v = _c(v)
    return float(_load().orc_sum(_p(v), v.size))


def distance_matrix(X):
    """Sec. 2: d_jk = ||x_j - x_k|| from coordinate differences."""
    X = _c(X)
    n, m = X.shape
    D = np.empty((n, n))
    _load().orc_distance_matrix(_p(X), n, m, _p(D))
    return D


def similarity_matrix(X, t):
    """Sec. 2: Z = exp[-t d]."""
    X = _c(X)
    n, m = X.shape
    Z = np.empty((n, n))
    _load().orc_similarity_matrix(_p(X), n, m, float(t), _p(Z))
    return Z


def min_distance(X) -> float:
    X = _c(X)
    return float(_load().orc_min_distance(_p(X), X.shape[0], X.shape[1]))


def tplus_bound(X) -> float:
    """Sec. 1: t_+ <= log(n-1) / min_{j != k} d_jk."""
    X = _c(X)
    return float(_load().orc_tplus_bound(_p(X), X.shape[0], X.shape[1]))


def cholesky(A):
    """Sec. 3.2: lower Cholesky factor (left-looking), ENOTPD on a non-positive pivot."""
    L = _c(A).copy()
    st = _load().orc_cholesky(_p(L), L.shape[0])
    if st:
        raise OracleError(ENOTPD, f"cholesky (pivot {st - 1})")
    return L


def forward(L, b):
    L, b = _c(L), _c(b)
    y = np.empty_like(b)
    _load().orc_forward(_p(L), L.shape[0], _p(b), _p(y))
    return y


def backward(L, y):
    L, y = _c(L), _c(y)
    x = np.empty_like(y)
    _load().orc_backward(_p(L), L.shape[0], _p(y), _p(x))
    return x


def residual_rows(X, t, w, rows=None, b=None):
    """r_j = b_j - sum_k Z_jk w_k (Z regenerated, compensated sums) and the row sums of Z."""
    X, w = _c(X), _c(w)
    n, m = X.shape
    bb = None if b is None else _c(b)
    rr = None if rows is None else _c(rows, np.int64)
    cnt = n if rr is None else rr.size
    r = np.empty(cnt)
    rs = np.empty(cnt)
    _load().orc_residual_rows(_p(X), n, m, float(t), _p(w), _p(bb), _p(rr), cnt, _p(r), _p(rs))
    return r, rs


def relative_residual(X, t, w, b=None) -> float:
    """||b - Zw||_inf / (||Z||_inf ||w||_inf)."""
    X, w = _c(X), _c(w)
    bb = None if b is None else _c(b)
    return float(_load().orc_relative_residual(_p(X), X.shape[0], X.shape[1], float(t), _p(w), _p(bb)))


def solve(X, t, b=None, ir_steps=2):
    """Solve Z x = b (b = 1 gives the weighting).  Returns (x, info dict)."""
    X = _c(X)
    n, m = X.shape
    bb = None if b is None else _c(b)
    x = np.empty(n)
    info = np.empty(3)
    st = _load().orc_solve(_p(X), n, m, float(t), _p(bb), int(ir_steps), _p(x), _p(info))
    if st:
        raise OracleError(st, "solve")
    return x, {"rel_residual": info[0], "z_norm_inf": info[1], "x_norm_inf": info[2]}


def weighting(X, t, ir_steps=2):
    """Sec. 2, Eq. weighting: w with Zw = 1 and Mag = 1^T w.
    Returns (w, mag, info) with info = rel_residual, min_w, max_abs_w."""
    X = _c(X)
    n, m = X.shape
    w = np.empty(n)
    out = np.empty(4)
    st = _load().orc_weighting(_p(X), n, m, float(t), int(ir_steps), _p(w), _p(out))
    if st:
        raise OracleError(st, "weighting")
    return w, float(out[0]), {"rel_residual": out[1], "min_w": out[2], "max_abs_w": out[3]}


def weighting_lapack(X, t, ir_steps=2):
    """Sec. 2, Eq. weighting with a library Cholesky as the factor step: Z from
    orc_similarity_matrix, Z = L L^T by LAPACK's dpotrf (scipy), the solve with
    L, then `ir_steps` FP64 refinement steps whose residual is orc_residual_rows
    (compensated row sums, Z regenerated); Mag by the compensated sum.  The
    same steps as ``weighting`` with the plain C Cholesky replaced by the
    library one, for sizes where the plain loops take minutes (n >= 32768).
    Returns (w, mag, info) like ``weighting``, info also holding LAPACK's
    estimate of kappa_1(Z) (dpocon); pinned by the same closed forms and by
    agreement with ``weighting``."""
    import scipy.linalg
    X = _c(X)
    n, m = X.shape
    Z = similarity_matrix(X, t)
    # Z is symmetric: its transpose is the Fortran-ordered matrix LAPACK
    # factors in place
    c = scipy.linalg.cho_factor(Z.T, lower=True, overwrite_a=True, check_finite=False)
    w = scipy.linalg.cho_solve(c, np.ones(n), check_finite=False)
    rs = None
    for _ in range(ir_steps):
        r, rs = residual_rows(X, t, w)
        w = w + scipy.linalg.cho_solve(c, r, check_finite=False)
    if rs is None:
        rs = residual_rows(X, t, w)[1]
    # LAPACK's estimate of 1/kappa_1(Z) from the factor (dpocon; ||Z||_1 is
    # the largest row sum, Z being symmetric with positive entries)
    rcond, _ = scipy.linalg.lapack.dpocon(c[0], float(rs.max()), uplo="L")
    del c, Z
    return w, kahan_sum(w), {"rel_residual": relative_residual(X, t, w), "min_w": float(w.min()),
                             "max_abs_w": float(np.abs(w).max()),
                             "kappa1_est": (1.0 / rcond) if rcond > 0 else float("inf")}


def magnitude(X, t, ir_steps=2) -> float:
    return weighting(X, t, ir_steps)[1]


def tplus(X, t_lo=1e-3, t_hi=0.0, rel_tol=1e-6, ir_steps=2, method="bisection"):
    """Sec. 2 cutoff by bisection (default) or Ridders' method on min_j w_j(t).
    Returns dict with t_plus, bracket, below, probes, w, mag.  t_hi <= 0 uses
    the Sec. 1 bound."""
    X = _c(X)
    n, m = X.shape
    out = np.zeros(3)
    below = ctypes.c_int(0)
    probes = ctypes.c_int(0)
    w = np.empty(n)
    mag = ctypes.c_double(0.0)
    fn = {"bisection": _load().orc_tplus, "ridders": _load().orc_tplus_ridders}[method]
    st = fn(_p(X), n, m, float(t_lo), float(t_hi), float(rel_tol), int(ir_steps),
            _p(out), ctypes.byref(below), ctypes.byref(probes), _p(w), ctypes.byref(mag))
    if st:
        raise OracleError(st, "tplus")
    return {"t_plus": out[0], "bracket": (out[1], out[2]), "below": bool(below.value),
            "probes": probes.value, "w": w, "mag": mag.value}


def scale_zero(X, ir_steps=2):
    """App. C, Eq. scaleZero: w0 = d^{-1} 1 / (1^T d^{-1} 1) by a pivoted LU of
    the distance matrix and FP64 refinement.  Returns (w0, s = 1^T d^{-1} 1,
    info with the relative residual of d v = 1 and ||d||_inf)."""
    X = _c(X)
    n, m = X.shape
    w0 = np.empty(n)
    out = np.zeros(3)
    st = _load().orc_scale_zero(_p(X), n, m, int(ir_steps), _p(w0), _p(out))
    if st:
        raise OracleError(st, "scale_zero")
    return w0, float(out[0]), {"rel_residual": float(out[1]), "d_norm_inf": float(out[2])}


def grad(X, t, w=None, lam=None):
    """Adjoint gradients (implicit differentiation of Zw = 1).

    lam = Z^{-1} dL/dw; lam = None means L = Mag (lam = w).  Returns
    (dL_dt, dL_dx[n, m])."""
    X = _c(X)
    n, m = X.shape
    if w is None:
        w = weighting(X, t)[0]
    w = _c(w)
    lam = w if lam is None else _c(lam)
    dt = ctypes.c_double(0.0)
    dx = np.empty((n, m))
    _load().orc_grad(_p(X), n, m, float(t), _p(w), _p(lam), ctypes.byref(dt), _p(dx))
    return dt.value, dx


def grad_loss(X, t, dL_dw, w=None, ir_steps=2):
    """Gradient of a general loss L(w): lambda = Z^{-1} dL/dw by the oracle solve."""
    X = _c(X)
    if w is None:
        w = weighting(X, t, ir_steps)[0]
    lam, _ = solve(X, t, b=_c(dL_dw), ir_steps=ir_steps)
    return grad(X, t, w, lam)
