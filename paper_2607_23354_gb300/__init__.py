"""GB300 metric-magnitude solver: Python binding of the C ABI in
``include/magnitude.h`` (ctypes; argument marshalling only).

Every step of the computation runs in the CUDA kernels of
``_build/libmagnitude.so``.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: importing works anywhere, but every call
raises ``RuntimeError`` when the library is not built or no CUDA device is
present.

Paper: "Scalably computing metric magnitude" (arXiv 2607.23354), Sec. 2:
Z = exp[-t d] for Euclidean d, the weighting w solves Zw = 1 (Eq. weighting),
the magnitude is 1^T w, and the cutoff t_+ is the least t with w >= 0.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from dataclasses import dataclass, fields

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmagnitude.so")

# enum mag_status
MAG_OK, MAG_EINVAL, MAG_EDUPLICATE, MAG_ENOTPD, MAG_ENOCONV, MAG_ENOBRACKET, MAG_ENOMEM, MAG_ECUDA, \
    MAG_ETIMEOUT = range(9)
# enum mag_precision
PREC_AUTO, PREC_BF16, PREC_TF32, PREC_TF32X3, PREC_FP32, PREC_FP64, PREC_FP16X3, PREC_FP16 = range(8)
PRECISIONS = {"auto": PREC_AUTO, "bf16": PREC_BF16, "tf32": PREC_TF32, "tf32x3": PREC_TF32X3,
              "fp32": PREC_FP32, "fp64": PREC_FP64, "fp16x3": PREC_FP16X3, "fp16": PREC_FP16}
# #define MAG_NOALLOC_MAX_N, MAG_MAX_DIM
NOALLOC_MAX_N = 262144
MAX_DIM = 2048
# enum mag_residual_mode
RESID_MATRIX_FREE, RESID_STORED, RESID_AUTO = 0, 1, 2


class mag_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("residual_mode", ctypes.c_int32),
                ("ir_tol", ctypes.c_double), ("ir_max_iters", ctypes.c_int32),
                ("gmres_max_iters", ctypes.c_int32), ("allow_fallback", ctypes.c_int32),
                ("panel_tiles", ctypes.c_int32), ("workspace_limit_bytes", ctypes.c_double),
                ("profile", ctypes.c_int32), ("reuse_distances", ctypes.c_int32),
                ("lookahead", ctypes.c_int32), ("lookahead_sms", ctypes.c_int32),
                ("cta_pairs", ctypes.c_int32), ("tplus_method", ctypes.c_int32),
                ("wait_timeout_ns", ctypes.c_int64), ("out_of_core", ctypes.c_int32),
                ("deflate", ctypes.c_int32), ("host_limit_bytes", ctypes.c_double),
                ("gmres_matvec", ctypes.c_int32), ("fp16_gmres", ctypes.c_int32),
                ("batch_shape", ctypes.c_int32), ("sweep_kind", ctypes.c_int32),
                ("exact_distances", ctypes.c_int32), ("reserved4", ctypes.c_int32)]


class mag_info(ctypes.Structure):
    _fields_ = [("precision_used", ctypes.c_int32), ("ir_iters", ctypes.c_int32),
                ("gmres_iters", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("residual_mode", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("z_norm_inf", ctypes.c_double),
                ("w_norm_inf", ctypes.c_double), ("min_w", ctypes.c_double),
                ("gershgorin_lmin", ctypes.c_double), ("min_distance", ctypes.c_double),
                ("below_bracket", ctypes.c_int32), ("probes", ctypes.c_int32),
                ("ms_generate", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("useful_flops", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("residual_evals", ctypes.c_int32),
                ("update_launches", ctypes.c_int32), ("ms_update", ctypes.c_double),
                ("update_flops", ctypes.c_double), ("ms_update_panel", ctypes.c_double),
                ("ms_potrf", ctypes.c_double), ("ms_trsm", ctypes.c_double), ("ms_split", ctypes.c_double),
                ("probe_rho", ctypes.c_double), ("ms_probe", ctypes.c_double), ("t", ctypes.c_double),
                ("slabs", ctypes.c_int32), ("host_slabs", ctypes.c_int32), ("host_bytes", ctypes.c_double),
                ("host_read_bytes", ctypes.c_double), ("ms_host_read", ctypes.c_double),
                ("deflation_c", ctypes.c_double), ("factor_reused", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("ms_update_busy", ctypes.c_double),
                ("batch_threads", ctypes.c_int32), ("batch_ctas_per_sm", ctypes.c_int32),
                ("batch_tensor_cores", ctypes.c_int32), ("residual_evals_ff", ctypes.c_int32),
                ("batch_left_looking", ctypes.c_int32), ("sweeps_used", ctypes.c_int32),
                ("exact_distances", ctypes.c_int32), ("reserved6", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class mag_batch_desc(ctypes.Structure):
    _fields_ = [("point_offset", ctypes.c_int64), ("w_offset", ctypes.c_int64),
                ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("t", ctypes.c_double)]


_P = ctypes.c_void_p
_I64, _I32, _D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
# name -> (restype, argtypes); the exported symbols of include/magnitude.h
SIGNATURES = {
    "mag_options_default": (ctypes.c_int, [ctypes.POINTER(mag_options)]),
    "mag_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.POINTER(mag_options)]),
    "mag_ctx_set_options": (ctypes.c_int, [_P, ctypes.POINTER(mag_options)]),
    "mag_ctx_destroy": (ctypes.c_int, [_P]),
    "mag_last_error": (ctypes.c_char_p, [_P]),
    "mag_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mag_workspace_bytes": (ctypes.c_int, [_P, _I64, _I32, _DP]),
    "mag_min_distance": (ctypes.c_int, [_P, _P, _I64, _I32, _DP, _DP]),
    "mag_similarity_matrix": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _I32, _P]),
    "mag_cholesky_factor": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _I32, _P]),
    "mag_solve": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _P, _DP, ctypes.POINTER(mag_info)]),
    "mag_solve_multi": (ctypes.c_int, [_P, _P, _I64, _I32, _DP, _I32, _P, _DP, ctypes.POINTER(mag_info)]),
    "mag_solve_rhs": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _P, _P, ctypes.POINTER(mag_info)]),
    "mag_residual": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _P, _P, _P, _DP]),
    "mag_residual_noalloc": (ctypes.c_int, [_P, _I64, _I32, _D, _P, _P, _P, _DP, _P]),
    "mag_sweep_tplus": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _D, _D, _DP, _DP, _P, _DP,
                                       ctypes.POINTER(mag_info)]),
    "mag_grad": (ctypes.c_int, [_P, _P, _I64, _I32, _D, _P, _P, _DP, _P, ctypes.POINTER(mag_info)]),
    "mag_scale_zero": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _DP, ctypes.POINTER(mag_info)]),
    "mag_solve_batch": (ctypes.c_int, [_P, ctypes.POINTER(mag_batch_desc), _I32, _P, _P, _P, _P,
                                       ctypes.POINTER(mag_info)]),
}

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load the shared library (it must have been built, see build.py)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"magnitude CUDA library not built: {p} is missing "
                                   "(run paper_2607_23354_gb300/build.py)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class MagnitudeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


def status_string(status: int) -> str:
    return load_library().mag_status_string(status).decode()


@dataclass
class Options:
    """Solver options (see struct mag_options)."""
    precision: str = "auto"
    residual_mode: str = "auto"
    ir_tol: float = 1e-14
    ir_max_iters: int = 12
    gmres_max_iters: int = 30
    allow_fallback: bool = True
    panel_tiles: int = 0
    workspace_limit_bytes: float = 0.0
    profile: bool = False
    reuse_distances: bool = True
    lookahead: bool = True
    lookahead_sms: int = 0
    cta_pairs: int = 1
    tplus_method: str = "bisection"
    wait_timeout_ns: int = 10_000_000_000
    out_of_core: int = 0
    deflate: int = 0
    host_limit_bytes: float = 0.0
    gmres_matvec: str = "float_float"  # or "fp64"
    fp16_gmres: int = 0
    batch_shape: int = 0  # 0 tuned, 1..7 fixed
    sweeps: str = "chain"  # "chain", "chain_fp32" (FP32 tiles always), "progress"
    exact_distances: bool = True

    def to_c(self) -> mag_options:
        o = mag_options()
        load_library().mag_options_default(ctypes.byref(o))
        o.precision = PRECISIONS[self.precision]
        o.residual_mode = {"matrix_free": RESID_MATRIX_FREE, "stored": RESID_STORED,
                           "auto": RESID_AUTO}[self.residual_mode]
        o.ir_tol = self.ir_tol
        o.ir_max_iters = self.ir_max_iters
        o.gmres_max_iters = self.gmres_max_iters
        o.allow_fallback = int(self.allow_fallback)
        o.panel_tiles = self.panel_tiles
        o.workspace_limit_bytes = self.workspace_limit_bytes
        o.profile = int(self.profile)
        o.reuse_distances = int(self.reuse_distances)
        o.lookahead = int(self.lookahead)
        o.lookahead_sms = int(self.lookahead_sms)
        o.cta_pairs = int(self.cta_pairs)
        o.tplus_method = {"bisection": 0, "ridders": 1}[self.tplus_method]
        o.wait_timeout_ns = int(self.wait_timeout_ns)
        o.out_of_core = int(self.out_of_core)
        o.deflate = int(self.deflate)
        o.host_limit_bytes = float(self.host_limit_bytes)
        if self.gmres_matvec not in ("float_float", "fp64"):
            raise ValueError(f"gmres_matvec must be 'float_float' or 'fp64', not {self.gmres_matvec!r}")
        o.gmres_matvec = 0 if self.gmres_matvec == "float_float" else 1
        o.fp16_gmres = int(self.fp16_gmres)
        o.batch_shape = int(self.batch_shape)
        kinds = {"chain": 0, "chain_fp32": 1, "progress": 2}
        if self.sweeps not in kinds:
            raise ValueError(f"sweeps must be one of {sorted(kinds)}, not {self.sweeps!r}")
        o.sweep_kind = kinds[self.sweeps]
        o.exact_distances = int(self.exact_distances)
        return o


class Context:
    """A mag_ctx bound to a CUDA device and stream (owns the solver workspace)."""

    def __init__(self, options: Options | None = None, stream: torch.cuda.Stream | None = None,
                 device=None):
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("magnitude: no CUDA device (the solver has no CPU path)")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.options = options or Options()
            h = _P()
            st = lib.mag_ctx_create(ctypes.byref(h), _P(self.stream.cuda_stream),
                                    ctypes.byref(self.options.to_c()))
        if st != MAG_OK:
            raise MagnitudeError(st, "mag_ctx_create failed")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mag_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, options: Options):
        self.options = options
        self._check(self._lib.mag_ctx_set_options(self._h, ctypes.byref(options.to_c())))

    def _check(self, st: int, ok=(MAG_OK,)):
        if st not in ok:
            raise MagnitudeError(st, self._lib.mag_last_error(self._h).decode())
        return st

    def _points(self, X: torch.Tensor) -> torch.Tensor:
        if not isinstance(X, torch.Tensor) or X.dim() != 2:
            raise TypeError("points must be a 2-D torch tensor (n x m)")
        if X.device != self.device:
            raise ValueError(f"points on {X.device}, context on {self.device}")
        return X.to(torch.float64).contiguous()

    # ---- entry points (same names as the C ABI) ----
    def workspace_bytes(self, n: int, m: int) -> float:
        b = ctypes.c_double(0.0)
        self._check(self._lib.mag_workspace_bytes(self._h, n, m, ctypes.byref(b)))
        return b.value

    def min_distance(self, X: torch.Tensor):
        X = self._points(X)
        dmin, tb = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._check(self._lib.mag_min_distance(self._h, _P(X.data_ptr()), X.shape[0], X.shape[1],
                                               ctypes.byref(dmin), ctypes.byref(tb)))
        return dmin.value, tb.value

    def similarity_matrix(self, X: torch.Tensor, t: float, precision: str = "fp64"):
        X = self._points(X)
        n, m = X.shape
        p = PRECISIONS[precision]
        Z = torch.empty(n, n, dtype=torch.float64 if p == PREC_FP64 else torch.float32, device=self.device)
        self._check(self._lib.mag_similarity_matrix(self._h, _P(X.data_ptr()), n, m, float(t), p,
                                                    _P(Z.data_ptr())))
        return Z

    def cholesky_factor(self, X: torch.Tensor, t: float, precision: str = "fp64"):
        X = self._points(X)
        n, m = X.shape
        p = PRECISIONS[precision]
        L = torch.empty(n, n, dtype=torch.float64 if p == PREC_FP64 else torch.float32, device=self.device)
        self._check(self._lib.mag_cholesky_factor(self._h, _P(X.data_ptr()), n, m, float(t), p,
                                                  _P(L.data_ptr())))
        return L

    def solve(self, X: torch.Tensor, t: float, w: torch.Tensor | None = None, allow_noconv=False):
        X = self._points(X)
        n, m = X.shape
        if w is None:
            w = torch.empty(n, dtype=torch.float64, device=self.device)
        mag = ctypes.c_double(0.0)
        info = mag_info()
        ok = (MAG_OK, MAG_ENOCONV) if allow_noconv else (MAG_OK,)
        st = self._check(self._lib.mag_solve(self._h, _P(X.data_ptr()), n, m, float(t), _P(w.data_ptr()),
                                             ctypes.byref(mag), ctypes.byref(info)), ok)
        d = info.as_dict()
        d["status"] = st
        return w, mag.value, d

    def solve_multi(self, X: torch.Tensor, ts, W: torch.Tensor | None = None):
        """Weightings for several t on the same points (distances computed once).
        A t of "bound" (or <= 0) is the Sec. 1 bound log(n-1)/min d, found by
        the call itself; infos[i]["t"] is the t solved.  Returns
        (W [len(ts), n], mags list, infos list)."""
        ts = [0.0 if (isinstance(t, str) and t == "bound") else t for t in ts]
        X = self._points(X)
        n, m = X.shape
        nt = len(ts)
        if W is None:
            W = torch.empty(nt, n, dtype=torch.float64, device=self.device)
        tt = (ctypes.c_double * nt)(*[float(t) for t in ts])
        mg = (ctypes.c_double * nt)()
        infos = (mag_info * nt)()
        self._check(self._lib.mag_solve_multi(self._h, _P(X.data_ptr()), n, m, ctypes.cast(tt, _DP), nt,
                                              _P(W.data_ptr()), ctypes.cast(mg, _DP), infos))
        return W, list(mg), [i.as_dict() for i in infos]

    def solve_rhs(self, X: torch.Tensor, t: float, b: torch.Tensor):
        X = self._points(X)
        n, m = X.shape
        b = b.to(device=self.device, dtype=torch.float64).contiguous()
        x = torch.empty(n, dtype=torch.float64, device=self.device)
        info = mag_info()
        self._check(self._lib.mag_solve_rhs(self._h, _P(X.data_ptr()), n, m, float(t), _P(b.data_ptr()),
                                            _P(x.data_ptr()), ctypes.byref(info)))
        return x, info.as_dict()

    def residual(self, X: torch.Tensor, t: float, w: torch.Tensor, b: torch.Tensor | None = None,
                 want_r: bool = True):
        """r = b - Z w in FP64 (Z regenerated); returns (r or None, norms dict)."""
        X = self._points(X)
        n, m = X.shape
        w = w.to(device=self.device, dtype=torch.float64).contiguous()
        bb = None if b is None else b.to(device=self.device, dtype=torch.float64).contiguous()
        r = torch.empty(n, dtype=torch.float64, device=self.device) if want_r else None
        nr = (ctypes.c_double * 4)()
        self._check(self._lib.mag_residual(self._h, _P(X.data_ptr()), n, m, float(t), _P(w.data_ptr()),
                                           _P(0) if bb is None else _P(bb.data_ptr()),
                                           _P(0) if r is None else _P(r.data_ptr()), ctypes.cast(nr, _DP)))
        return r, {"rel_residual": nr[0], "r_norm_inf": nr[1], "z_norm_inf": nr[2], "w_norm_inf": nr[3]}

    def sweep_tplus(self, X: torch.Tensor, t_lo: float = 1e-3, t_hi: float = 0.0, rel_tol: float = 1e-6,
                    method: str | None = None):
        """Sec. 2 cutoff t_+ (feasible end of a bracket at most rel_tol wide).
        method: "bisection" or "ridders" (default: the context's options)."""
        X = self._points(X)
        n, m = X.shape
        w = torch.empty(n, dtype=torch.float64, device=self.device)
        tp, mag = ctypes.c_double(0.0), ctypes.c_double(0.0)
        br = (ctypes.c_double * 2)()
        info = mag_info()
        saved = self.options
        if method is not None and method != saved.tplus_method:
            self.set_options(dataclasses.replace(saved, tplus_method=method))
        try:
            self._check(self._lib.mag_sweep_tplus(self._h, _P(X.data_ptr()), n, m, float(t_lo), float(t_hi),
                                                  float(rel_tol), ctypes.byref(tp),
                                                  ctypes.cast(br, _DP), _P(w.data_ptr()),
                                                  ctypes.byref(mag), ctypes.byref(info)))
        finally:
            if self.options is not saved:
                self.set_options(saved)
        d = info.as_dict()
        return {"t_plus": tp.value, "bracket": (br[0], br[1]), "w": w, "mag": mag.value,
                "below": bool(d["below_bracket"]), "probes": d["probes"], "info": d}

    def scale_zero(self, X: torch.Tensor):
        """App. C, Eq. scaleZero: w0 = d^{-1} 1 / 1^T d^{-1} 1.  Returns
        (w0 [n], s = 1^T d^{-1} 1, info)."""
        X = self._points(X)
        n, m = X.shape
        w0 = torch.empty(n, dtype=torch.float64, device=self.device)
        sv = ctypes.c_double(0.0)
        info = mag_info()
        st = self._check(self._lib.mag_scale_zero(self._h, _P(X.data_ptr()), n, m, _P(w0.data_ptr()),
                                                  ctypes.byref(sv), ctypes.byref(info)))
        d = info.as_dict()
        d["status"] = st
        return w0, sv.value, d

    def grad(self, X: torch.Tensor, t: float, w: torch.Tensor | None = None,
             dL_dw: torch.Tensor | None = None):
        X = self._points(X)
        n, m = X.shape
        dx = torch.empty(n, m, dtype=torch.float64, device=self.device)
        dt = ctypes.c_double(0.0)
        info = mag_info()
        wp = _P(0) if w is None else _P(w.to(torch.float64).contiguous().data_ptr())
        if dL_dw is not None:
            dL_dw = dL_dw.to(device=self.device, dtype=torch.float64).contiguous()
        gp = _P(0) if dL_dw is None else _P(dL_dw.data_ptr())
        keep = (w, dL_dw)  # noqa: F841  (keep converted tensors alive during the call)
        self._check(self._lib.mag_grad(self._h, _P(X.data_ptr()), n, m, float(t), wp, gp, ctypes.byref(dt),
                                       _P(dx.data_ptr()), ctypes.byref(info)))
        return dt.value, dx

    def solve_batch(self, clouds, ts):
        """Solve every cloud at every t.  clouds: list of (n_i x m) tensors on
        this device; ts: list of t values.  Returns (list of w per (cloud, t),
        mags tensor [len(clouds), len(ts)], statuses)."""
        flat = [c.to(torch.float64).contiguous() for c in clouds]
        offs, descs, w_off = [], [], 0
        p_off = 0
        for c in flat:
            offs.append(p_off)
            p_off += c.numel()
        P = torch.cat([c.reshape(-1) for c in flat]) if flat else torch.empty(0, dtype=torch.float64,
                                                                            device=self.device)
        for i, c in enumerate(flat):
            for t in ts:
                descs.append(mag_batch_desc(offs[i], w_off, c.shape[0], c.shape[1], float(t)))
                w_off += c.shape[0]
        D = (mag_batch_desc * len(descs))(*descs)
        W = torch.empty(w_off, dtype=torch.float64, device=self.device)
        M = torch.empty(len(descs), dtype=torch.float64, device=self.device)
        S = torch.empty(len(descs), dtype=torch.int32, device=self.device)
        info = mag_info()
        S.fill_(-1)
        st = self._lib.mag_solve_batch(self._h, D, len(descs), _P(P.data_ptr()), _P(W.data_ptr()),
                                       _P(M.data_ptr()), _P(S.data_ptr()), ctypes.byref(info))
        self.last_batch_info = info.as_dict()
        # per-problem failures are reported in S; raise only for a call-level error
        if st != MAG_OK and not bool((S == st).any()):
            self._check(st)
        ws = []
        for d in descs:
            ws.append(W[d.w_offset:d.w_offset + d.n])
        return ws, M.reshape(len(flat), len(ts)), S.reshape(len(flat), len(ts))


def residual_noalloc(X: torch.Tensor, t: float, w: torch.Tensor, b: torch.Tensor | None = None,
                     stream: torch.cuda.Stream | None = None):
    """mag_residual_noalloc: r = b - Z w with no device allocation inside the
    library (static scratch; n <= NOALLOC_MAX_N).  Returns (r, norms dict);
    r is allocated here by PyTorch, not by the library."""
    lib = load_library()
    if not isinstance(X, torch.Tensor) or X.dim() != 2 or not X.is_cuda:
        raise TypeError("points must be a 2-D CUDA tensor (n x m)")
    n, m = X.shape
    for name, v in (("w", w), ("b", b)):
        if v is not None and (not isinstance(v, torch.Tensor) or v.numel() != n):
            raise ValueError(f"{name} must be a tensor of n = {n} entries")
    # the library picks its static scratch on the current device: make it X's
    with torch.cuda.device(X.device):
        X = X.to(torch.float64).contiguous()
        w = w.to(device=X.device, dtype=torch.float64).contiguous().reshape(n)
        bb = None if b is None else b.to(device=X.device, dtype=torch.float64).contiguous().reshape(n)
        r = torch.empty(n, dtype=torch.float64, device=X.device)
        nr = (ctypes.c_double * 4)()
        s = stream if stream is not None else torch.cuda.current_stream(X.device)
        if s.device != X.device:
            raise ValueError(f"stream on {s.device}, points on {X.device}")
        st = lib.mag_residual_noalloc(_P(X.data_ptr()), n, m, float(t), _P(w.data_ptr()),
                                      _P(0) if bb is None else _P(bb.data_ptr()), _P(r.data_ptr()),
                                      ctypes.cast(nr, _DP), _P(s.cuda_stream))
    if st != MAG_OK:
        raise MagnitudeError(st, "mag_residual_noalloc failed" +
                             (f" (n = {n} > {NOALLOC_MAX_N})" if st == MAG_ENOMEM else ""))
    return r, {"rel_residual": nr[0], "r_norm_inf": nr[1], "z_norm_inf": nr[2], "w_norm_inf": nr[3]}


_ctx_cache: dict = {}


def default_context(options: Options | None = None) -> Context:
    """A cached context for the current device and stream."""
    dev = torch.cuda.current_device()
    key = (dev, torch.cuda.current_stream().cuda_stream)
    ctx = _ctx_cache.get(key)
    if ctx is None:
        ctx = Context(options)
        _ctx_cache[key] = ctx
    elif options is not None and options != ctx.options:
        ctx.set_options(options)
    return ctx


def solve(X, t, options: Options | None = None):
    """w, Mag for Z = exp[-t d] (Sec. 2).  X: (n, m) CUDA tensor."""
    w, mag, _ = default_context(options).solve(X, t)
    return w, mag


def sweep_tplus(X, t_lo=1e-3, t_hi=0.0, rel_tol=1e-6, options: Options | None = None,
                method: str | None = None):
    return default_context(options).sweep_tplus(X, t_lo, t_hi, rel_tol, method=method)


def scale_zero(X, options: Options | None = None):
    return default_context(options).scale_zero(X)


class MagnitudeFn(torch.autograd.Function):
    """(X, t) -> (w, Mag) with the adjoint gradients of mag_grad.

    Backward: for upstream grads gw (of w) and gM (of Mag), the loss gradient
    with respect to w is g = gw + gM 1, handed to mag_grad as is; the library
    solves lambda = Z^{-1} g with the same solver (lambda = gM w without a
    solve when g is constant) and forms dL/dt and dL/dX in one fused pass."""

    @staticmethod
    def forward(ctx, X, t):
        tt = float(t)
        w, mag, _ = default_context().solve(X.detach(), tt)
        ctx.save_for_backward(X, w)
        ctx.t = tt
        return w, torch.tensor(mag, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, gw, gM):
        X, w = ctx.saved_tensors
        c = default_context()
        g = torch.zeros_like(w) if gw is None else gw.to(torch.float64).reshape(w.shape)
        if gM is not None:
            g = g + gM.to(torch.float64)
        dt, dx = c.grad(X.detach(), ctx.t, w=w, dL_dw=g.contiguous())
        dX = dx.to(X.dtype)
        dT = torch.tensor(dt, dtype=torch.float64, device=X.device)
        return dX, dT


def magnitude(X, t):
    """Differentiable (w, Mag) through MagnitudeFn."""
    if not isinstance(t, torch.Tensor):
        t = torch.tensor(float(t), dtype=torch.float64)
    return MagnitudeFn.apply(X, t)
