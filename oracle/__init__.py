"""FP64 CPU oracle for batched restarted reflected-Halpern PDHG (ctypes wrapper).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this package.  The CUDA library and its
Python binding never import it, and it never imports them.

The arithmetic lives in ``pdhg_oracle.c`` (plain C, FP64, one vector per LP,
no blocking); this file only compiles it with gcc and marshals numpy arrays.
Each wrapped function names the paper passage its C counterpart follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdhg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OPTIMAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, ITERATION_LIMIT, NUMERICAL = range(5)
STATUS_NAMES = ["OPTIMAL", "PRIMAL_INFEASIBLE", "DUAL_INFEASIBLE", "ITERATION_LIMIT", "NUMERICAL"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm hosts
    round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p),
                ("c", C.c_void_p), ("row_lo", C.c_void_p), ("row_hi", C.c_void_p),
                ("var_lo", C.c_void_p), ("var_hi", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("check_every", C.c_int32), ("ruiz_iters", C.c_int32), ("pock_chambolle", C.c_int32),
                ("lockstep", C.c_int32), ("beta_s", C.c_double), ("beta_n", C.c_double),
                ("beta_a", C.c_double), ("theta", C.c_double), ("mnorm_sign", C.c_double),
                ("restart_to_pdhg_output", C.c_int32), ("power_max_iter", C.c_int32),
                ("power_tol", C.c_double), ("power_seed", C.c_uint64), ("eps_infeas", C.c_double),
                ("threads", C.c_int32), ("detect_infeasibility", C.c_int32), ("mutation", C.c_int32),
                ("reduced_cost", C.c_int32)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iters", C.c_int64),
                ("obj", C.c_double), ("dual_obj", C.c_double), ("rel_primal", C.c_double),
                ("rel_dual", C.c_double), ("rel_gap", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        _lib.orc_default_options.argtypes = [C.POINTER(Options)]
        _lib.orc_norm2_estimate.restype = d
        _lib.orc_norm2_estimate.argtypes = [i32, i32, vp, vp, vp, i32, d, C.c_uint64, C.POINTER(i32)]
        _lib.orc_scaling.argtypes = [C.POINTER(_Problem), i32, i32, vp, vp]
        _lib.orc_kkt.argtypes = [C.POINTER(_Problem), i32, i32, d, d, d, vp, vp, vp]
        _lib.orc_kkt_rc.argtypes = [C.POINTER(_Problem), i32, i32, d, d, d, vp, vp, i32, vp]
        _lib.orc_robust_reduced_cost.argtypes = [i32, vp, vp, vp, vp, vp]
        _lib.orc_solve.restype = i32
        _lib.orc_solve.argtypes = [C.POINTER(_Problem), i32, vp, vp, vp, vp, vp, d, i64,
                                   C.POINTER(Options), vp, vp, vp, vp, C.POINTER(_Result), C.POINTER(d)]
        _lib.orc_prepare.restype = vp
        _lib.orc_prepare.argtypes = [C.POINTER(_Problem), C.POINTER(Options)]
        _lib.orc_prepared_eta.restype = d
        _lib.orc_prepared_eta.argtypes = [vp]
        _lib.orc_prepared_free.argtypes = [vp]
        _lib.orc_solve_prepared.restype = i32
        _lib.orc_solve_prepared.argtypes = [vp, i32, vp, vp, vp, vp, vp, d, i64, C.POINTER(Options), vp, vp, vp,
                                            vp, C.POINTER(_Result)]
        for f in ("orc_project_box", "orc_project_barrier", "orc_project_recession"):
            getattr(_lib, f).argtypes = [i32, vp, vp, vp, vp]
        _lib.orc_support.restype = d
        _lib.orc_support.argtypes = [i32, vp, vp, vp]
        _lib.orc_apply_T.argtypes = [C.POINTER(_Problem), vp, vp, vp, vp, vp, d, d, vp, vp, vp, vp]
        _lib.orc_mnorm2.restype = d
        _lib.orc_mnorm2.argtypes = [C.POINTER(_Problem), d, d, d, vp, vp]
        _lib.orc_set_mutation.argtypes = [i32]
        _lib.orc_splitmix64_at.restype = C.c_uint64
        _lib.orc_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    lib().orc_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


class _Held:
    """Keeps the contiguous arrays alive while C holds pointers to them."""

    def __init__(self, lp):
        self.row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
        self.vals = _f64(lp.vals)
        self.c, self.row_lo, self.row_hi = _f64(lp.c), _f64(lp.row_lo), _f64(lp.row_hi)
        self.var_lo, self.var_hi = _f64(lp.var_lo), _f64(lp.var_hi)
        self.p = _Problem(lp.m, lp.n, int(self.row_ptr[-1]), _ptr(self.row_ptr), _ptr(self.col_idx),
                          _ptr(self.vals), _ptr(self.c), _ptr(self.row_lo), _ptr(self.row_hi),
                          _ptr(self.var_lo), _ptr(self.var_hi))


@dataclass
class SolveResult:
    status: np.ndarray
    obj: np.ndarray
    dual_obj: np.ndarray
    rel_primal: np.ndarray
    rel_dual: np.ndarray
    rel_gap: np.ndarray
    iters: np.ndarray
    restarts: np.ndarray
    x: np.ndarray | None  # (num_lps, n)
    y: np.ndarray | None  # (num_lps, m)
    eta: float


def _spec_arrays(specs, q, lp, warm_x, warm_y, want_xy):
    kind = np.ascontiguousarray(specs.kind, dtype=np.int32)
    var = np.ascontiguousarray(specs.var, dtype=np.int32)
    lo, hi, sg = _f64(specs.lo), _f64(specs.hi), _f64(specs.sign)
    wx = None if warm_x is None else _f64(np.asarray(warm_x).reshape(q, lp.n))
    wy = None if warm_y is None else _f64(np.asarray(warm_y).reshape(q, lp.m))
    x = np.zeros((q, lp.n)) if want_xy else None
    y = np.zeros((q, lp.m)) if want_xy else None
    return kind, var, lo, hi, sg, wx, wy, x, y


def _result(res, q, x, y, eta):
    g = lambda f, dt: np.array([getattr(res[i], f) for i in range(q)], dtype=dt)
    return SolveResult(g("status", np.int32), g("obj", float), g("dual_obj", float),
                       g("rel_primal", float), g("rel_dual", float), g("rel_gap", float),
                       g("iters", np.int64), g("restarts", np.int32), x, y, eta)


def solve(lp, specs, tol: float = 1e-4, max_iter: int = 100000, options: Options | None = None,
          warm_x=None, warm_y=None, want_xy: bool = True, **kw) -> SolveResult:
    """Batched restarted reflected-Halpern PDHG (Sec. 4-5) on the CPU in FP64."""
    o = options if options is not None else default_options(**kw)
    h = _Held(lp)
    q = len(specs)
    kind, var, lo, hi, sg, wx, wy, x, y = _spec_arrays(specs, q, lp, warm_x, warm_y, want_xy)
    res = (_Result * max(q, 1))()
    eta = C.c_double(0.0)
    rc = lib().orc_solve(C.byref(h.p), q, _ptr(kind), _ptr(var), _ptr(lo), _ptr(hi), _ptr(sg), tol,
                         int(max_iter), C.byref(o), _ptr(wx), _ptr(wy), _ptr(x), _ptr(y), res,
                         C.byref(eta))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return _result(res, q, x, y, eta.value)


class Prepared:
    """The per-matrix set-up of ``solve`` (scaling, scaled values, eta, ||b~||)
    done once, for several solves on the same matrix.  ``solve`` on a
    Prepared gives the same results as the module-level ``solve`` with the
    same options; the set-up options are those given here."""

    def __init__(self, lp, options: Options | None = None, **kw):
        self.lp = lp
        self.options = options if options is not None else default_options(**kw)
        self._held = _Held(lp)
        self._h = lib().orc_prepare(C.byref(self._held.p), C.byref(self.options))
        if not self._h:
            raise ValueError("oracle set-up failed")
        self.eta = lib().orc_prepared_eta(self._h)

    def solve(self, specs, tol: float = 1e-4, max_iter: int = 100000, warm_x=None, warm_y=None,
              want_xy: bool = True, **kw) -> SolveResult:
        o = Options.from_buffer_copy(self.options)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise AttributeError(k)
            setattr(o, k, v)
        q = len(specs)
        kind, var, lo, hi, sg, wx, wy, x, y = _spec_arrays(specs, q, self.lp, warm_x, warm_y, want_xy)
        res = (_Result * max(q, 1))()
        rc = lib().orc_solve_prepared(self._h, q, _ptr(kind), _ptr(var), _ptr(lo), _ptr(hi), _ptr(sg), tol,
                                      int(max_iter), C.byref(o), _ptr(wx), _ptr(wy), _ptr(x), _ptr(y), res)
        if rc != 0:
            raise ValueError(f"oracle rejected the arguments (code {rc})")
        return _result(res, q, x, y, self.eta)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_prepared_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kkt(lp, kind: int, var: int, lo: float, hi: float, sign: float, x, y, reduced_cost: int = 0) -> dict:
    """Relative KKT of (x, y) for one LP in the original space (Eq. stopping);
    ``reduced_cost`` 1 takes the reduced cost robust to large bounds."""
    h = _Held(lp)
    x, y = _f64(x), _f64(y)
    out = np.zeros(5)
    lib().orc_kkt_rc(C.byref(h.p), int(kind), int(var), float(lo), float(hi), float(sign),
                     _ptr(x), _ptr(y), int(reduced_cost), _ptr(out))
    return dict(obj=out[0], dual_obj=out[1], rel_primal=out[2], rel_dual=out[3], rel_gap=out[4])


def kkt_spec(lp, specs, q: int, x, y, reduced_cost: int = 0) -> dict:
    return kkt(lp, specs.kind[q], specs.var[q], specs.lo[q], specs.hi[q], specs.sign[q], x, y, reduced_cost)


def norm2_estimate(lp, max_iter: int = 5000, tol: float = 1e-10, seed: int = 0x5EED):
    """Power-iteration estimate of ||A||_2 (reading of Sec. 4 "Step-size")."""
    h = _Held(lp)
    it = C.c_int32(0)
    v = lib().orc_norm2_estimate(lp.m, lp.n, _ptr(h.row_ptr), _ptr(h.col_idx), _ptr(h.vals),
                                 max_iter, tol, seed, C.byref(it))
    return v, it.value


def scaling(lp, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """Ruiz + Pock-Chambolle factors (D_r, D_c) with A~ = D_r A D_c."""
    h = _Held(lp)
    dr, dc = np.zeros(max(lp.m, 1)), np.zeros(max(lp.n, 1))
    lib().orc_scaling(C.byref(h.p), ruiz_iters, int(pock_chambolle), _ptr(dr), _ptr(dc))
    return dr[:lp.m], dc[:lp.n]


def _elementwise(name, v, a, b):
    v, a, b = _f64(v), _f64(a), _f64(b)
    out = np.zeros_like(v)
    getattr(lib(), name)(v.shape[0], _ptr(v), _ptr(a), _ptr(b), _ptr(out))
    return out


def project_box(v, a, b):
    return _elementwise("orc_project_box", v, a, b)


def project_barrier(v, a, b):
    return _elementwise("orc_project_barrier", v, a, b)


def project_recession(v, a, b):
    return _elementwise("orc_project_recession", v, a, b)


def robust_reduced_cost(v, x, a, b):
    """Elementwise reduced cost robust to large finite bounds (Sec. 4
    "Stopping criteria", PDLP's Appendix A variant) of components v at x."""
    v, x, a, b = _f64(v), _f64(x), _f64(a), _f64(b)
    out = np.zeros_like(v)
    lib().orc_robust_reduced_cost(v.shape[0], _ptr(v), _ptr(x), _ptr(a), _ptr(b), _ptr(out))
    return out


def support(v, a, b) -> float:
    v, a, b = _f64(v), _f64(a), _f64(b)
    return lib().orc_support(v.shape[0], _ptr(v), _ptr(a), _ptr(b))


def apply_T(lp, c, xl, xu, l, u, tau: float, sigma: float, x, y):
    """The PDHG operator T of Sec. 4 on the data of ``lp`` (A only) with the
    given objective and bounds; returns (x^, y^)."""
    h = _Held(lp)
    args = [_f64(v) for v in (c, xl, xu, l, u)]
    x, y = _f64(x), _f64(y)
    xh, yh = np.zeros(lp.n), np.zeros(lp.m)
    lib().orc_apply_T(C.byref(h.p), *[_ptr(a) for a in args], float(tau), float(sigma), _ptr(x), _ptr(y),
                      _ptr(xh), _ptr(yh))
    return xh, yh


def mnorm2(lp, w: float, eta: float, sign: float, dx, dy) -> float:
    """Squared M-norm of (dx, dy) (Eq. residual) with cross-term sign ``sign``."""
    h = _Held(lp)
    dx, dy = _f64(dx), _f64(dy)
    return lib().orc_mnorm2(C.byref(h.p), float(w), float(eta), float(sign), _ptr(dx), _ptr(dy))


def set_mutation(k: int) -> None:
    """Plant mistake ``k`` (0 = none) for direct calls; test use only."""
    lib().orc_set_mutation(int(k))


def splitmix64_at(seed: int, index: int) -> int:
    return int(lib().orc_splitmix64_at(seed, index))
