"""ctypes binding of liblpb.so (include/lpb.h): argument marshalling only.

Every function named ``lpb_*`` here is the C entry point of the same name;
the compute runs in the library's CUDA kernels.  There is no CPU fallback:
importing this module without a built library, or calling it without a CUDA
device, raises.

``Handle`` / ``Batch`` are small conveniences over those calls for numpy
inputs (CSR arrays, bound vectors, override records) and torch device
tensors (the ``*_dev`` variant).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpb.so")

LPB_OK, LPB_ERR_INVALID_ARG, LPB_ERR_OOM, LPB_ERR_CUDA, LPB_ERR_TIMEOUT, LPB_ERR_DEVICE_CHECK, LPB_ERR_BAD_INDEX = range(7)
ERR_NAMES = ["LPB_OK", "LPB_ERR_INVALID_ARG", "LPB_ERR_OOM", "LPB_ERR_CUDA", "LPB_ERR_TIMEOUT",
             "LPB_ERR_DEVICE_CHECK", "LPB_ERR_BAD_INDEX"]
OPTIMAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, ITERATION_LIMIT, NUMERICAL = range(5)
STATUS_NAMES = ["OPTIMAL", "PRIMAL_INFEASIBLE", "DUAL_INFEASIBLE", "ITERATION_LIMIT", "NUMERICAL"]
FP64, MIXED = 0, 1
POLISH_DFLOAT, POLISH_FP64 = 0, 1
RC_BARRIER, RC_ROBUST = 0, 1
LPB_MAX_JOINT = 64  # most handles in one lpb_solve_multi call

# every symbol include/lpb.h declares
EXPORTS = ["lpb_default_options", "lpb_create", "lpb_solve", "lpb_solve_dev", "lpb_result", "lpb_results",
           "lpb_result_device", "lpb_batch_profile", "lpb_handle_info", "lpb_scaling", "lpb_batch_free",
           "lpb_destroy", "lpb_last_error", "lpb_scaling_noalloc", "lpb_obbt_tighten", "lpb_get_tuning",
           "lpb_set_tuning", "lpb_autotune", "lpb_tune_batch", "lpb_solve_multi"]
# every symbol include/lpb_serve.h declares
SERVE_EXPORTS = ["lpb_server_default_options", "lpb_server_create", "lpb_server_attach", "lpb_server_submit",
                 "lpb_server_poll", "lpb_server_wait", "lpb_server_result", "lpb_server_results",
                 "lpb_server_request_info", "lpb_server_release", "lpb_server_stats_get", "lpb_server_destroy"]
REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)


class LpbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES[code] if 0 <= code < len(ERR_NAMES) else code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("check_every", C.c_int32), ("ruiz_iters", C.c_int32),
                ("pock_chambolle", C.c_int32), ("beta_s", C.c_double), ("beta_n", C.c_double),
                ("beta_a", C.c_double), ("theta", C.c_double), ("mnorm_sign", C.c_double),
                ("restart_to_pdhg_output", C.c_int32), ("power_max_iter", C.c_int32),
                ("power_tol", C.c_double), ("power_seed", C.c_uint64), ("eps_infeas", C.c_double),
                ("detect_infeasibility", C.c_int32), ("profile", C.c_int32), ("cuda_stream", C.c_void_p),
                ("device", C.c_int32), ("fp64_polish", C.c_int32), ("polish_stall_checks", C.c_int32),
                ("polish_arith", C.c_int32), ("eps_dual", C.c_double), ("use_graphs", C.c_int32),
                ("use_pdl", C.c_int32), ("stream_priority", C.c_int32), ("reduced_cost", C.c_int32)]


class Spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("var", C.c_int32), ("lo", C.c_double), ("hi", C.c_double),
                ("sign", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iters", C.c_int64), ("obj", C.c_double),
                ("dual_obj", C.c_double), ("rel_primal", C.c_double), ("rel_dual", C.c_double),
                ("rel_gap", C.c_double), ("safe_bound", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 4), ("ms", C.c_double * 4), ("bytes", C.c_double * 4),
                ("setup_ms", C.c_double), ("checks", C.c_int64), ("compactions", C.c_int64),
                ("kernels", C.c_int64), ("fp64_switch_iter", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("long_row_primal", C.c_int32), ("long_row_dual", C.c_int32), ("lane_shift_primal", C.c_int32),
                ("lane_shift_dual", C.c_int32)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("lane_columns", C.c_int32), ("polish_columns", C.c_int32),
                ("max_groups", C.c_int32), ("device", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("matrix_id", C.c_int32), ("num_lps", C.c_int32), ("specs", C.c_void_p), ("tol", C.c_double),
                ("max_iter", C.c_int64), ("warm_x", C.c_void_p), ("warm_y", C.c_void_p),
                ("warm_request", C.c_int64), ("warm_lp", C.c_int32)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("num_lps", C.c_int32), ("optimal", C.c_int32), ("infeasible", C.c_int32),
                ("iteration_limit", C.c_int32), ("other", C.c_int32), ("iters", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("footprint_bytes", C.c_int64), ("polished", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("done", C.c_int64), ("lps_solved", C.c_int64), ("intervals", C.c_int64),
                ("column_iters", C.c_int64), ("admitted_while_busy", C.c_int64), ("migrations", C.c_int64),
                ("busy_s", C.c_double), ("hbm_used_bytes", C.c_int64), ("hbm_budget_bytes", C.c_int64),
                ("kernels", C.c_int64)]


SPEC_DTYPE = np.dtype([("kind", "<i4"), ("var", "<i4"), ("lo", "<f8"), ("hi", "<f8"), ("sign", "<f8")])
assert SPEC_DTYPE.itemsize == C.sizeof(Spec)

_lib = None


def load(path: str = LIB_PATH):
    """Load liblpb.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    lib = C.CDLL(path)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.lpb_default_options.argtypes = [C.POINTER(Options)]
    lib.lpb_default_options.restype = None
    lib.lpb_create.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(Options), C.POINTER(vp)]
    lib.lpb_solve.argtypes = [vp, i32, vp, d, i64, vp, vp, C.POINTER(vp)]
    lib.lpb_solve_dev.argtypes = [vp, i32, vp, d, i64, vp, vp, C.POINTER(vp)]
    lib.lpb_solve_multi.argtypes = [i32, vp, vp, vp, d, i64, vp]
    lib.lpb_result.argtypes = [vp, i32, C.POINTER(Result), vp, vp]
    lib.lpb_results.argtypes = [vp, vp]
    lib.lpb_result_device.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
    lib.lpb_batch_profile.argtypes = [vp, C.POINTER(Profile)]
    lib.lpb_handle_info.argtypes = [vp, C.POINTER(d), C.POINTER(d), C.POINTER(i32)]
    lib.lpb_scaling.argtypes = [vp, vp, vp]
    lib.lpb_batch_free.argtypes = [vp]
    lib.lpb_batch_free.restype = None
    lib.lpb_destroy.argtypes = [vp]
    lib.lpb_destroy.restype = None
    lib.lpb_last_error.restype = C.c_char_p
    lib.lpb_scaling_noalloc.argtypes = [i32, i32, i32, vp, vp, vp, i32, i32, vp, vp, vp]
    lib.lpb_obbt_tighten.argtypes = [vp, vp, vp, vp, d, vp, vp, C.POINTER(i32)]
    lib.lpb_obbt_tighten.restype = C.c_int
    lib.lpb_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    lib.lpb_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    lib.lpb_autotune.argtypes = [vp, i32, C.POINTER(Tuning)]
    lib.lpb_tune_batch.argtypes = [vp, vp, i32, vp, C.POINTER(i32)]
    for f in ("lpb_get_tuning", "lpb_set_tuning", "lpb_autotune", "lpb_tune_batch"):
        getattr(lib, f).restype = C.c_int
    lib.lpb_server_default_options.argtypes = [C.POINTER(ServerOptions)]
    lib.lpb_server_default_options.restype = None
    lib.lpb_server_create.argtypes = [C.POINTER(ServerOptions), C.POINTER(vp)]
    lib.lpb_server_attach.argtypes = [vp, vp, C.POINTER(i32)]
    lib.lpb_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(i64)]
    lib.lpb_server_poll.argtypes = [vp, i64, C.POINTER(i32)]
    lib.lpb_server_wait.argtypes = [vp, i64, d]
    lib.lpb_server_result.argtypes = [vp, i64, i32, C.POINTER(Result), vp, vp]
    lib.lpb_server_results.argtypes = [vp, i64, vp]
    lib.lpb_server_request_info.argtypes = [vp, i64, C.POINTER(RequestInfo)]
    lib.lpb_server_release.argtypes = [vp, i64]
    lib.lpb_server_stats_get.argtypes = [vp, C.POINTER(ServerStats)]
    lib.lpb_server_destroy.argtypes = [vp]
    lib.lpb_server_destroy.restype = None
    for f in ("lpb_create", "lpb_solve", "lpb_solve_dev", "lpb_solve_multi", "lpb_result", "lpb_results", "lpb_result_device",
              "lpb_batch_profile", "lpb_handle_info", "lpb_scaling", "lpb_scaling_noalloc", "lpb_server_create",
              "lpb_server_attach", "lpb_server_submit", "lpb_server_poll", "lpb_server_wait", "lpb_server_result",
              "lpb_server_results", "lpb_server_request_info", "lpb_server_release", "lpb_server_stats_get"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != LPB_OK:
        raise LpbError(code, load().lpb_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------

def lpb_default_options(**overrides) -> Options:
    o = Options()
    load().lpb_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def lpb_create(m, n, row_ptr, col_idx, vals, c, row_lo, row_hi, var_lo, var_hi, options: Options | None = None):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    cc, rl, ru, xl, xu = f(c), f(row_lo), f(row_hi), f(var_lo), f(var_hi)
    h = C.c_void_p()
    _check(load().lpb_create(int(m), int(n), int(rp[-1]), _ptr(rp), _ptr(ci) if ci.size else None,
                             _ptr(va) if va.size else None, _ptr(cc), _ptr(rl) if rl.size else None,
                             _ptr(ru) if ru.size else None, _ptr(xl), _ptr(xu),
                             C.byref(options) if options is not None else None, C.byref(h)))
    return h


def lpb_solve(h, specs: np.ndarray, tol: float, max_iter: int, warm_x=None, warm_y=None):
    sp = np.ascontiguousarray(specs, dtype=SPEC_DTYPE)
    wx = None if warm_x is None else np.ascontiguousarray(warm_x, dtype=np.float64)
    wy = None if warm_y is None else np.ascontiguousarray(warm_y, dtype=np.float64)
    b = C.c_void_p()
    _check(load().lpb_solve(h, int(sp.shape[0]), _ptr(sp) if sp.size else None, float(tol), int(max_iter),
                            _ptr(wx), _ptr(wy), C.byref(b)))
    return b


def lpb_solve_dev(h, num_lps: int, specs_dev_ptr: int, tol: float, max_iter: int, warm_x_dev_ptr=None,
                  warm_y_dev_ptr=None):
    b = C.c_void_p()
    _check(load().lpb_solve_dev(h, int(num_lps), specs_dev_ptr, float(tol), int(max_iter), warm_x_dev_ptr,
                                warm_y_dev_ptr, C.byref(b)))
    return b


def lpb_solve_multi(handles, specs, tol: float, max_iter: int):
    """handles: handle pointers; specs: one SPEC_DTYPE array per handle.
    Returns one batch pointer per handle."""
    k = len(handles)
    sps = [np.ascontiguousarray(sp, dtype=SPEC_DTYPE) for sp in specs]
    if len(sps) != k:
        raise ValueError("one spec array per handle")
    hv = (C.c_void_p * k)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    nv = (C.c_int32 * k)(*[int(sp.shape[0]) for sp in sps])
    pv = (C.c_void_p * k)(*[sp.ctypes.data if sp.size else None for sp in sps])
    out = (C.c_void_p * k)()
    _check(load().lpb_solve_multi(k, hv, nv, pv, float(tol), int(max_iter), out))
    return [C.c_void_p(out[i]) for i in range(k)]


def lpb_result(b, lp: int, n: int, m: int, want_xy: bool = True):
    r = Result()
    x = np.zeros(n) if want_xy else None
    y = np.zeros(max(m, 1)) if want_xy else None
    _check(load().lpb_result(b, int(lp), C.byref(r), _ptr(x), _ptr(y)))
    return r, x, (y[:m] if y is not None else None)


def lpb_results(b, num_lps: int) -> np.ndarray:
    out = (Result * max(num_lps, 1))()
    _check(load().lpb_results(b, out))
    arr = np.ctypeslib.as_array(out)[:num_lps]
    return arr.copy()


def lpb_result_device(b):
    x, y = C.c_void_p(), C.c_void_p()
    _check(load().lpb_result_device(b, C.byref(x), C.byref(y)))
    return x.value, y.value


def lpb_batch_profile(b) -> Profile:
    p = Profile()
    _check(load().lpb_batch_profile(b, C.byref(p)))
    return p


def lpb_handle_info(h):
    eta, est, it = C.c_double(), C.c_double(), C.c_int32()
    _check(load().lpb_handle_info(h, C.byref(eta), C.byref(est), C.byref(it)))
    return eta.value, est.value, it.value


def lpb_scaling(h, m: int, n: int):
    dr, dc = np.zeros(max(m, 1)), np.zeros(n)
    _check(load().lpb_scaling(h, _ptr(dr), _ptr(dc)))
    return dr[:m], dc


def lpb_scaling_noalloc(m: int, n: int, nnz: int, row_ptr_dev: int, col_idx_dev: int, vals_dev: int,
                        ruiz_iters: int, pock_chambolle: int, d_row_dev: int, d_col_dev: int, stream=None) -> None:
    """Equilibration factors into caller-owned device buffers, using the
    library's fixed device scratch (no allocation).  Pointers are device
    addresses (e.g. torch ``data_ptr()``); ``stream`` a cudaStream_t or None."""
    _check(load().lpb_scaling_noalloc(int(m), int(n), int(nnz), row_ptr_dev, col_idx_dev, vals_dev,
                                      int(ruiz_iters), int(pock_chambolle), d_row_dev, d_col_dev, stream))


def lpb_obbt_tighten(b, specs: np.ndarray, var_lo, var_hi, min_gain: float = 1e-4):
    """New variable bounds from a solved OBBT batch: (new_lo, new_hi, updated)."""
    sp = np.ascontiguousarray(specs, dtype=SPEC_DTYPE)
    lo = np.ascontiguousarray(var_lo, dtype=np.float64)
    hi = np.ascontiguousarray(var_hi, dtype=np.float64)
    nlo, nhi = np.empty_like(lo), np.empty_like(hi)
    cnt = C.c_int32()
    _check(load().lpb_obbt_tighten(b, _ptr(sp) if sp.size else None, _ptr(lo), _ptr(hi), float(min_gain), _ptr(nlo),
                                   _ptr(nhi), C.byref(cnt)))
    return nlo, nhi, cnt.value


def lpb_get_tuning(h) -> Tuning:
    t = Tuning()
    _check(load().lpb_get_tuning(h, C.byref(t)))
    return t


def lpb_set_tuning(h, t: Tuning) -> None:
    _check(load().lpb_set_tuning(h, C.byref(t)))


def lpb_autotune(h, num_lps: int) -> Tuning:
    t = Tuning()
    _check(load().lpb_autotune(h, int(num_lps), C.byref(t)))
    return t


def lpb_tune_batch(h, widths):
    """(microseconds per iteration for each width, index of the best width)"""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    us = np.zeros(w.size)
    best = C.c_int32()
    _check(load().lpb_tune_batch(h, _ptr(w), int(w.size), _ptr(us), C.byref(best)))
    return us, best.value


def lpb_batch_free(b) -> None:
    load().lpb_batch_free(b)


def lpb_destroy(h) -> None:
    load().lpb_destroy(h)


def lpb_last_error() -> str:
    return load().lpb_last_error().decode()


# include/lpb_serve.h

def lpb_server_default_options(**overrides) -> ServerOptions:
    o = ServerOptions()
    load().lpb_server_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def lpb_server_create(options: ServerOptions | None = None):
    s = C.c_void_p()
    _check(load().lpb_server_create(C.byref(options) if options is not None else None, C.byref(s)))
    return s


def lpb_server_attach(srv, h) -> int:
    mid = C.c_int32()
    _check(load().lpb_server_attach(srv, h, C.byref(mid)))
    return mid.value


def lpb_server_submit(srv, matrix_id: int, specs: np.ndarray, tol: float, max_iter: int, warm_x=None, warm_y=None,
                      warm_request: int = -1, warm_lp: int = 0) -> int:
    sp = np.ascontiguousarray(specs, dtype=SPEC_DTYPE)
    wx = None if warm_x is None else np.ascontiguousarray(warm_x, dtype=np.float64)
    wy = None if warm_y is None else np.ascontiguousarray(warm_y, dtype=np.float64)
    q = Request(int(matrix_id), int(sp.shape[0]), _ptr(sp), float(tol), int(max_iter), _ptr(wx), _ptr(wy),
                int(warm_request), int(warm_lp))
    rid = C.c_int64()
    _check(load().lpb_server_submit(srv, C.byref(q), C.byref(rid)))
    return rid.value


def lpb_server_poll(srv, rid: int) -> bool:
    done = C.c_int32()
    _check(load().lpb_server_poll(srv, int(rid), C.byref(done)))
    return bool(done.value)


def lpb_server_wait(srv, rid: int, timeout_s: float = -1.0) -> None:
    _check(load().lpb_server_wait(srv, int(rid), float(timeout_s)))


def lpb_server_result(srv, rid: int, lp: int, n: int, m: int, want_xy: bool = True):
    r = Result()
    x = np.zeros(n) if want_xy else None
    y = np.zeros(max(m, 1)) if want_xy else None
    _check(load().lpb_server_result(srv, int(rid), int(lp), C.byref(r), _ptr(x), _ptr(y)))
    return r, x, (y[:m] if y is not None else None)


def lpb_server_results(srv, rid: int, num_lps: int) -> np.ndarray:
    out = (Result * max(num_lps, 1))()
    _check(load().lpb_server_results(srv, int(rid), out))
    return np.ctypeslib.as_array(out)[:num_lps].copy()


def lpb_server_request_info(srv, rid: int) -> RequestInfo:
    info = RequestInfo()
    _check(load().lpb_server_request_info(srv, int(rid), C.byref(info)))
    return info


def lpb_server_release(srv, rid: int) -> None:
    _check(load().lpb_server_release(srv, int(rid)))


def lpb_server_stats_get(srv) -> ServerStats:
    st = ServerStats()
    _check(load().lpb_server_stats_get(srv, C.byref(st)))
    return st


def lpb_server_destroy(srv) -> None:
    load().lpb_server_destroy(srv)


# ---------------------------------------------------------------------------
# conveniences
# ---------------------------------------------------------------------------

def specs_array(kind, var, lo=None, hi=None, sign=None) -> np.ndarray:
    kind = np.asarray(kind)
    a = np.zeros(kind.shape[0], dtype=SPEC_DTYPE)
    a["kind"] = kind
    a["var"] = var
    a["lo"] = -np.inf if lo is None else lo
    a["hi"] = np.inf if hi is None else hi
    a["sign"] = 1.0 if sign is None else sign
    return a


def specs_from(s) -> np.ndarray:
    """From any object with kind/var/lo/hi/sign arrays (e.g. lpgen.Specs)."""
    return specs_array(s.kind, s.var, s.lo, s.hi, s.sign)


class Batch:
    def __init__(self, handle: "Handle", ptr):
        self.h = handle
        self.ptr = ptr
        self.n, self.m = handle.n, handle.m

    def results(self) -> np.ndarray:
        return lpb_results(self.ptr, self.num_lps)

    @property
    def num_lps(self) -> int:
        return self._num

    def result(self, lp: int, want_xy: bool = True):
        return lpb_result(self.ptr, lp, self.n, self.m, want_xy)

    def device_xy(self):
        return lpb_result_device(self.ptr)

    def profile(self) -> Profile:
        return lpb_batch_profile(self.ptr)

    def free(self):
        if self.ptr is not None:
            lpb_batch_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Handle:
    """One shared A with base vectors, resident on the GPU."""

    def __init__(self, lp, options: Options | None = None, **opts):
        if options is None:
            options = lpb_default_options(**opts)
        self.m, self.n = int(lp.m), int(lp.n)
        self.options = options
        self.ptr = lpb_create(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.vals, lp.c, lp.row_lo, lp.row_hi,
                              lp.var_lo, lp.var_hi, options)

    def solve(self, specs, tol: float = 1e-4, max_iter: int = 100000, warm_x=None, warm_y=None) -> Batch:
        sp = specs if isinstance(specs, np.ndarray) else specs_from(specs)
        b = Batch(self, lpb_solve(self.ptr, sp, tol, max_iter, warm_x, warm_y))
        b._num = int(sp.shape[0])
        return b

    def solve_dev(self, specs_dev, tol: float = 1e-4, max_iter: int = 100000, warm_x=None, warm_y=None) -> Batch:
        """specs_dev: a torch uint8 tensor on the handle's device holding
        num_lps packed records (SPEC_DTYPE layout); warm_* torch float64
        device tensors or None."""
        num = specs_dev.numel() // SPEC_DTYPE.itemsize
        b = Batch(self, lpb_solve_dev(self.ptr, num, specs_dev.data_ptr(), tol, max_iter,
                                      None if warm_x is None else warm_x.data_ptr(),
                                      None if warm_y is None else warm_y.data_ptr()))
        b._num = num
        return b

    @staticmethod
    def solve_multi(handles, specs, tol: float = 1e-4, max_iter: int = 100000):
        """Batches on several handles solved together (lpb_solve_multi):
        specs[i] for handles[i]; one Batch per handle."""
        sps = [sp if isinstance(sp, np.ndarray) else specs_from(sp) for sp in specs]
        ptrs = lpb_solve_multi([h.ptr for h in handles], sps, tol, max_iter)
        out = []
        for h, sp, p in zip(handles, sps, ptrs):
            b = Batch(h, p)
            b._num = int(sp.shape[0])
            out.append(b)
        return out

    def info(self):
        return lpb_handle_info(self.ptr)

    def tuning(self) -> Tuning:
        return lpb_get_tuning(self.ptr)

    def set_tuning(self, t: Tuning) -> None:
        lpb_set_tuning(self.ptr, t)

    def autotune(self, num_lps: int) -> Tuning:
        return lpb_autotune(self.ptr, num_lps)

    def tune_batch(self, widths):
        return lpb_tune_batch(self.ptr, widths)

    def scaling(self):
        return lpb_scaling(self.ptr, self.m, self.n)

    def close(self):
        if self.ptr is not None:
            lpb_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of solve requests over attached handles."""

    def __init__(self, options: ServerOptions | None = None, **opts):
        if options is None:
            options = lpb_server_default_options(**opts)
        self.ptr = lpb_server_create(options)
        self.handles = []

    def attach(self, handle: Handle) -> int:
        mid = lpb_server_attach(self.ptr, handle.ptr)
        self.handles.append(handle)
        return mid

    def submit(self, matrix_id: int, specs, tol: float = 1e-4, max_iter: int = 100000, warm_x=None, warm_y=None,
               warm_request: int = -1, warm_lp: int = 0) -> int:
        sp = specs if isinstance(specs, np.ndarray) else specs_from(specs)
        return lpb_server_submit(self.ptr, matrix_id, sp, tol, max_iter, warm_x, warm_y, warm_request, warm_lp)

    def poll(self, rid: int) -> bool:
        return lpb_server_poll(self.ptr, rid)

    def wait(self, rid: int, timeout_s: float = -1.0) -> None:
        lpb_server_wait(self.ptr, rid, timeout_s)

    def info(self, rid: int) -> RequestInfo:
        return lpb_server_request_info(self.ptr, rid)

    def results(self, rid: int) -> np.ndarray:
        return lpb_server_results(self.ptr, rid, self.info(rid).num_lps)

    def result(self, rid: int, matrix_id: int, lp: int, want_xy: bool = True):
        h = self.handles[matrix_id]
        return lpb_server_result(self.ptr, rid, lp, h.n, h.m, want_xy)

    def release(self, rid: int) -> None:
        lpb_server_release(self.ptr, rid)

    def stats(self) -> ServerStats:
        return lpb_server_stats_get(self.ptr)

    def close(self):
        if self.ptr is not None:
            lpb_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
