"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
exports every function include/lpb.h declares, and the ctypes mirrors of the
header's structs have the header's sizes and offsets.  No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lpb.h")
SERVE_HEADER = os.path.join(ROOT, "include", "lpb_serve.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2601_21990_gb300 import _build, lpb

    _build.build()
    return lpb.load()


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lpb_err|void|const char\*)\s+(lpb_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_expected_calls():
    names = declared_functions()
    for n in ("lpb_create", "lpb_solve", "lpb_solve_dev", "lpb_result", "lpb_batch_free", "lpb_destroy",
              "lpb_last_error", "lpb_default_options"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions() + declared_functions(SERVE_HEADER):
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2601_21990_gb300 import lpb

    assert sorted(lpb.EXPORTS) == declared_functions()
    assert sorted(lpb.SERVE_EXPORTS) == declared_functions(SERVE_HEADER)


def test_serve_struct_layouts_match_header(tmp_path):
    from paper_2601_21990_gb300 import lpb

    src = tmp_path / "szs.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lpb_serve.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(lpb_server_options), sizeof(lpb_request), sizeof(lpb_request_info),
         sizeof(lpb_server_stats));
  printf("%zu %zu %zu\\n", offsetof(lpb_request, warm_request), offsetof(lpb_request_info, t_submit),
         offsetof(lpb_server_stats, busy_s));
  return 0;
}
""")
    exe = tmp_path / "szs"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    v = [int(x) for x in subprocess.check_output([str(exe)]).decode().split()]
    assert v[:4] == [ctypes.sizeof(lpb.ServerOptions), ctypes.sizeof(lpb.Request), ctypes.sizeof(lpb.RequestInfo),
                     ctypes.sizeof(lpb.ServerStats)]
    assert v[4:] == [lpb.Request.warm_request.offset, lpb.RequestInfo.t_submit.offset, lpb.ServerStats.busy_s.offset]


def test_server_create_without_device_fails_cleanly(lib):
    """No GPU here: creating a server returns an error code, never aborts."""
    import torch

    from paper_2601_21990_gb300 import lpb

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lpb.LpbError):
        lpb.Server()


def test_default_options(lib):
    from paper_2601_21990_gb300 import lpb

    o = lpb.lpb_default_options()
    assert o.precision == lpb.MIXED and o.check_every == 64 and o.ruiz_iters == 10
    assert (o.beta_s, o.beta_n, o.beta_a, o.theta, o.mnorm_sign) == (0.2, 0.8, 0.36, 0.5, -1.0)
    assert o.device == -1 and o.cuda_stream is None


def test_option_validation_rejects_bad_values(lib):
    """Option checks run before any device call, so they need no GPU."""
    from paper_2601_21990_gb300 import lpb

    assert lpb.lpb_default_options().reduced_cost == lpb.RC_BARRIER
    ok = dict(m=1, n=2, row_ptr=[0, 2], col_idx=[0, 1], vals=[1.0, 1.0], c=[1.0, 1.0], row_lo=[0.0],
              row_hi=[1.0], var_lo=[0.0, 0.0], var_hi=[1.0, 1.0])
    bad = [dict(reduced_cost=2), dict(reduced_cost=-1), dict(polish_arith=5), dict(precision=7),
           dict(check_every=0), dict(theta=1.5), dict(beta_s=-0.1), dict(power_max_iter=0)]
    for b in bad:
        with pytest.raises(lpb.LpbError) as e:
            lpb.lpb_create(**ok, options=lpb.lpb_default_options(**b))
        assert e.value.code == lpb.LPB_ERR_INVALID_ARG, b


def test_struct_layouts_match_header(tmp_path):
    from paper_2601_21990_gb300 import lpb

    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lpb.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(lpb_options), sizeof(lpb_lp_spec), sizeof(lpb_lp_result), sizeof(lpb_profile));
  printf("%zu %zu %zu\\n", offsetof(lpb_options, cuda_stream), offsetof(lpb_options, device), offsetof(lpb_profile, kernels));
  return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = [int(v) for v in out]
    assert sizes[:4] == [ctypes.sizeof(lpb.Options), ctypes.sizeof(lpb.Spec), ctypes.sizeof(lpb.Result),
                         ctypes.sizeof(lpb.Profile)]
    assert sizes[4] == lpb.Options.cuda_stream.offset
    assert sizes[5] == lpb.Options.device.offset
    assert sizes[6] == lpb.Profile.kernels.offset


def test_no_device_is_an_error_not_a_fallback(lib):
    """Without a GPU the library returns an error code; nothing computes on
    the CPU."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import lpgen
    from paper_2601_21990_gb300 import lpb

    w = lpgen.sb_small()
    with pytest.raises(lpb.LpbError) as e:
        lpb.Handle(w.lp)
    assert e.value.code == lpb.LPB_ERR_CUDA


def test_host_validation_rejects_bad_csr(lib):
    """Argument checks run before any device call."""
    import numpy as np

    from paper_2601_21990_gb300 import lpb

    inf = np.inf
    ok = dict(m=1, n=2, row_ptr=[0, 2], col_idx=[0, 1], vals=[1.0, 1.0], c=[1.0, 1.0], row_lo=[0.0],
              row_hi=[1.0], var_lo=[0.0, 0.0], var_hi=[1.0, 1.0])
    bad = [dict(col_idx=[0, 2]), dict(vals=[1.0, np.nan]), dict(row_lo=[2.0]), dict(var_lo=[0.0, 2.0]),
           dict(row_ptr=[1, 2]), dict(c=[inf, 1.0]), dict(row_lo=[inf]), dict(var_hi=[1.0, -inf])]
    for b in bad:
        kw = dict(ok)
        kw.update(b)
        with pytest.raises(lpb.LpbError) as e:
            lpb.lpb_create(**kw)
        assert e.value.code == lpb.LPB_ERR_INVALID_ARG, b


def test_joint_solve_argument_checks_need_no_device(lib):
    """lpb_solve_multi rejects a bad count or NULL arrays before any device
    call (and sets the last error), so these run without a GPU."""
    import ctypes as C

    from paper_2601_21990_gb300 import lpb

    out = (C.c_void_p * 2)()
    hv = (C.c_void_p * 2)()
    nv = (C.c_int32 * 2)(1, 1)
    pv = (C.c_void_p * 2)()
    cases = [(0, hv, nv, pv, out), (lpb.LPB_MAX_JOINT + 1, hv, nv, pv, out), (1, None, nv, pv, out),
             (1, hv, None, pv, out), (1, hv, nv, None, out), (1, hv, nv, pv, None), (2, hv, nv, pv, out)]
    for k, h, n, p, o in cases:
        assert lib.lpb_solve_multi(k, h, n, p, 1e-4, 100, o) == lpb.LPB_ERR_INVALID_ARG, k
        assert lib.lpb_last_error()
    assert lib.lpb_solve_multi(1, hv, nv, pv, 0.0, 100, out) == lpb.LPB_ERR_INVALID_ARG  # tol
