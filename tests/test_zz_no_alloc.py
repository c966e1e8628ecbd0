"""lpb_scaling_noalloc: equilibration factors for callers that cannot
allocate device memory (code running under CUDA graph capture, callers that
must not trigger the allocator's synchronization, hosts that own all device
memory through their own pool).  The entry point uses the library's fixed
device scratch; its factors must match those lpb_create computes (read back
with lpb_scaling) on two calls in a row, the second reusing the scratch the
first left behind.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the tolerance the scaling parity test against the oracle uses


def test_scaling_noalloc_matches_create_on_two_calls():
    import torch

    from paper_2601_21990_gb300 import _build, lpb

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    _build.build()
    lpb.load()
    w = lpgen.sb_powerlaw(seed=0)
    lp = w.lp
    h = lpb.Handle(lp, precision=lpb.MIXED, ruiz_iters=10, pock_chambolle=1)
    dr_ref, dc_ref = h.scaling()
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.tensor(lp.row_ptr.astype(np.int32), device=dev)
    ci = torch.tensor(lp.col_idx.astype(np.int32), device=dev)
    va = torch.tensor(lp.vals.astype(np.float64), device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        dr = torch.full((lp.m,), -1.0, dtype=torch.float64, device=dev)
        dc = torch.full((lp.n,), -1.0, dtype=torch.float64, device=dev)
        lpb.lpb_scaling_noalloc(lp.m, lp.n, lp.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 10, 1,
                                dr.data_ptr(), dc.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        np.testing.assert_allclose(dr.cpu().numpy(), dr_ref, rtol=RTOL)
        np.testing.assert_allclose(dc.cpu().numpy(), dc_ref, rtol=RTOL)
    h.close()


def test_scaling_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2601_21990_gb300 import _build, lpb

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    _build.build()
    lpb.load()
    with pytest.raises(lpb.LpbError) as e:
        lpb.lpb_scaling_noalloc(2_000_000, 200_000, 0, 1, None, None, 10, 1, 1, 1, None)
    assert e.value.code == lpb.LPB_ERR_INVALID_ARG
    assert "scratch" in lpb.lpb_last_error()
