"""The no-allocation 2-way entry point (ps_metrics_2way_static).

It is for callers that cannot let a library call cudaMalloc (their device
memory is owned by their own allocator or a fixed start-up budget): its only
scratch is a static array in the library's device image.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel

pytestmark = pytest.mark.gpu
RTOL32 = 1e-5


def _run_both(ps, handle, V, out_dtype):
    import torch
    nf, nv = V.shape
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    tdt = torch.float32 if out_dtype == ps.PS_F32 else torch.float64
    ref = torch.empty(nv * (nv - 1) // 2, dtype=tdt, device="cuda")
    got = torch.full((nv * (nv - 1) // 2,), float("nan"), dtype=tdt, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), ps.PS_PATH_FP32, 0, ref.data_ptr(), out_dtype, st),
             handle.h)
    status = ps.ps_metrics_2way_static(ctypes.byref(m), got.data_ptr(), out_dtype, st)
    assert status == ps.PS_OK, ps.ps_last_error(None)
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.cpu().numpy()


def test_static_entry_matches_allocating_entry_twice(ps, handle):
    # two calls in a row with different sizes: the second must not see the
    # first call's scratch contents
    cases = [((1000, 777, 1), ps.PS_F32), ((1500, 300, 2), ps.PS_F64)]
    for (nv, nf, sub), odt in cases:
        V = synth.zero_inflated(nv, nf, synth.seed_for(6, sub))
        got, ref = _run_both(ps, handle, V, odt)
        assert not np.isnan(got).any()
        assert_rel(got, ref, RTOL32, f"static nv={nv}")


def test_static_entry_rejects_limits(ps, handle):
    import torch
    X = torch.zeros(8, 70000, device="cuda")
    out = torch.zeros(16, device="cuda")
    m = ps.matrix(X)  # nv = 70000 > PS_STATIC_MAX_NV
    assert ps.ps_metrics_2way_static(ctypes.byref(m), out.data_ptr(), ps.PS_F32, 0) == ps.PS_ERR_INVALID_ARG
    assert b"static scratch" in ps.ps_last_error(None)
    Xd = torch.zeros(8, 100, dtype=torch.float64, device="cuda")
    md = ps.matrix(Xd)
    assert ps.ps_metrics_2way_static(ctypes.byref(md), out.data_ptr(), ps.PS_F32, 0) == ps.PS_ERR_INVALID_ARG
    host = np.zeros((8, 100), np.float32)
    mh = ps.matrix(host)
    assert ps.ps_metrics_2way_static(ctypes.byref(mh), out.data_ptr(), ps.PS_F32, 0) == ps.PS_ERR_INVALID_ARG
