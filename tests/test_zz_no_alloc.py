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
    # first call's scratch contents.  Same values as ps_metrics_2way bit for
    # bit (both kernels sum in the same order and round the same way), and
    # sampled pairs against the FP64 oracle
    import oracle
    cases = [((1000, 777, 1), ps.PS_F32), ((1500, 300, 2), ps.PS_F64)]
    for (nv, nf, sub), odt in cases:
        V = synth.zero_inflated(nv, nf, synth.seed_for(6, sub))
        got, ref = _run_both(ps, handle, V, odt)
        assert not np.isnan(got).any()
        np.testing.assert_array_equal(got, ref)
        pairs = synth.sample_pairs(nv, 3000, seed=sub)
        idx = pairs[:, 0] * (2 * nv - pairs[:, 0] - 1) // 2 + (pairs[:, 1] - pairs[:, 0] - 1)
        assert_rel(got[idx], oracle.c2_pairs(oracle.to_vector_major(V), pairs), RTOL32, f"static nv={nv}")


def test_static_entry_allocates_no_device_memory(ps, handle):
    # the property the entry point exists for: across a call (after the
    # first one on this device, which loads the library's kernels) the
    # device's free memory does not change
    import torch
    nv, nf = 4000, 500
    V = synth.zero_inflated(nv, nf, synth.seed_for(6, 3))
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    out = torch.empty(nv * (nv - 1) // 2, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert ps.ps_metrics_2way_static(ctypes.byref(m), out.data_ptr(), ps.PS_F32, st) == ps.PS_OK
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    assert ps.ps_metrics_2way_static(ctypes.byref(m), out.data_ptr(), ps.PS_F32, st) == ps.PS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.equal(out, first)


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
