"""Per-handle configuration (ps_config): debug input checks, the paper's DP
arithmetic as a run-time precision, reading and replacing a handle's
configuration, and the autotune cache named by the configuration."""
import ctypes
import json

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel, metrics_2way

pytestmark = pytest.mark.gpu


def test_debug_checks_reject_invalid_input(ps):
    # Section 2.1 assumes v >= 0; with debug_checks a negative, NaN or
    # infinite entry is an argument error and the output stays untouched
    import torch
    h = ps.Handle(0, debug_checks=1)
    try:
        V = synth.zero_inflated(200, 30, synth.seed_for(1, 501))
        ref = oracle.c2_packed(oracle.to_vector_major(V))
        assert_rel(metrics_2way(ps, h, V), ref, 1e-5, "valid input")
        for bad in (-1.0, float("nan"), float("inf")):
            W = V.copy()
            W[7, 123] = bad
            X = torch.from_numpy(W).cuda()
            m = ps.matrix(X)
            out = torch.full((200 * 199 // 2,), 7.0, device="cuda")
            st = ps.ps_metrics_2way(h.h, ctypes.byref(m), ps.PS_PATH_FP32, 0, out.data_ptr(), ps.PS_F32,
                                    torch.cuda.current_stream().cuda_stream)
            assert st == ps.PS_ERR_INVALID_ARG, bad
            assert b"debug check" in ps.ps_last_error(h.h)
            assert torch.all(out == 7.0)
            # vector-major FP64 input takes the same check
            m64 = ps.matrix(torch.from_numpy(np.ascontiguousarray(W.T).astype(np.float64)).cuda(),
                            ps.PS_LAYOUT_VECTOR_MAJOR)
            out3 = torch.empty(ps.ps_slab_size(200, 0, 200), device="cuda")
            assert ps.ps_metrics_3way(h.h, ctypes.byref(m64), 0, 200, out3.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream) == ps.PS_ERR_INVALID_ARG
    finally:
        h.close()


def test_fp64_precision_handle(ps):
    # the paper's DP build as a handle setting: the sharded 2-way call runs
    # the FP64 kernel (agreement with the FP64 oracle to ~1e-13), the calls
    # without an FP64 kernel say so
    import torch
    h = ps.Handle(0, precision=ps.PS_PATH_FP64)
    try:
        nv, nf = 700, 333
        V = synth.zero_inflated(nv, nf, synth.seed_for(1, 502), dtype=np.float64)
        ref = oracle.c2_packed(oracle.to_vector_major(V))
        X = torch.from_numpy(V).cuda()
        m = ps.matrix(X)
        out = torch.full((nv * (nv - 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
        for p in range(3):
            ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), 3, p, out.data_ptr(), ps.PS_F64,
                                             torch.cuda.current_stream().cuda_stream), h.h)
        torch.cuda.synchronize()
        assert_rel(out.cpu().numpy(), ref, 1e-13, "fp64 precision, parts")
        out3 = torch.empty(ps.ps_slab_size(nv, 0, nv), device="cuda")
        assert ps.ps_metrics_3way(h.h, ctypes.byref(m), 0, nv, out3.data_ptr(), 0) == ps.PS_ERR_UNSUPPORTED
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert ps.ps_threshold_2way(h.h, ctypes.byref(m), 0.5, None, 0, cnt.data_ptr(), 0) == ps.PS_ERR_UNSUPPORTED
    finally:
        h.close()


def test_get_and_set_config(ps):
    # a handle's kernel choice changes between calls; values stay bit-identical
    h = ps.Handle(0, mgemm_band=3, wait_limit_ns=500_000_000)
    try:
        c = h.get_config()
        assert c.mgemm_band == 3 and c.wait_limit_ns == 500_000_000
        V = synth.zero_inflated(1000, 100, synth.seed_for(1, 503))
        a = metrics_2way(ps, h, V)
        h.set_config(mgemm_feed=2, mgemm_band=0)
        c = h.get_config()
        assert c.mgemm_feed == 2 and c.mgemm_band == 0 and c.wait_limit_ns == 500_000_000
        np.testing.assert_array_equal(metrics_2way(ps, h, V), a)
        bad = h.get_config()
        bad.tma_slice = 7
        assert ps.ps_set_config(h.h, ctypes.byref(bad)) == ps.PS_ERR_INVALID_ARG
    finally:
        h.close()


def test_autotune_cache_from_config(ps, tmp_path):
    # ps_autotune_batched with cache_path NULL writes the configured cache;
    # a second handle with the same configured cache uses the stored variant
    import torch
    from test_gpu_batched import _make_batch, SHAPES
    path = str(tmp_path / "tune.jsonl")
    probs, keep = _make_batch(ps, SHAPES[:3], 9100)
    st = torch.cuda.current_stream().cuda_stream
    h = ps.Handle(0, autotune_cache=path)
    try:
        assert h.get_config().autotune_cache == path.encode()
        buf = ctypes.create_string_buffer(128)
        ps.check(ps.ps_autotune_batched(h.h, probs, 3, None, buf, 128, st), h.h)
        line = json.loads(open(path).read().strip())
        assert line["problems"] == 3
    finally:
        h.close()
    h2 = ps.Handle(0, autotune_cache=path)
    try:
        ps.check(ps.ps_metrics_batched(h2.h, probs, 3, ps.PS_BATCH_PERSISTENT, st), h2.h)
        torch.cuda.synchronize()
        for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(SHAPES[:3], keep)):
            Vv = oracle.to_vector_major(V)
            ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, nv)
            assert_rel(o.cpu().numpy(), ref, 1e-5, f"cached-variant problem {t}")
    finally:
        h2.close()
