"""Batched uneven instances: the persistent graph-captured launch must give
bit-identical results to one call per instance, and both must match the
oracle; the autotuner records its choice in a JSON cache."""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel

pytestmark = pytest.mark.gpu


def _make_batch(ps, shapes, seed):
    import torch
    keep, probs = [], (ps.ps_problem * len(shapes))()
    for t, (way, nv, nf) in enumerate(shapes):
        V = synth.zero_inflated(nv, nf, seed + t)
        ld = (nv + 3) // 4 * 4  # batched inputs need ld % 4 == 0
        Xp = torch.full((nf, ld), float("nan"), device="cuda")
        Xp[:, :nv] = torch.from_numpy(V).cuda()
        X = Xp[:, :nv]
        n = nv * (nv - 1) // 2 if way == 2 else ps.ps_slab_size(nv, 0, nv)
        out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        probs[t].V = ps.matrix(X)
        probs[t].way = way
        probs[t].out_dtype = ps.PS_F32
        probs[t].out = out.data_ptr()
        keep.append((V, X, out))
    return probs, keep


SHAPES = [(2, 256, 512), (3, 300, 700), (2, 1000, 96), (2, 129, 2000), (3, 130, 64), (2, 2, 5),
          (3, 3, 17), (2, 700, 1500), (3, 257, 300)]


def test_batched_matches_per_instance_and_oracle(ps, handle):
    import torch
    probs, keep = _make_batch(ps, SHAPES, 4000)
    st = torch.cuda.current_stream().cuda_stream
    ps.check(ps.ps_metrics_batched(handle.h, probs, len(SHAPES), ps.PS_BATCH_PERSISTENT, st), handle.h)
    got = [o.cpu().numpy().copy() for _, _, o in keep]
    # replay of the cached graph after changing the inputs in place
    for (V, X, o) in keep:
        o.fill_(float("nan"))
    ps.check(ps.ps_metrics_batched(handle.h, probs, len(SHAPES), ps.PS_BATCH_PERSISTENT, st), handle.h)
    again = [o.cpu().numpy().copy() for _, _, o in keep]
    for a, b in zip(got, again):
        np.testing.assert_array_equal(a, b)
    for (V, X, o) in keep:
        o.fill_(float("nan"))
    ps.check(ps.ps_metrics_batched(handle.h, probs, len(SHAPES), ps.PS_BATCH_PER_INSTANCE, st), handle.h)
    torch.cuda.synchronize()
    for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(SHAPES, keep)):
        ref_gpu = o.cpu().numpy()
        np.testing.assert_array_equal(got[t], ref_gpu)
        Vv = oracle.to_vector_major(V)
        ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, nv)
        assert_rel(got[t], ref, 1e-5, f"batched problem {t}")


def test_batched_new_data_same_buffers(ps, handle):
    import torch
    probs, keep = _make_batch(ps, SHAPES[:4], 5000)
    st = torch.cuda.current_stream().cuda_stream
    ps.check(ps.ps_metrics_batched(handle.h, probs, 4, ps.PS_BATCH_PERSISTENT, st), handle.h)
    # new values in the same device buffers: the replayed graph must see them
    for t, (V, X, o) in enumerate(keep):
        V2 = synth.zero_inflated(V.shape[1], V.shape[0], 6000 + t)
        X.copy_(torch.from_numpy(V2).cuda())
        keep[t] = (V2, X, o)
    ps.check(ps.ps_metrics_batched(handle.h, probs, 4, ps.PS_BATCH_PERSISTENT, st), handle.h)
    torch.cuda.synchronize()
    for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(SHAPES[:4], keep)):
        Vv = oracle.to_vector_major(V)
        ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, nv)
        assert_rel(o.cpu().numpy(), ref, 1e-5, f"new data problem {t}")


def test_autotuner_writes_cache_and_reuses_it(ps, handle, tmp_path):
    import torch
    probs, keep = _make_batch(ps, SHAPES[:5], 7000)
    st = torch.cuda.current_stream().cuda_stream
    path = str(tmp_path / "tune.jsonl")
    buf = ctypes.create_string_buffer(128)
    ps.check(ps.ps_autotune_batched(handle.h, probs, 5, path.encode(), buf, 128, st), handle.h)
    lines = [json.loads(x) for x in open(path)]
    assert len(lines) == 1 and len(lines[0]["ms"]) == 10  # the TMA-fed kernel and 9 cp.async variants
    assert str(lines[0]["variant"]) in lines[0]["ms"]
    buf2 = ctypes.create_string_buffer(128)
    ps.check(ps.ps_autotune_batched(handle.h, probs, 5, path.encode(), buf2, 128, st), handle.h)
    assert b"cached" in buf2.value
    assert len(open(path).readlines()) == 1
    ps.check(ps.ps_metrics_batched(handle.h, probs, 5, ps.PS_BATCH_PERSISTENT, st), handle.h)
    torch.cuda.synchronize()
    for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(SHAPES[:5], keep)):
        Vv = oracle.to_vector_major(V)
        ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, nv)
        assert_rel(o.cpu().numpy(), ref, 1e-5, f"tuned problem {t}")


def test_batched_rejects_bad_problems(ps, handle):
    import torch
    probs, keep = _make_batch(ps, SHAPES[:2], 8000)
    probs[1].way = 4
    assert ps.ps_metrics_batched(handle.h, probs, 2, 0, 0) == ps.PS_ERR_INVALID_ARG
    probs[1].way = 3
    probs[1].V.dtype = ps.PS_F64
    assert ps.ps_metrics_batched(handle.h, probs, 2, 0, 0) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_metrics_batched(handle.h, probs, 0, 0, 0) == ps.PS_ERR_INVALID_ARG


def test_dependency_wait_timeout_reports_and_handle_recovers(ps):
    # The timeout path of the persistent launch, in the allowed form: a
    # dependency count that nothing completes.  test_batched_stall raises the
    # first 3-way problem's n2-table target by one store that never comes
    # (TMA-fed kernel; the cp.async kernel raises problem 0's sums target);
    # with a 1 ms wait limit the first 3-way epilogue that waits on it gives
    # up, raises the launch's error flag, every later wait sees the flag, and
    # the call returns PS_ERR_TIMEOUT.  No kernel is altered and no GPU wait
    # is unbounded.  The next call on the same handle is normal and correct.
    import time
    import torch
    h = ps.Handle(0, wait_limit_ns=1_000_000)
    try:
        probs, keep = _make_batch(ps, SHAPES[:4], 9300)
        st = torch.cuda.current_stream().cuda_stream
        h.set_config(test_batched_stall=1)
        t0 = time.perf_counter()
        s = ps.ps_metrics_batched(h.h, probs, 4, ps.PS_BATCH_PERSISTENT, st)
        dt = time.perf_counter() - t0
        assert s == ps.PS_ERR_TIMEOUT, ps.ps_last_error(h.h)
        assert b"timed out" in ps.ps_last_error(h.h)
        assert dt < 30.0
        assert h.get_config().test_batched_stall == 0  # one-shot
        for (V, X, o) in keep:
            o.fill_(float("nan"))
        ps.check(ps.ps_metrics_batched(h.h, probs, 4, ps.PS_BATCH_PERSISTENT, st), h.h)
        torch.cuda.synchronize()
        for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(SHAPES[:4], keep)):
            Vv = oracle.to_vector_major(V)
            ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, nv)
            assert_rel(o.cpu().numpy(), ref, 1e-5, f"after timeout, problem {t}")
        # the other entry points of the handle work too
        from gpu_run import metrics_2way
        V = synth.zero_inflated(300, 40, synth.seed_for(4, 9301))
        assert_rel(metrics_2way(ps, h, V), oracle.c2_packed(oracle.to_vector_major(V)), 1e-5, "2-way after")
    finally:
        h.close()


def test_config4_shapes_sampled(ps, handle):
    # the 64 uneven instances of the batched workload (48 2-way with nv in
    # [256, 4096], 16 3-way with nv in [256, 1024], nf in [512, 8192]) in one
    # persistent launch: sampled pairs and triples of every instance against
    # the oracle, and bit-identity with one call per instance
    import torch
    shapes = synth.batched_shapes(synth.seed_for(4))
    assert len(shapes) == 64 and sum(w == 3 for w, _, _ in shapes) == 16
    probs, keep = _make_batch(ps, shapes, synth.seed_for(4, 1))
    st = torch.cuda.current_stream().cuda_stream
    ps.check(ps.ps_metrics_batched(handle.h, probs, 64, ps.PS_BATCH_PERSISTENT, st), handle.h)
    torch.cuda.synchronize()
    got = [o.cpu().numpy().copy() for _, _, o in keep]
    for t, ((way, nv, nf), (V, X, o)) in enumerate(zip(shapes, keep)):
        Vv = oracle.to_vector_major(V)
        if way == 2:
            pairs = synth.sample_pairs(nv, 300, seed=t)
            pairs = np.concatenate([pairs, [[0, 1], [0, nv - 1], [nv - 2, nv - 1], [127, 128]]])
            idx = pairs[:, 0] * (2 * nv - pairs[:, 0] - 1) // 2 + (pairs[:, 1] - pairs[:, 0] - 1)
            assert_rel(got[t][idx], oracle.c2_pairs(Vv, pairs), 1e-5, f"instance {t} pairs")
        else:
            from gpu_run import slab_index
            tr = synth.sample_triples(nv, 300, seed=t)
            tr = np.concatenate([tr, [[0, 1, 2], [0, 1, nv - 1], [nv - 3, nv - 2, nv - 1], [126, 127, 128]]])
            idx = slab_index(nv, 0, tr[:, 0], tr[:, 1], tr[:, 2])
            assert_rel(got[t][idx], oracle.c3_triples(Vv, tr), 1e-5, f"instance {t} triples")
        assert np.all(np.isfinite(got[t])) and got[t].min() >= 0.0 and got[t].max() <= 1.0
    for (V, X, o) in keep:
        o.fill_(float("nan"))
    ps.check(ps.ps_metrics_batched(handle.h, probs, 64, ps.PS_BATCH_PER_INSTANCE, st), handle.h)
    torch.cuda.synchronize()
    for t, (V, X, o) in enumerate(keep):
        np.testing.assert_array_equal(got[t], o.cpu().numpy(), err_msg=f"instance {t}")
