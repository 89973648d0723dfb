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
    assert len(lines) == 1 and len(lines[0]["ms"]) == 9
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
