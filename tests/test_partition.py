"""Sharding of the unique outputs over ranks (one GPU per rank, V replicated,
no collective on the data path).  Host logic only: the partition comes from
the C library (ps_partition, no GPU needed); each gloo rank computes its
shard with the oracle as the CPU stand-in for its GPU, and the shards are
gathered and checked against the full result."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1705_08210_gb300 import synth


def _part(ps, nv, way, n, p):
    b, e, ob, oe = (ctypes.c_int64() for _ in range(4))
    assert ps.ps_partition(nv, way, n, p, ctypes.byref(b), ctypes.byref(e), ctypes.byref(ob),
                           ctypes.byref(oe)) == ps.PS_OK
    return b.value, e.value, ob.value, oe.value


@pytest.mark.parametrize("nv", [3, 130, 1000, 32768])
@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_partitions_cover_and_balance(ps, nv, nparts):
    for way in (2, 3):
        parts = [_part(ps, nv, way, nparts, p) for p in range(nparts)]
        assert parts[0][0] == 0 and parts[-1][1] == nv
        total = nv * (nv - 1) // 2 if way == 2 else nv * (nv - 1) * (nv - 2) // 6
        assert parts[0][2] == 0 and parts[-1][3] == total
        for a, b in zip(parts, parts[1:]):
            assert a[1] == b[0] and a[3] == b[2]           # contiguous, disjoint
        if way == 2:
            assert all(p[0] % 128 == 0 or p[0] == nv for p in parts)  # whole 128-row tiles
        if nv >= 1000 and nparts > 1:
            work = np.array([p[3] - p[2] for p in parts], dtype=np.float64)
            slack = (128 * nv) if way == 2 else (2 * nv * nv)
            assert np.all(np.abs(work - total / nparts) <= slack), work


def test_partition_rejects_bad_arguments(ps):
    b = ctypes.c_int64()
    assert ps.ps_partition(10, 4, 2, 0, ctypes.byref(b), ctypes.byref(b), None, None) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_partition(10, 2, 2, 2, ctypes.byref(b), ctypes.byref(b), None, None) == ps.PS_ERR_INVALID_ARG


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, nv, nf):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1705_08210_gb300 import ps
    V = oracle.to_vector_major(synth.zero_inflated(nv, nf, synth.seed_for(9, 1)))
    # 2-way: rows [b, e) of the packed triangle
    b, e, ob, oe = _part(ps, nv, 2, world, rank)
    pairs = np.array([(i, j) for i in range(b, e) for j in range(i + 1, nv)], dtype=np.int64).reshape(-1, 2)
    shard2 = torch.from_numpy(oracle.c2_pairs(V, pairs) if len(pairs) else np.zeros(0))
    assert shard2.numel() == oe - ob
    # 3-way: pivots [jb, je)
    jb, je, ob3, oe3 = _part(ps, nv, 3, world, rank)
    shard3 = torch.from_numpy(oracle.c3_slab(V, jb, je))
    assert shard3.numel() == oe3 - ob3
    got2 = [None] * world
    got3 = [None] * world
    dist.all_gather_object(got2, shard2)
    dist.all_gather_object(got3, shard3)
    if rank == 0:
        np.testing.assert_array_equal(torch.cat(got2).numpy(), oracle.c2_packed(V))
        np.testing.assert_array_equal(torch.cat(got3).numpy(), oracle.c3_slab(V, 0, nv))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_merge(ps):
    mp.start_processes(_rank, args=(2, _free_port(), 300, 24), nprocs=2, join=True, start_method="spawn")
