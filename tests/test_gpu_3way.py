"""GPU parity of the 3-way path (Section 2.2 eq. (1), Section 3.2) against the
oracle, on the pivot-slab layout."""
import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel, metrics_3way, slab_index

pytestmark = pytest.mark.gpu
RTOL32 = 1e-5


@pytest.mark.parametrize("nv,nf", [(3, 1), (4, 17), (5, 0), (64, 100), (129, 33), (200, 64), (257, 20)])
def test_all_triples_small(ps, handle, nv, nf):
    V = synth.zero_inflated(nv, nf, synth.seed_for(3, nv * 11 + nf))
    ref = oracle.c3_slab(oracle.to_vector_major(V), 0, nv)
    got = metrics_3way(ps, handle, V)
    assert_rel(got, ref, RTOL32, f"nv={nv} nf={nf}")


def test_slabs_concatenate_bit_exact(ps, handle):
    nv, nf = 300, 70
    V = synth.zero_inflated(nv, nf, synth.seed_for(3, 1))
    full = metrics_3way(ps, handle, V)
    parts = [metrics_3way(ps, handle, V, a, b) for a, b in [(0, 1), (1, 128), (128, 129), (129, 300)]]
    np.testing.assert_array_equal(np.concatenate(parts), full)


def test_integer_data_bit_exact(ps, handle):
    nv, nf = 150, 500
    V = synth.integer_levels(nv, nf, synth.seed_for(3, 2))
    ref = oracle.c3_slab(oracle.to_vector_major(V), 0, nv)
    got = metrics_3way(ps, handle, V)
    np.testing.assert_array_equal(got, ref.astype(np.float32))


def test_vector_major_and_f64_input(ps, handle):
    nv, nf = 140, 45
    V = synth.zero_inflated(nv, nf, synth.seed_for(3, 3), dtype=np.float64)
    ref = oracle.c3_slab(oracle.to_vector_major(V), 0, nv)
    assert_rel(metrics_3way(ps, handle, V), ref, RTOL32, "f64 field-major")
    assert_rel(metrics_3way(ps, handle, np.ascontiguousarray(V.T), layout=1), ref, RTOL32, "f64 vector-major")


def test_config3_full_size_sampled(ps, handle):
    """2048 x 4096 FP32, all 1.43e9 triples; 20000 sampled triples + tile
    corners against the oracle; every value in [0, 1]."""
    import torch
    nv, nf = 2048, 4096
    V = synth.zero_inflated(nv, nf, synth.seed_for(3))
    got_all = metrics_3way(ps, handle, V)
    assert got_all.size == nv * (nv - 1) * (nv - 2) // 6
    assert got_all.min() >= 0.0 and got_all.max() <= 1.0
    t = synth.sample_triples(nv, 20000, seed=9)
    t = np.concatenate([t, [[0, 1, 2], [126, 127, 128], [127, 128, 129], [0, 1, nv - 1], [nv - 3, nv - 2, nv - 1]]])
    got = got_all[slab_index(nv, 0, t[:, 0], t[:, 1], t[:, 2])]
    ref = oracle.c3_triples(oracle.to_vector_major(V), t)
    err = assert_rel(got, ref, RTOL32, "config3 sampled")
    print(f"config3 sampled max rel err {err:.3e}")
    del got_all
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nv,nf", [(129, 16), (300, 70), (517, 200)])
def test_operand_feeds_bit_identical(ps, handle, nv, nf):
    # the TMA-fed kernel (pivot min applied per slice in shared memory, warps
    # skipping blocks outside the pivot's rectangle; work items claimed from
    # a counter or assigned round-robin) and the cp.async kernels (8 and 16
    # warps) sum every triple in the same order: bit-identical slabs, whole
    # and by pivot ranges
    V = synth.zero_inflated(nv, nf, synth.seed_for(3, 81 + nv + nf))
    res = {}
    for feed, warps, sched in (("cpasync", "8", 0), ("cpasync", "16", 0), ("tma", "0", 1), ("tma", "0", 2)):
        h = ps.Handle(0, mgemm3_feed=2 if feed == "cpasync" else 1, mgemm_warps=int(warps),
                      mgemm3_schedule=sched)
        try:
            res[feed + warps + str(sched)] = [metrics_3way(ps, h, V),
                                 np.concatenate([metrics_3way(ps, h, V, a, b)
                                                 for a, b in [(0, 5), (5, min(130, nv)), (min(130, nv), nv)]])]
        finally:
            h.close()
    ref = oracle.c3_slab(oracle.to_vector_major(V), 0, nv)
    assert_rel(res["tma01"][0], ref, RTOL32, f"tma nv={nv} nf={nf}")
    for key, r in res.items():
        np.testing.assert_array_equal(r[0], res["cpasync80"][0], err_msg=key)
        np.testing.assert_array_equal(r[1], res["cpasync80"][0], err_msg=key + " pivot ranges")
