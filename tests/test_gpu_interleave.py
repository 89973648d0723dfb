"""Calls of every kind and many shapes interleaved on ONE handle, each 3-way
result checked against the oracle (Section 2.2 eq. (1)) and each 2-way
result against the oracle (Section 2.1).

State that lives in the handle across calls is what this exercises: the
grid-wide tile and work-item counters of the TMA kernels (zeroed before each
launch), the 3-way work-item table, workspace slots that grow (and are
reallocated) while earlier launches may still be queued, the cached batched
graphs, and switching the 3-way work schedule between calls."""
import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel, metrics_2way, metrics_3way, threshold_3way

pytestmark = pytest.mark.gpu
RTOL32 = 1e-5

# (nv, nf) of the 3-way calls: ragged tiles, one and several 64-field
# slices, sizes that grow and shrink the workspace
SHAPES3 = [(200, 64), (129, 33), (300, 70), (64, 100), (257, 20), (200, 64), (517, 130), (130, 16), (200, 64)]


def _batch(ps, seed):
    from test_gpu_batched import _make_batch
    shapes = [(2, 256, 512), (3, 150, 96), (2, 700, 40), (3, 131, 200)]
    return shapes, _make_batch(ps, shapes, seed)


@pytest.mark.parametrize("rounds", [2])
def test_interleaved_calls_one_handle(ps, rounds):
    import torch
    h = ps.Handle(0)
    try:
        st = torch.cuda.current_stream().cuda_stream
        for r in range(rounds):
            for n, (nv, nf) in enumerate(SHAPES3):
                # alternate the 3-way work schedule: counter-claimed and static
                h.set_config(mgemm3_schedule=1 + (n + r) % 2)
                V3 = synth.zero_inflated(nv, nf, synth.seed_for(3, 700 + 13 * n + r))
                Vv3 = oracle.to_vector_major(V3)
                # a 2-way call of another shape just before (shares the n2
                # launcher's counter word and the sums slot)
                V2 = synth.zero_inflated(nv + 37 * n + 1, 1 + (nf * 3) % 97, synth.seed_for(1, 800 + n + r))
                g2 = metrics_2way(ps, h, V2)
                got = metrics_3way(ps, h, V3)
                assert_rel(got, oracle.c3_slab(Vv3, 0, nv), RTOL32, f"round {r} 3-way {n} nv={nv} nf={nf}")
                assert_rel(g2, oracle.c2_packed(oracle.to_vector_major(V2)), RTOL32, f"round {r} 2-way {n}")
                # a pivot range of the same matrix right after
                jb, je = nv // 3, nv // 3 + 5
                assert_rel(metrics_3way(ps, h, V3, jb, je), oracle.c3_slab(Vv3, jb, je), RTOL32,
                           f"round {r} slab {n}")
                if n % 3 == 0 and nv <= 300:
                    # thresholded 3-way (its own n2 table and block list):
                    # the same triples as the oracle outside the FP32
                    # disagreement band around tau, values within tolerance
                    tau = 0.35
                    ref_t, ref_v, total = oracle.threshold_3way(Vv3, tau)
                    s, c, trip, vals = threshold_3way(ps, h, V3, tau, capacity=total + 1000)
                    assert s == ps.PS_OK
                    sure = np.abs(ref_v - tau) > 1e-5 * tau
                    got = dict(zip(map(tuple, trip.tolist()), vals.tolist()))
                    for key, v in zip(map(tuple, ref_t[sure].tolist()), ref_v[sure]):
                        assert key in got and abs(got[key] - v) <= RTOL32 * v, (r, n, key)
                if n % 3 == 1:
                    # thresholded 2-way, checked the same way
                    from gpu_run import threshold_2way
                    ref_p, ref_v = oracle.threshold_2way(oracle.to_vector_major(V2), 0.3)
                    s, c, pairs, vals = threshold_2way(ps, h, V2, 0.3, capacity=len(ref_p) + 1000)
                    assert s == ps.PS_OK
                    sure = np.abs(ref_v - 0.3) > 1e-5 * 0.3
                    got = set(map(tuple, pairs.tolist()))
                    assert set(map(tuple, ref_p[sure].tolist())) <= got
                if n % 3 == 2:
                    # batched launch (cached graph after the first round)
                    shapes, (probs, keep) = _batch(ps, 9500 + n)
                    ps.check(ps.ps_metrics_batched(h.h, probs, len(shapes), ps.PS_BATCH_PERSISTENT, st), h.h)
                    torch.cuda.synchronize()
                    for t, ((way, bnv, bnf), (V, X, o)) in enumerate(zip(shapes, keep)):
                        Vv = oracle.to_vector_major(V)
                        ref = oracle.c2_packed(Vv) if way == 2 else oracle.c3_slab(Vv, 0, bnv)
                        assert_rel(o.cpu().numpy(), ref, RTOL32, f"round {r} batched {n}.{t}")
    finally:
        h.close()


def test_repeated_3way_same_handle_both_schedules(ps):
    # the exact case that once failed inside the full suite (nv = 200,
    # n_f = 64: one 64-field slice per work item, so the producer runs two
    # items ahead of the warps), many times in a row on one handle, with both
    # schedules; every result bit-identical to the first and to the oracle
    h = ps.Handle(0)
    try:
        nv, nf = 200, 64
        V = synth.zero_inflated(nv, nf, synth.seed_for(3, nv * 11 + nf))
        ref = oracle.c3_slab(oracle.to_vector_major(V), 0, nv)
        first = metrics_3way(ps, h, V)
        assert_rel(first, ref, RTOL32, "first")
        for k in range(40):
            h.set_config(mgemm3_schedule=1 + k % 2)
            np.testing.assert_array_equal(metrics_3way(ps, h, V), first, err_msg=f"repeat {k}")
    finally:
        h.close()
