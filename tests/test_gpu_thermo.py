"""GPU parity of the quantized thermometer path (tensor cores) against the
oracle evaluated on the quantized levels: bit-exact.  The quantizer itself
(percentile P and every level) is integer work and must match bit for bit."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import metrics_2way

pytestmark = pytest.mark.gpu


def _quantize_gpu(ps, handle, V, levels):
    import torch
    X = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    nf, nv = V.shape
    q = torch.empty(nf * nv, dtype=torch.uint8, device="cuda")
    P = torch.empty(1, dtype=torch.float32, device="cuda")
    m = ps.matrix(X)
    ps.check(ps.ps_quantize(handle.h, ctypes.byref(m), levels, P.data_ptr(), q.data_ptr(),
                            torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    return float(P.item()), q.cpu().numpy().reshape(nf, nv)


@pytest.mark.parametrize("nv,nf,levels,pz", [(300, 200, 16, 0.85), (64, 33, 5, 0.5), (7, 3, 2, 0.2),
                                             (1000, 1000, 16, 0.99)])
def test_quantizer_bit_exact(ps, handle, nv, nf, levels, pz):
    V = synth.zero_inflated(nv, nf, synth.seed_for(2, nv + nf), p_zero=pz)
    P, q = _quantize_gpu(ps, handle, V, levels)
    Pref = oracle.percentile_nonzero(V)
    assert P == Pref
    np.testing.assert_array_equal(q, oracle.quantize(V, levels, Pref))


def test_quantizer_all_zero(ps, handle):
    V = np.zeros((10, 20), np.float32)
    P, q = _quantize_gpu(ps, handle, V, 16)
    assert P == 0.0 and not q.any()


def _levels_c2(V, levels):
    P = oracle.percentile_nonzero(V)
    Q = oracle.quantize(V, levels, P).astype(np.float64)   # field-major levels
    return oracle.c2_packed(oracle.to_vector_major(Q))


@pytest.mark.parametrize("nv,nf,levels", [(2, 1, 16), (3, 7, 16), (100, 128, 16), (255, 200, 16),
                                          (256, 129, 16), (257, 64, 5), (600, 300, 16), (513, 77, 2)])
def test_thermo_2way_bit_exact(ps, handle, nv, nf, levels):
    V = synth.zero_inflated(nv, nf, synth.seed_for(2, 7 * nv + nf))
    ref = _levels_c2(V, levels)
    got = metrics_2way(ps, handle, V, path=ps.PS_PATH_THERMO, levels=levels)
    np.testing.assert_array_equal(got, ref.astype(np.float32))
    got64 = metrics_2way(ps, handle, V, path=ps.PS_PATH_THERMO, levels=levels, out_dtype=np.float64)
    np.testing.assert_array_equal(got64, ref)


def test_thermo_integer_input_equals_fp32_path(ps, handle):
    # integer data already on levels 0..15 with max 15 at the percentile:
    # the quantizer is the identity and both paths give the same numbers
    V = synth.integer_levels(700, 900, synth.seed_for(2, 3))
    V[0, 0] = 15.0
    P = oracle.percentile_nonzero(V)
    if P != 15.0:
        pytest.skip("percentile is not the top level for this draw")
    got_t = metrics_2way(ps, handle, V, path=ps.PS_PATH_THERMO, levels=16)
    got_f = metrics_2way(ps, handle, V, path=ps.PS_PATH_FP32)
    np.testing.assert_array_equal(got_t, got_f)


def test_thermo_config2_full_size_sampled(ps, handle):
    """32768 x 8192, L=16: sampled pairs bit-exact against the oracle on the
    quantized levels; quantization error against the FP64 oracle on the
    original values reported."""
    import torch
    nv, nf, L = 32768, 8192, 16
    V = synth.zero_inflated(nv, nf, synth.seed_for(2))
    X = torch.from_numpy(V).cuda()
    out = torch.empty(nv * (nv - 1) // 2, dtype=torch.float32, device="cuda")
    m = ps.matrix(X)
    ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), ps.PS_PATH_THERMO, L, out.data_ptr(), 0,
                                torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    pairs = synth.sample_pairs(nv, 20000, seed=5)
    pairs = np.concatenate([pairs, [[0, 1], [127, 128], [255, 256], [0, nv - 1], [nv - 2, nv - 1]]])
    got = out[torch.from_numpy(oracle.pair_index(nv, pairs[:, 0], pairs[:, 1])).cuda()].cpu().numpy()
    P = oracle.percentile_nonzero(V)
    cols = np.unique(pairs)
    remap = {v: t for t, v in enumerate(cols)}
    rp = np.vectorize(remap.get)(pairs)
    Q = oracle.quantize(np.ascontiguousarray(V[:, cols]), L, P).astype(np.float64)
    ref = oracle.c2_pairs(oracle.to_vector_major(Q), rp)
    np.testing.assert_array_equal(got, ref.astype(np.float32))
    orig = oracle.c2_pairs(oracle.to_vector_major(V[:, cols]), rp)
    err = np.abs(got.astype(np.float64) - orig)
    print(f"quantization error vs FP64 oracle: max {err.max():.4f} mean {err.mean():.5f} "
          f"p99 {np.percentile(err, 99):.4f}")


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("sync_kb", [0, 1, 7])
def test_thermo_multi_round_producer_sync(ps, handle, sync_kb, tile_m):
    # 20 x 20 tile blocks of 256 -> 210 tiles over 152 persistent CTAs (two
    # rounds); 30 k-blocks per tile; the producers meet every sync_kb
    # k-blocks (0: never, 7: a ragged last chunk).  Results stay bit-exact.
    # (tile_m: the 128 x 256 tile with two accumulators, or the 256 x 256 tile)
    h = ps.Handle(0, thermo_meet_kb=sync_kb if sync_kb else -1, thermo_tile_m=tile_m)
    try:
        nv, nf, L = 5000, 200, 16
        V = synth.zero_inflated(nv, nf, synth.seed_for(2, 90))
        ref = _levels_c2(V, L)
        got = metrics_2way(ps, h, V, path=ps.PS_PATH_THERMO, levels=L)
        np.testing.assert_array_equal(got, ref.astype(np.float32))
    finally:
        h.close()


def test_thermo_u8_codes_bit_exact(ps, handle):
    # one-byte codes of the quantized-level metric: the FP32 metric is exact
    # on both sides, so the codes match bit for bit
    V = synth.zero_inflated(600, 300, synth.seed_for(2, 91))
    ref = _levels_c2(V, 16)
    got = metrics_2way(ps, handle, V, path=ps.PS_PATH_THERMO, levels=16, out_dtype=np.uint8)
    np.testing.assert_array_equal(got, oracle.metric_code(ref))
