"""The packed half2 variant of the 2-way path (PS_PATH_HALF2): FP16-rounded
inputs (scaled by a power of two), packed min, FP32 compensated accumulation.
Error bound: the FP16 rounding of each input (2^-11 relative for scaled
values in the normal range) plus the FP32 bound of the other paths; 1e-3
relative is stated for zero-inflated data; integer data are exact."""
import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel, metrics_2way

pytestmark = pytest.mark.gpu
RTOL_HALF = 1e-3


@pytest.mark.parametrize("nv,nf", [(2, 1), (5, 3), (129, 17), (300, 1000), (1100, 333)])
def test_half2_close_to_oracle(ps, handle, nv, nf):
    V = synth.zero_inflated(nv, nf, synth.seed_for(2, 50 + nv + nf))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V, path=ps.PS_PATH_HALF2)
    err = assert_rel(got, ref, RTOL_HALF, f"half2 nv={nv} nf={nf}")
    print(f"half2 nv={nv} nf={nf}: max rel err {err:.2e}")


def test_half2_integer_data_bit_exact(ps, handle):
    V = synth.integer_levels(600, 1501, synth.seed_for(2, 60))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, path=ps.PS_PATH_HALF2), ref.astype(np.float32))
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, path=ps.PS_PATH_HALF2, out_dtype=np.float64), ref)


@pytest.mark.parametrize("warps", [8, 16])
def test_half2_tile_warps(ps, warps):
    # both tile configurations of the half2 kernel (8 x 8 or 8 x 4 outputs
    # per lane) give the same values
    h = ps.Handle(0, mgemm_warps=warps)
    try:
        V = synth.zero_inflated(700, 333, synth.seed_for(2, 70))
        ref = oracle.c2_packed(oracle.to_vector_major(V))
        assert_rel(metrics_2way(ps, h, V, path=ps.PS_PATH_HALF2), ref, RTOL_HALF, f"half2 warps={warps}")
    finally:
        h.close()
