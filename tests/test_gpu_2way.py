"""GPU parity of the 2-way path (Section 2.1, Section 3.1) against the oracle.

Tolerance: FP32 paths 1e-5 relative (the accumulation carries at most 64
roundings of a 64-term partial sum, 64 * 2^-24 = 3.8e-6, plus the FP32
rounding of the operands and of the ratio); the FP64 path 1e-12; integer
data bit-exact."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth
from gpu_run import assert_rel, metrics_2way

pytestmark = pytest.mark.gpu
RTOL32 = 1e-5


def test_config1_all_pairs_fp32_path(ps, handle):
    # 1024 x 512 FP64, packed FP64 output, FP32 min/add numerators
    V = synth.zero_inflated(1024, 512, synth.seed_for(1), dtype=np.float64)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V, path=ps.PS_PATH_FP32, out_dtype=np.float64)
    err = assert_rel(got, ref, RTOL32, "config1 fp32 path")
    print(f"config1 fp32 path max rel err {err:.3e}")


def test_config1_all_pairs_fp64_path(ps, handle):
    V = synth.zero_inflated(1024, 512, synth.seed_for(1), dtype=np.float64)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V, path=ps.PS_PATH_FP64, out_dtype=np.float64)
    assert_rel(got, ref, 1e-12, "config1 fp64 path")


@pytest.mark.parametrize("nv", [2, 3, 5, 127, 128, 129, 300])
@pytest.mark.parametrize("nf", [0, 1, 15, 17, 100, 1000])
def test_ragged_shapes(ps, handle, nv, nf):
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, nv * 7 + nf), dtype=np.float32)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V)
    assert_rel(got, ref, RTOL32, f"nv={nv} nf={nf}")


@pytest.mark.parametrize("nv,nf", [(1500, 40), (700, 3000)])
def test_integer_data_bit_exact(ps, handle, nv, nf):
    # n_f = 40 takes the small-n_f kernel with the branch-free division
    V = synth.integer_levels(nv, nf, synth.seed_for(1, 99))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got32 = metrics_2way(ps, handle, V)
    np.testing.assert_array_equal(got32, ref.astype(np.float32))
    got64 = metrics_2way(ps, handle, V, out_dtype=np.float64)
    np.testing.assert_array_equal(got64, ref)
    got64p = metrics_2way(ps, handle, V, path=ps.PS_PATH_FP64, out_dtype=np.float64)
    np.testing.assert_array_equal(got64p, ref)


def test_all_zero_vectors_and_duplicates(ps, handle):
    V = synth.zero_inflated(200, 64, synth.seed_for(1, 5))
    V[:, 3] = 0.0          # all-zero vector
    V[:, 4] = 0.0
    V[:, 10] = V[:, 11]    # duplicate pair
    got = metrics_2way(ps, handle, V, out_dtype=np.float64)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    assert got[oracle.pair_index(200, 3, 4)] == 0.0
    assert_rel(got, ref, RTOL32, "zeros/duplicates")
    assert abs(got[oracle.pair_index(200, 10, 11)] - 1.0) < 1e-6


def test_layouts_strides_and_host_buffers(ps, handle):
    nv, nf = 333, 257
    V32 = synth.zero_inflated(nv, nf, synth.seed_for(1, 6))
    base = metrics_2way(ps, handle, V32)
    ref = oracle.c2_packed(oracle.to_vector_major(V32))
    assert_rel(base, ref, RTOL32, "base")
    # vector-major copy of the same data
    np.testing.assert_array_equal(metrics_2way(ps, handle, np.ascontiguousarray(V32.T), layout=1), base)
    # padded leading dimension with NaN garbage in the padding
    P = np.full((nf, nv + 13), np.nan, dtype=np.float32)
    P[:, :nv] = V32
    np.testing.assert_array_equal(metrics_2way(ps, handle, P[:, :nv]), base)
    # host (pageable numpy) input and output
    np.testing.assert_array_equal(metrics_2way(ps, handle, V32, on_host=True), base)
    # FP64 input rounded to the same FP32 values gives the same numerators
    got64 = metrics_2way(ps, handle, V32.astype(np.float64), out_dtype=np.float64)
    assert_rel(got64, ref, RTOL32, "f64 input")


def test_invalid_arguments(ps, handle):
    import torch
    X = torch.zeros(4, 10, device="cuda")
    out = torch.zeros(100, device="cuda")
    m = ps.matrix(X)
    st = 0
    bad = ps.ps_matrix(m.data, 1, 4, 10, 0, 0)  # nv = 1
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(bad), 0, 0, out.data_ptr(), 0, st) == ps.PS_ERR_INVALID_ARG
    bad = ps.ps_matrix(m.data, 10, 4, 5, 0, 0)  # ld < nv
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(bad), 0, 0, out.data_ptr(), 0, st) == ps.PS_ERR_INVALID_ARG
    bad = ps.ps_matrix(m.data, 10, 4, 10, 0, 7)  # layout
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(bad), 0, 0, out.data_ptr(), 0, st) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(m), 0, 0, None, 0, st) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(m), 9, 0, out.data_ptr(), 0, st) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(m), 2, 1, out.data_ptr(), 0, st) == ps.PS_ERR_INVALID_ARG
    assert b"levels" in ps.ps_last_error(handle.h)


def test_config2_full_size_sampled(ps, handle):
    """32768 x 8192 FP32 in the benchmark's launch configuration; 20000 sampled
    pairs against the oracle, all values in [0, 1]."""
    import torch
    nv, nf = 32768, 8192
    V = synth.zero_inflated(nv, nf, synth.seed_for(2))
    X = torch.from_numpy(V).cuda()
    out = torch.empty(nv * (nv - 1) // 2, dtype=torch.float32, device="cuda")
    m = ps.matrix(X)
    ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), 0, 0, out.data_ptr(), 0,
                                torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    assert float(out.min()) >= 0.0 and float(out.max()) <= 1.0
    pairs = synth.sample_pairs(nv, 20000, seed=7)
    # include tile corners and the last pair
    pairs = np.concatenate([pairs, [[0, 1], [127, 128], [0, nv - 1], [nv - 2, nv - 1], [128, 255]]])
    idx = torch.from_numpy(oracle.pair_index(nv, pairs[:, 0], pairs[:, 1])).cuda()
    got = out[idx].cpu().numpy()
    Vv = np.ascontiguousarray(V[:, np.unique(pairs)].T).astype(np.float64)
    remap = {v: t for t, v in enumerate(np.unique(pairs))}
    rp = np.vectorize(remap.get)(pairs)
    ref = oracle.c2_pairs(Vv, rp)
    err = assert_rel(got, ref, RTOL32, "config2 sampled")
    print(f"config2 sampled max rel err {err:.3e}")


def test_parts_assemble_full_result(ps, handle):
    import torch
    nv, nf = 1000, 300
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 31))
    full = metrics_2way(ps, handle, V)
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    out = torch.full((nv * (nv - 1) // 2,), float("nan"), device="cuda")
    for p in range(3):
        ps.check(ps.ps_metrics_2way_part(handle.h, ctypes.byref(m), 3, p, out.data_ptr(), 0,
                                         torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), full)


def test_host_output_banded_path_matches_device(ps, handle):
    # nv >= 1024: the host-output call computes in row bands and overlaps
    # the device-to-host copies; results must equal the device-output call
    nv, nf = 1500, 120
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 41))
    dev = metrics_2way(ps, handle, V)
    host = metrics_2way(ps, handle, V, on_host=True)
    np.testing.assert_array_equal(host, dev)
    host64 = metrics_2way(ps, handle, V, on_host=True, out_dtype=np.float64)
    np.testing.assert_array_equal(host64, metrics_2way(ps, handle, V, out_dtype=np.float64))


@pytest.mark.parametrize("band", [1, 2, 3])
def test_tile_walk_bands(ps, handle, band):
    # the 2-way tile walk in bands of `band` tile rows (the default band is
    # wider than these small cases, so narrow bands exercise the diagonal
    # triangles, the column chunks and the ragged last band): every pair is
    # computed once, whole-matrix, by parts and through the host-output bands
    import torch
    h = ps.Handle(0, mgemm_band=band)
    try:
        nv, nf = 1300, 77
        V = synth.zero_inflated(nv, nf, synth.seed_for(1, 51 + band))
        ref = oracle.c2_packed(oracle.to_vector_major(V))
        got = metrics_2way(ps, h, V)
        assert_rel(got, ref, RTOL32, f"band {band}")
        np.testing.assert_array_equal(metrics_2way(ps, h, V, on_host=True), got)
        X = torch.from_numpy(V).cuda()
        m = ps.matrix(X)
        out = torch.full((nv * (nv - 1) // 2,), float("nan"), device="cuda")
        for p in range(3):
            ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), 3, p, out.data_ptr(), 0,
                                             torch.cuda.current_stream().cuda_stream), h.h)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), got)
        half = metrics_2way(ps, h, V, path=ps.PS_PATH_HALF2)
        assert_rel(half, ref, 1e-3, f"half2 band {band}")
    finally:
        h.close()


def test_u8_metric_codes(ps, handle):
    # one-byte codes (PS_U8): integer data bit-exact; general data equal to
    # the oracle's code except where 255*c2 lies within the FP32 tolerance of
    # a rounding boundary (there the two sides may differ by one)
    import torch
    V = synth.integer_levels(700, 301, synth.seed_for(1, 61))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, out_dtype=np.uint8), oracle.metric_code(ref))
    V = synth.zero_inflated(1100, 500, synth.seed_for(1, 62))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V, out_dtype=np.uint8).astype(np.int64)
    want = oracle.metric_code(ref).astype(np.int64)
    diff = got != want
    assert np.all(np.abs(got - want) <= 1)
    x = 255.0 * ref[diff]
    assert np.all(np.abs(x - np.floor(x) - 0.5) <= 255.0 * RTOL32 * ref[diff] + 1e-6), x
    print(f"u8 codes: {int(diff.sum())} of {diff.size} at a rounding boundary")
    # host output (row bands with overlapped copies) and parts give the same bytes
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, out_dtype=np.uint8, on_host=True), got)
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    out = torch.zeros(ref.size, dtype=torch.uint8, device="cuda")
    for p in range(3):
        ps.check(ps.ps_metrics_2way_part(handle.h, ctypes.byref(m), 3, p, out.data_ptr(), ps.PS_U8,
                                         torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), got)


def test_u8_rejected_on_other_paths(ps, handle):
    V = synth.zero_inflated(10, 5, synth.seed_for(1, 63))
    for path in (ps.PS_PATH_FP64, ps.PS_PATH_HALF2):
        with pytest.raises(ps.PSError):
            metrics_2way(ps, handle, V, path=path, out_dtype=np.uint8)


@pytest.mark.parametrize("nv,nf", [(129, 33), (300, 1000), (1300, 77), (700, 16), (4096, 64)])
def test_operand_feeds_bit_identical(ps, handle, nv, nf):
    # the TMA-fed kernel (16-, 32- and 64-field slices; tiles claimed from a
    # counter or assigned round-robin) and the cp.async kernel
    # run the same micro-kernel in the same order: every output bit-identical,
    # for FP32, FP64 and one-byte outputs, by parts, and in the 3-way n2 table
    import torch
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 71 + nv + nf))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    results = {}
    for feed, bk, dyn in (("cpasync", "16", "1"), ("tma", "16", "1"), ("tma", "32", "1"), ("tma", "64", "1"),
                          ("tma", "32", "0"), ("tma-packed-adds", "32", "1"), ("tma-scalar-adds", "32", "1"),
                          ("tma-lookahead1", "32", "1")):
        # dyn 0: static round-robin tiles; add forms other than the mixed
        # default (n_f > 256 only): all packed, all scalar; a producer one
        # slice ahead instead of three
        adds = {"tma-packed-adds": 1, "tma-scalar-adds": 2}.get(feed, 0)
        h = ps.Handle(0, mgemm_feed=2 if feed == "cpasync" else 1, tma_slice=int(bk),
                      tma_schedule=1 if dyn == "1" else 2, mgemm_add=adds,
                      tma_lookahead=1 if feed == "tma-lookahead1" else 0)
        try:
            r = [metrics_2way(ps, h, V), metrics_2way(ps, h, V, out_dtype=np.float64),
                 metrics_2way(ps, h, V, out_dtype=np.uint8)]
            X = torch.from_numpy(V).cuda()
            m = ps.matrix(X)
            out = torch.full((nv * (nv - 1) // 2,), float("nan"), device="cuda")
            for p in range(3):
                ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), 3, p, out.data_ptr(), 0,
                                                 torch.cuda.current_stream().cuda_stream), h.h)
            torch.cuda.synchronize()
            r.append(out.cpu().numpy())
            if nv <= 300:
                from gpu_run import metrics_3way
                r.append(metrics_3way(ps, h, V))
            results[(feed, bk, dyn)] = r
        finally:
            h.close()
    assert_rel(results[("tma", "16", "1")][0], ref, RTOL32, f"tma nv={nv} nf={nf}")
    base = results[("cpasync", "16", "1")]
    for key, r in results.items():
        for a, b in zip(r, base):
            np.testing.assert_array_equal(a, b, err_msg=str(key))


def test_tma_producer_meetings(ps, handle):
    # the TMA producers' grid-wide meetings (cooperative launch; off by
    # default) change no value: 210 tiles over 152 CTAs (two rounds, the
    # second partial), meetings every 2 slices, whole matrix and row bands
    import torch
    nv, nf = 2560, 200
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 91))
    base = metrics_2way(ps, handle, V)
    h = ps.Handle(0, tma_schedule=2, tma_meet=2)
    try:
        np.testing.assert_array_equal(metrics_2way(ps, h, V), base)
        np.testing.assert_array_equal(metrics_2way(ps, h, V, on_host=True), base)
        X = torch.from_numpy(V).cuda()
        m = ps.matrix(X)
        out = torch.full((nv * (nv - 1) // 2,), float("nan"), device="cuda")
        for p in range(3):
            ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), 3, p, out.data_ptr(), 0,
                                             torch.cuda.current_stream().cuda_stream), h.h)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), base)
    finally:
        h.close()


@pytest.mark.parametrize("scale", [1e-37, 1e36])
def test_fast_division_fallback_range(ps, handle, scale):
    # n_f <= 256 takes the branch-free division; denominators below 2^-120
    # or above 2^120 are outside its range, so the warps rewrite their
    # outputs with __fdiv_rn: same values as the oracle and, bit for bit, as
    # the cp.async kernel (which always divides with __fdiv_rn)
    V = (synth.zero_inflated(300, 40, synth.seed_for(1, 95)).astype(np.float64) * scale).astype(np.float32)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    got = metrics_2way(ps, handle, V)
    assert_rel(got, ref, RTOL32, f"scale {scale}")
    h = ps.Handle(0, mgemm_feed=2)
    try:
        np.testing.assert_array_equal(metrics_2way(ps, h, V), got)
    finally:
        h.close()


@pytest.mark.parametrize("case", ["zero_inflated", "integer", "wide_range", "tiny_fallback", "huge_fallback"])
@pytest.mark.parametrize("nf", [16, 64, 200])
def test_lean_division_bit_identical(ps, handle, case, nf):
    # the small-n_f epilogue (branch-free correctly rounded division, FP32
    # sums with 1.0 for all-zero vectors, one range check per call) against
    # the cp.async kernel, which divides with __fdiv_rn: every FP32 output
    # and one-byte code bit-identical.  Integer data give many quotients that
    # are powers of two; zero-inflated data at n_f = 16 many all-zero
    # vectors; the fallback cases fall outside the range (smallest value
    # below 2^-80, or sums above 2^100) and take __fdiv_rn everywhere.
    nv = 3000
    seed = synth.seed_for(1, 600 + nf)
    if case == "integer":
        V = synth.integer_levels(nv, nf, seed)
    else:
        V = synth.zero_inflated(nv, nf, seed)
        if case == "wide_range":
            rng = np.random.default_rng(seed)
            V = (V * np.exp(rng.uniform(-14.0, 14.0, size=(1, nv)))).astype(np.float32)
        elif case == "tiny_fallback":
            V = (V.astype(np.float64) * 2.0 ** -90).astype(np.float32)
        elif case == "huge_fallback":
            V = (V.astype(np.float64) * 2.0 ** 100).astype(np.float32)
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    lean32 = metrics_2way(ps, handle, V)
    lean8 = metrics_2way(ps, handle, V, out_dtype=np.uint8)
    if case == "integer":
        np.testing.assert_array_equal(lean32, ref.astype(np.float32))
    else:
        assert_rel(lean32, ref, RTOL32, f"lean {case} nf={nf}")
    h = ps.Handle(0, mgemm_feed=2)
    try:
        np.testing.assert_array_equal(metrics_2way(ps, h, V), lean32)
        np.testing.assert_array_equal(metrics_2way(ps, h, V, out_dtype=np.uint8), lean8)
    finally:
        h.close()


@pytest.mark.parametrize("nv,nf", [(129, 1), (1000, 7), (1300, 16), (257, 17), (1000, 32), (1300, 33), (640, 64),
                                   (2100, 16)])
def test_narrow_kernel_layouts_bit_identical(ps, nv, nf):
    # the n_f <= 64 kernel (each warp writes its previous tile's metrics
    # while it computes the next tile) against the general TMA kernel: FP32
    # metrics and one-byte codes bit-identical, FP32 within the rounding
    # bound of the FP64 oracle.  Ragged nv leaves partial tiles on the right
    # edge; nv = 2100 gives runs of interior tiles between diagonal ones.
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 700 + nf))
    ref = oracle.c2_packed(oracle.to_vector_major(V))
    outs = {}
    for key, fields in (("narrow", dict(mgemm_narrow=1)), ("general", dict(mgemm_narrow=2))):
        h = ps.Handle(0, **fields)
        try:
            outs[key] = (metrics_2way(ps, h, V), metrics_2way(ps, h, V, out_dtype=np.uint8))
        finally:
            h.close()
    assert_rel(outs["narrow"][0], ref, RTOL32, f"narrow nv={nv} nf={nf}")
    np.testing.assert_array_equal(outs["narrow"][0], outs["general"][0])
    np.testing.assert_array_equal(outs["narrow"][1], outs["general"][1])


@pytest.mark.parametrize("nv,nf,dt", [(1300, 300, np.float32), (1100, 256, np.uint8), (1024, 512, np.float64)])
def test_host_output_direct_and_staged_bit_identical(ps, nv, nf, dt):
    # a pinned host output at n_f >= 256 is written by the kernel through
    # its device mapping; host_direct=1 stages it and copies in row bands;
    # both equal the device-output call bit for bit
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 800 + nf))
    out_dtype = {np.float32: ps.PS_F32, np.uint8: ps.PS_U8, np.float64: ps.PS_F64}[dt]
    res = []
    for direct in (0, 1):
        h = ps.Handle(0, host_direct=direct)
        try:
            res.append(metrics_2way(ps, h, V, out_dtype=dt, on_host="pinned"))
            dev = metrics_2way(ps, h, V, out_dtype=dt)
        finally:
            h.close()
        np.testing.assert_array_equal(res[-1], dev)
    np.testing.assert_array_equal(res[0], res[1])
    if dt is not np.uint8:
        assert_rel(res[0], oracle.c2_packed(oracle.to_vector_major(V)), RTOL32, "host output")


@pytest.mark.parametrize("nv,nf", [(1300, 16), (2100, 40)])
def test_narrow_kernel_parts_and_bands(ps, handle, nv, nf):
    # the n_f <= 64 kernel over row ranges: the sharded parts and the row
    # bands of the host-output call assemble the whole-triangle result bit
    # for bit
    import torch
    V = synth.zero_inflated(nv, nf, synth.seed_for(1, 900 + nf))
    full = metrics_2way(ps, handle, V)
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    out = torch.full((nv * (nv - 1) // 2,), float("nan"), device="cuda")
    for p in range(3):
        ps.check(ps.ps_metrics_2way_part(handle.h, ctypes.byref(m), 3, p, out.data_ptr(), 0,
                                         torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), full)
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, on_host=True), full)
    np.testing.assert_array_equal(metrics_2way(ps, handle, V, on_host="pinned"), full)
