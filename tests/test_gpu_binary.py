"""Bit-packed 0/1 input (PS_B1, Section 2.3's Sorenson case).  With
PS_PATH_THERMO the bits are the tensor-core operand; other paths unpack them.
The data are integers, so every result is bit-exact against the oracle on the
same 0/1 values."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth

pytestmark = pytest.mark.gpu


def _run2(ps, handle, words, nf, path, out_dtype=np.float32, on_host=False):
    import torch
    nv = words.shape[0]
    n = nv * (nv - 1) // 2
    code = {np.float32: ps.PS_F32, np.float64: ps.PS_F64, np.uint8: ps.PS_U8}[out_dtype]
    if on_host:
        W = np.ascontiguousarray(words)
        out = np.empty(n, dtype=out_dtype)
        m = ps.bit_matrix(W, nf)
        ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), path, 0, out.ctypes.data, code, 0), handle.h)
        return out
    W = torch.from_numpy(words.view(np.int32)).cuda()
    tdt = {np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8}[out_dtype]
    out = torch.empty(n, dtype=tdt, device="cuda")
    m = ps.bit_matrix(W, nf)
    ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), path, 0, out.data_ptr(), code,
                                torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nv,nf,ld", [(2, 1, None), (3, 31, None), (130, 32, None), (257, 100, 7),
                                      (600, 1000, None), (5000, 700, 40)])
def test_b1_tensor_path_bit_exact(ps, handle, nv, nf, ld):
    dense, words = synth.binary_bits(nv, nf, synth.seed_for(7, nv + nf), ld_words=ld)
    ref = oracle.c2_packed(oracle.to_vector_major(dense))
    got = _run2(ps, handle, words, nf, ps.PS_PATH_THERMO)
    np.testing.assert_array_equal(got, ref.astype(np.float32))
    if nv <= 600:
        np.testing.assert_array_equal(_run2(ps, handle, words, nf, ps.PS_PATH_THERMO, np.float64), ref)
        np.testing.assert_array_equal(_run2(ps, handle, words, nf, ps.PS_PATH_THERMO, np.uint8),
                                      oracle.metric_code(ref))


def test_b1_unpacked_paths_and_host_input(ps, handle):
    nv, nf = 300, 77
    dense, words = synth.binary_bits(nv, nf, synth.seed_for(7, 1), ld_words=4)
    ref = oracle.c2_packed(oracle.to_vector_major(dense))
    for path in (ps.PS_PATH_FP32, ps.PS_PATH_FP64, ps.PS_PATH_HALF2):
        np.testing.assert_array_equal(_run2(ps, handle, words, nf, path), ref.astype(np.float32))
    np.testing.assert_array_equal(_run2(ps, handle, words, nf, ps.PS_PATH_THERMO, on_host=True),
                                  ref.astype(np.float32))


def test_b1_3way_and_threshold(ps, handle):
    import torch
    nv, nf = 120, 45
    dense, words = synth.binary_bits(nv, nf, synth.seed_for(7, 2), p_one=0.4)
    Vv = oracle.to_vector_major(dense)
    W = torch.from_numpy(words.view(np.int32)).cuda()
    m = ps.bit_matrix(W, nf)
    n = ps.ps_slab_size(nv, 0, nv)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ps.check(ps.ps_metrics_3way(handle.h, ctypes.byref(m), 0, nv, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.c3_slab(Vv, 0, nv).astype(np.float32))
    rp, rv = oracle.threshold_2way(Vv, 0.5)
    res = (ps.ps_pair * max(len(rp), 1))()
    cnt = ctypes.c_int64(-1)
    ps.check(ps.ps_threshold_2way(handle.h, ctypes.byref(m), 0.5, ctypes.addressof(res), len(rp),
                                  ctypes.addressof(cnt), 0), handle.h)
    assert cnt.value == len(rp)
    raw = np.frombuffer(res, dtype=np.int32).reshape(-1, 3)[:len(rp)]
    np.testing.assert_array_equal(raw[:, :2], rp)


def test_b1_invalid_descriptors(ps, handle):
    nv, nf = 10, 70
    _, words = synth.binary_bits(nv, nf, synth.seed_for(7, 3))
    out = np.empty(nv * (nv - 1) // 2, dtype=np.float32)
    m = ps.bit_matrix(np.ascontiguousarray(words), nf)
    bad = ps.ps_matrix(m.data, nv, nf, m.ld, ps.PS_B1, ps.PS_LAYOUT_FIELD_MAJOR)
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(bad), ps.PS_PATH_THERMO, 0, out.ctypes.data,
                              ps.PS_F32, 0) == ps.PS_ERR_INVALID_ARG
    bad = ps.ps_matrix(m.data, nv, nf, 2, ps.PS_B1, ps.PS_LAYOUT_VECTOR_MAJOR)  # ld < ceil(70/32)
    assert ps.ps_metrics_2way(handle.h, ctypes.byref(bad), ps.PS_PATH_THERMO, 0, out.ctypes.data,
                              ps.PS_F32, 0) == ps.PS_ERR_INVALID_ARG
