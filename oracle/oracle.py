"""ctypes wrapper around ps_oracle.c, the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg may import this module.  It shares no code
with the CUDA library.

Arrays passed in are vector-major (vector i is row i); helpers accept the
library's field-major layout through ``to_vector_major``.

Paper references (arXiv 1705.08210): Section 2.1 (2-way metric c2),
Section 2.2 eq. (1) (3-way metric c3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libps_oracle.so")

__all__ = [
    "build_oracle", "num_threads", "set_num_threads", "vector_sums", "n2",
    "n3prime", "n2_packed", "c2_packed", "c2_pairs", "c3_triples",
    "n3prime_triples", "slab_size", "c3_slab", "threshold_3way",
    "percentile_nonzero", "quantize", "pair_index", "to_vector_major",
    "metric_code", "threshold_2way",
]

_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ps_oracle.c with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_oracle())
    d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_vector_sums.argtypes = [p, i64, i64, p]
    lib.oracle_n2.argtypes = [p, i64, i64, i64]
    lib.oracle_n2.restype = d
    lib.oracle_n3prime.argtypes = [p, i64, i64, i64, i64]
    lib.oracle_n3prime.restype = d
    lib.oracle_n2_packed.argtypes = [p, i64, i64, p]
    lib.oracle_c2_packed.argtypes = [p, i64, i64, p]
    lib.oracle_c2_pairs.argtypes = [p, i64, i64, p, i64, p]
    lib.oracle_c3_triples.argtypes = [p, i64, i64, p, i64, p]
    lib.oracle_n3prime_triples.argtypes = [p, i64, p, i64, p]
    lib.oracle_slab_size.argtypes = [i64, i64, i64]
    lib.oracle_slab_size.restype = i64
    lib.oracle_c3_slab.argtypes = [p, i64, i64, i64, i64, p]
    lib.oracle_threshold_3way.argtypes = [p, i64, i64, d, p, p, i64]
    lib.oracle_threshold_3way.restype = i64
    lib.oracle_percentile_nonzero.argtypes = [p, i64, d]
    lib.oracle_percentile_nonzero.restype = ctypes.c_float
    lib.oracle_quantize.argtypes = [p, i64, ctypes.c_int, ctypes.c_float, p]
    _lib = lib
    return lib


def _f64(V):
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim != 2:
        raise ValueError("V must be 2-D (nv, nf), vector-major")
    return V


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def to_vector_major(V_field_major: np.ndarray) -> np.ndarray:
    """(nf, nv) field-major array -> (nv, nf) vector-major float64 copy."""
    return np.ascontiguousarray(np.asarray(V_field_major, dtype=np.float64).T)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def pair_index(nv: int, i, j):
    """Packed strict-upper-triangle position of pair (i, j), i < j."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (2 * nv - i - 1) // 2 + (j - i - 1)


def vector_sums(V) -> np.ndarray:
    """Section 2.1: S_i = sum_q v_iq."""
    V = _f64(V)
    S = np.empty(V.shape[0], dtype=np.float64)
    _load().oracle_vector_sums(_ptr(V), V.shape[0], V.shape[1], _ptr(S))
    return S


def n2(V, i: int, j: int) -> float:
    V = _f64(V)
    return float(_load().oracle_n2(_ptr(V), V.shape[1], int(i), int(j)))


def n3prime(V, i: int, j: int, k: int) -> float:
    V = _f64(V)
    return float(_load().oracle_n3prime(_ptr(V), V.shape[1], int(i), int(j), int(k)))


def n2_packed(V) -> np.ndarray:
    V = _f64(V)
    nv, nf = V.shape
    out = np.empty(nv * (nv - 1) // 2, dtype=np.float64)
    _load().oracle_n2_packed(_ptr(V), nv, nf, _ptr(out))
    return out


def c2_packed(V) -> np.ndarray:
    """All c2 (Section 2.1) for i<j, packed strict upper triangle, row-major."""
    V = _f64(V)
    nv, nf = V.shape
    out = np.empty(nv * (nv - 1) // 2, dtype=np.float64)
    _load().oracle_c2_packed(_ptr(V), nv, nf, _ptr(out))
    return out


def c2_pairs(V, pairs) -> np.ndarray:
    V = _f64(V)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.empty(pairs.shape[0], dtype=np.float64)
    _load().oracle_c2_pairs(_ptr(V), V.shape[0], V.shape[1], _ptr(pairs), pairs.shape[0], _ptr(out))
    return out


def c3_triples(V, triples) -> np.ndarray:
    """c3 (Section 2.2, eq. (1)) for an explicit list of (i, j, k)."""
    V = _f64(V)
    t = np.ascontiguousarray(triples, dtype=np.int64).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    _load().oracle_c3_triples(_ptr(V), V.shape[0], V.shape[1], _ptr(t), t.shape[0], _ptr(out))
    return out


def n3prime_triples(V, triples) -> np.ndarray:
    V = _f64(V)
    t = np.ascontiguousarray(triples, dtype=np.int64).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    _load().oracle_n3prime_triples(_ptr(V), V.shape[1], _ptr(t), t.shape[0], _ptr(out))
    return out


def slab_size(nv: int, j_begin: int, j_end: int) -> int:
    return int(_load().oracle_slab_size(int(nv), int(j_begin), int(j_end)))


def c3_slab(V, j_begin: int, j_end: int) -> np.ndarray:
    """All c3 with pivot j in [j_begin, j_end), pivot-slab order."""
    V = _f64(V)
    nv, nf = V.shape
    out = np.empty(slab_size(nv, j_begin, j_end), dtype=np.float64)
    _load().oracle_c3_slab(_ptr(V), nv, nf, int(j_begin), int(j_end), _ptr(out))
    return out


def threshold_3way(V, tau: float, capacity: int | None = None):
    """All (i, j, k, c3) with c3 >= tau in lexicographic order.

    Returns (ijk[count_written, 3] int32, values float64, total_count)."""
    V = _f64(V)
    nv, nf = V.shape
    if capacity is None:
        capacity = max(1, nv * (nv - 1) * (nv - 2) // 6)
    ijk = np.empty((capacity, 3), dtype=np.int32)
    val = np.empty(capacity, dtype=np.float64)
    total = int(_load().oracle_threshold_3way(_ptr(V), nv, nf, float(tau), _ptr(ijk), _ptr(val), capacity))
    w = min(total, capacity)
    return ijk[:w].copy(), val[:w].copy(), total


def percentile_nonzero(x, p: float = 0.999) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    return float(_load().oracle_percentile_nonzero(_ptr(x), x.size, float(p)))


def quantize(x, levels: int, P: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.empty(x.shape, dtype=np.int32)
    _load().oracle_quantize(_ptr(x), x.size, int(levels), ctypes.c_float(P), _ptr(q))
    return q


def metric_code(c) -> np.ndarray:
    """One-byte code of metric values (Section 6.8, the realistic sample
    problem: every metric is written as one unsigned byte holding about 2.5
    significant figures; the paper gives no formula).  Reading: the linear
    code rint(255 c), round half to even, with the decision taken in FP32 on
    the FP32-rounded metric (the precision the kernels decide in); codes above
    255 clamp to 255.  Decoding code / 255 is within 1/510 of c in [0, 1]."""
    c32 = np.asarray(c, dtype=np.float64).astype(np.float32)
    q = np.rint(np.float32(255.0) * c32)
    return np.minimum(q, np.float32(255.0)).astype(np.uint8)


def threshold_2way(V, tau: float):
    """Every pair i < j with c2 >= tau (inclusive), sorted by (i, j): the
    plain definition over c2_packed.  Returns (pairs[n, 2], values[n])."""
    V = _f64(V)
    nv = V.shape[0]
    c = c2_packed(V)
    ii, jj = np.triu_indices(nv, 1)  # row-major strict upper triangle = packed order
    keep = c >= tau
    return np.stack([ii[keep], jj[keep]], axis=1).astype(np.int64), c[keep]
