"""Thin ctypes binding of libps.so (include/ps.h); argument marshalling only.

Every computation runs in the CUDA library.  Importing this module loads
``_build/libps.so`` and raises ``ImportError`` if it has not been built
(``python -m paper_1705_08210_gb300.build_lib``) -- there is no fallback.

Function names follow the C ABI.  ``ps_*`` functions take raw integers /
pointers exactly like the C calls; ``matrix()`` builds a ``ps_matrix`` from a
torch tensor or numpy array, and ``check()`` turns a status into an
exception.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libps.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libps.so not built at {LIB_PATH}; run paper_1705_08210_gb300.build_lib.build()")

_lib = ctypes.CDLL(LIB_PATH)

PS_OK, PS_ERR_INVALID_ARG, PS_ERR_OOM, PS_ERR_CUDA, PS_ERR_CAPACITY, PS_ERR_TIMEOUT, PS_ERR_UNSUPPORTED = range(7)
PS_F32, PS_F64, PS_U8, PS_B1 = 0, 1, 2, 3  # PS_U8: one-byte codes (output); PS_B1: bit-packed 0/1 input
PS_PATH_FP32, PS_PATH_FP64, PS_PATH_THERMO, PS_PATH_HALF2 = 0, 1, 2, 3
PS_LAYOUT_FIELD_MAJOR, PS_LAYOUT_VECTOR_MAJOR = 0, 1


class ps_matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("nv", ctypes.c_int64), ("nf", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32)]


class ps_config(ctypes.Structure):
    """Handle configuration (include/ps.h); 0 = automatic in every kernel-choice field."""
    _fields_ = [("precision", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("wait_limit_ns", ctypes.c_int64), ("autotune_cache", ctypes.c_char_p),
                ("mgemm_feed", ctypes.c_int32), ("mgemm3_feed", ctypes.c_int32),
                ("mgemm_tile", ctypes.c_int32), ("mgemm_warps", ctypes.c_int32),
                ("mgemm_unroll", ctypes.c_int32), ("mgemm_add", ctypes.c_int32),
                ("mgemm_band", ctypes.c_int32), ("tma_slice", ctypes.c_int32),
                ("tma_unroll", ctypes.c_int32), ("tma_stages", ctypes.c_int32),
                ("tma_schedule", ctypes.c_int32), ("tma_meet", ctypes.c_int32),
                ("mgemm3_schedule", ctypes.c_int32), ("thermo_tile_m", ctypes.c_int32),
                ("thermo_meet_kb", ctypes.c_int32), ("test_batched_stall", ctypes.c_int32),
                ("mgemm_narrow", ctypes.c_int32), ("tma_lookahead", ctypes.c_int32),
                ("host_direct", ctypes.c_int32)]


class ps_problem(ctypes.Structure):
    _fields_ = [("V", ps_matrix), ("way", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("out", ctypes.c_void_p)]


PS_BATCH_PERSISTENT, PS_BATCH_PER_INSTANCE = 0, 1


class ps_pair(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("value", ctypes.c_float)]


class ps_triple(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("k", ctypes.c_int32),
                ("value", ctypes.c_float)]


_h = ctypes.c_void_p
_p = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64
_M = ctypes.POINTER(ps_matrix)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


ps_config_init = _sig("ps_config_init", None, [ctypes.POINTER(ps_config)])
ps_create = _sig("ps_create", ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.POINTER(ps_config)])
ps_get_config = _sig("ps_get_config", ctypes.c_int, [_h, ctypes.POINTER(ps_config)])
ps_set_config = _sig("ps_set_config", ctypes.c_int, [_h, ctypes.POINTER(ps_config)])
ps_destroy = _sig("ps_destroy", ctypes.c_int, [_h])
ps_status_string = _sig("ps_status_string", ctypes.c_char_p, [ctypes.c_int])
ps_last_error = _sig("ps_last_error", ctypes.c_char_p, [_h])
ps_version = _sig("ps_version", ctypes.c_char_p, [])
ps_vector_sums = _sig("ps_vector_sums", ctypes.c_int, [_h, _M, _p, _p])
ps_metrics_2way = _sig("ps_metrics_2way", ctypes.c_int, [_h, _M, _i32, _i32, _p, _i32, _p])
ps_slab_size = _sig("ps_slab_size", _i64, [_i64, _i64, _i64])
ps_metrics_3way = _sig("ps_metrics_3way", ctypes.c_int, [_h, _M, _i64, _i64, _p, _p])
ps_threshold_3way = _sig("ps_threshold_3way", ctypes.c_int,
                         [_h, _M, ctypes.c_float, _i32, _p, _i64, _p, _p])
ps_threshold_2way = _sig("ps_threshold_2way", ctypes.c_int, [_h, _M, ctypes.c_float, _p, _i64, _p, _p])
ps_quantize = _sig("ps_quantize", ctypes.c_int, [_h, _M, _i32, _p, _p, _p])
ps_timing_enable = _sig("ps_timing_enable", ctypes.c_int, [_h, _i32])
ps_timing_read = _sig("ps_timing_read", ctypes.c_int,
                      [_h, ctypes.c_char_p, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)])
ps_metrics_batched = _sig("ps_metrics_batched", ctypes.c_int,
                          [_h, ctypes.POINTER(ps_problem), _i32, _i32, _p])
ps_autotune_batched = _sig("ps_autotune_batched", ctypes.c_int,
                           [_h, ctypes.POINTER(ps_problem), _i32, ctypes.c_char_p, ctypes.c_char_p, _i32, _p])
ps_proposal_init = _sig("ps_proposal_init", ctypes.c_int, [_h, _i32, ctypes.c_uint64])
ps_proposal_param_count = _sig("ps_proposal_param_count", _i64, [_h])
ps_proposal_params = _sig("ps_proposal_params", ctypes.c_int, [_h, _i32, _p, _i64, _p])
ps_proposal_pair_grad = _sig("ps_proposal_pair_grad", ctypes.c_int, [_h, _M, _p, _p, _i64, _p, _p, _p, _p])
ps_proposal_train = _sig("ps_proposal_train", ctypes.c_int,
                         [_h, _M, _i32, ctypes.c_float, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                          _p, _p])
ps_proposal_last_stats = _sig("ps_proposal_last_stats", ctypes.c_int,
                              [_h, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)])
ps_partition = _sig("ps_partition", ctypes.c_int,
                    [_i64, _i32, _i32, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                     ctypes.POINTER(_i64)])
ps_metrics_2way_part = _sig("ps_metrics_2way_part", ctypes.c_int, [_h, _M, _i32, _i32, _p, _i32, _p])
ps_metrics_2way_static = _sig("ps_metrics_2way_static", ctypes.c_int, [_M, _p, _i32, _p])
ps_probe_minadd_peak = _sig("ps_probe_minadd_peak", ctypes.c_int,
                            [_h, _i32, ctypes.POINTER(ctypes.c_double)])

EXPORTED = [n for n in globals() if n.startswith("ps_") and callable(globals()[n])
            and n not in ("ps_matrix", "ps_pair", "ps_triple", "ps_problem", "ps_config")]


class PSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{ps_status_string(status).decode()}: {msg}")
        self.status = status


def check(status: int, handle=None) -> int:
    if status != PS_OK:
        raise PSError(status, ps_last_error(handle).decode(errors="replace"))
    return status


def config(**fields) -> ps_config:
    """ps_config with the library defaults, then the given fields set
    (autotune_cache may be a str)."""
    c = ps_config()
    ps_config_init(ctypes.byref(c))
    names = {f[0] for f in ps_config._fields_}
    for k, v in fields.items():
        if k not in names:
            raise ValueError(f"ps_config has no field {k!r}")
        if k == "autotune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(c, k, v)
    return c


class Handle:
    """Owns a ps_handle for one CUDA device; keyword arguments are ps_config
    fields (the rest keep their defaults)."""

    def __init__(self, device: int = 0, cfg: ps_config | None = None, **fields):
        self.h = _h()
        if cfg is None:
            cfg = config(**fields)
        self._cfg = cfg  # keeps autotune_cache's bytes alive for the call
        check(ps_create(ctypes.byref(self.h), int(device), ctypes.byref(cfg)))

    def get_config(self) -> ps_config:
        c = ps_config()
        check(ps_get_config(self.h, ctypes.byref(c)), self.h)
        return c

    def set_config(self, **fields) -> None:
        """Change the given ps_config fields of this handle."""
        c = self.get_config()
        for k, v in fields.items():
            if k == "autotune_cache" and isinstance(v, str):
                v = v.encode()
            setattr(c, k, v)
        self._cfg = c
        check(ps_set_config(self.h, ctypes.byref(c)), self.h)

    def close(self):
        if self.h:
            ps_destroy(self.h)
            self.h = _h()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _ptr_of(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    return int(x)


def _dtype_of(x) -> int:
    name = str(x.dtype)
    if "float32" in name:
        return PS_F32
    if "float64" in name:
        return PS_F64
    raise TypeError(f"unsupported dtype {name}")


def matrix(X, layout: int = PS_LAYOUT_FIELD_MAJOR) -> ps_matrix:
    """ps_matrix for a 2-D array.

    layout FIELD_MAJOR: X has shape (nf, nv) (row q = field q of every vector);
    layout VECTOR_MAJOR: X has shape (nv, nf).  Rows may be padded (stride)."""
    if X.ndim != 2:
        raise ValueError("matrix must be 2-D")
    if hasattr(X, "stride") and callable(X.stride):
        s0, s1 = X.stride()
    else:
        s0, s1 = (st // X.itemsize for st in X.strides)
    rows, cols = X.shape
    if rows * cols == 0 or rows == 1:
        s0, s1 = cols, 1  # strides of empty / single-row arrays carry no layout
    if s1 != 1 and cols > 1:
        raise ValueError("inner dimension must be contiguous")
    if layout == PS_LAYOUT_FIELD_MAJOR:
        nf, nv = X.shape
    else:
        nv, nf = X.shape
    return ps_matrix(_ptr_of(X), nv, nf, max(int(s0), cols, 1), _dtype_of(X), layout)


def bit_matrix(words, nf: int) -> ps_matrix:
    """ps_matrix (PS_B1) for bit-packed 0/1 vectors: `words` is an (nv, ld)
    uint32 array (torch or numpy), field q of vector i in bit q % 32 of
    word [i, q // 32]."""
    if hasattr(words, "stride") and callable(words.stride):
        ld = words.stride()[0]
    else:
        ld = words.strides[0] // 4
    nv = words.shape[0]
    return ps_matrix(_ptr_of(words), nv, int(nf), max(int(ld), 1), PS_B1, PS_LAYOUT_VECTOR_MAJOR)


def stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)
