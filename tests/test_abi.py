"""The C-ABI library loads and exports every symbol include/ps.h declares.

Runs without a GPU: only host-side entry points are called."""
import ctypes
import os
import re

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ps_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["ps_create", "ps_destroy", "ps_metrics_2way", "ps_metrics_3way",
                     "ps_threshold_3way", "ps_vector_sums", "ps_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(ps):
    lib = ctypes.CDLL(ps.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(ps):
    assert set(declared_symbols()) <= set(ps.EXPORTED)


def test_status_strings(ps):
    for code in range(7):
        assert ps.ps_status_string(code).decode().startswith("PS_")
    assert ps.ps_status_string(99) == b"PS_ERR_UNKNOWN"


def test_slab_size_matches_oracle_count(ps):
    for nv in [3, 4, 10, 257]:
        for jb, je in [(0, nv), (1, nv // 2), (nv // 2, nv), (2, 2)]:
            assert ps.ps_slab_size(nv, jb, je) == oracle.slab_size(nv, jb, je)
    assert ps.ps_slab_size(10, 5, 3) == -1
    assert ps.ps_slab_size(10, 0, 11) == -1
    # closed form at a large size (no overflow)
    nv = 8192
    assert ps.ps_slab_size(nv, 0, nv) == nv * (nv - 1) * (nv - 2) // 6


def test_null_handle_is_rejected_without_gpu(ps):
    m = ps.ps_matrix(0, 10, 10, 10, 0, 0)
    assert ps.ps_metrics_2way(None, ctypes.byref(m), 0, 0, None, 0, None) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_metrics_3way(None, ctypes.byref(m), 0, 10, None, None) == ps.PS_ERR_INVALID_ARG
    assert ps.ps_last_error(None)


def test_version_string(ps):
    assert b"sm_103a" in ps.ps_version()


def test_config_defaults_and_validation_without_gpu(ps):
    # ps_config_init's defaults; ps_create checks the configuration before it
    # looks for a device, so every out-of-range field is rejected here
    c = ps.config()
    assert c.precision == ps.PS_PATH_FP32 and c.debug_checks == 0
    assert c.wait_limit_ns == 2_000_000_000 and c.autotune_cache is None
    for name, _ in ps.ps_config._fields_:
        if name not in ("precision", "wait_limit_ns", "autotune_cache"):
            assert getattr(c, name) == 0, name
    h = ps._h()
    for field, value in [("precision", ps.PS_PATH_THERMO), ("debug_checks", 2), ("wait_limit_ns", 10),
                         ("wait_limit_ns", 10**12), ("mgemm_feed", 3), ("mgemm3_feed", -1), ("mgemm_tile", 96),
                         ("mgemm_warps", 4), ("mgemm_unroll", 5), ("mgemm_add", 4), ("mgemm_band", 65),
                         ("tma_slice", 48), ("tma_unroll", 12), ("tma_stages", 5), ("tma_schedule", 3),
                         ("tma_meet", -1), ("mgemm3_schedule", 9), ("thermo_tile_m", 64),
                         ("thermo_meet_kb", -2), ("test_batched_stall", 2), ("mgemm_narrow", 3),
                         ("tma_lookahead", 8), ("host_direct", 2)]:
        bad = ps.config(**{field: value})
        assert ps.ps_create(ctypes.byref(h), 0, ctypes.byref(bad)) == ps.PS_ERR_INVALID_ARG, field
        assert field.encode() in ps.ps_last_error(None)
    assert ps.ps_create(None, 0, None) == ps.PS_ERR_INVALID_ARG
