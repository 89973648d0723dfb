"""Helpers for the GPU parity tests: call the C ABI with torch buffers."""
import ctypes

import numpy as np


def _torch():
    import torch
    return torch


def metrics_2way(ps, handle, V, path=0, out_dtype=np.float32, layout=0, levels=0,
                 on_host=False, stream=None):
    """Run ps_metrics_2way on a numpy matrix (shape per `layout`); returns numpy.
    on_host: True = pageable host input and output; "pinned" = pageable host
    input, pinned (device-mapped) host output."""
    torch = _torch()
    if layout == 0:
        nf, nv = V.shape
    else:
        nv, nf = V.shape
    npairs = nv * (nv - 1) // 2
    tdt = {np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8}[out_dtype]
    if on_host:
        X = np.ascontiguousarray(V)
        if on_host == "pinned":
            out_p = torch.empty(npairs, dtype=tdt).pin_memory()
            out = out_p.numpy()
        else:
            out = np.empty(npairs, dtype=out_dtype)
        m = ps.matrix(X, layout)
        optr = out.ctypes.data
    else:
        X = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        out_t = torch.empty(npairs, dtype=tdt, device="cuda")
        m = ps.matrix(X, layout)
        optr = out_t.data_ptr()
    st = torch.cuda.current_stream() if stream is None else stream
    ps.check(ps.ps_metrics_2way(handle.h, ctypes.byref(m), path, levels, optr,
                                {np.float32: 0, np.float64: 1, np.uint8: 2}[out_dtype], st.cuda_stream),
             handle.h)
    torch.cuda.synchronize()
    return out if on_host else out_t.cpu().numpy()


def metrics_3way(ps, handle, V, jb=None, je=None, layout=0):
    torch = _torch()
    nv = V.shape[1] if layout == 0 else V.shape[0]
    jb = 0 if jb is None else jb
    je = nv if je is None else je
    n = ps.ps_slab_size(nv, jb, je)
    X = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    m = ps.matrix(X, layout)
    ps.check(ps.ps_metrics_3way(handle.h, ctypes.byref(m), jb, je, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream), handle.h)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy()


def assert_rel(got, ref, rtol, what=""):
    """|got - ref| <= rtol * |ref| elementwise (zeros must be exact)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    err = np.abs(got - ref)
    bad = err > rtol * np.abs(ref)
    if bad.any():
        idx = np.flatnonzero(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside rtol={rtol}; first "
                             f"{[(int(t), float(got[t]), float(ref[t])) for t in idx]}")
    nz = ref != 0
    return float((err[nz] / np.abs(ref[nz])).max()) if nz.any() else 0.0


def slab_index(nv, jb, i, j, k):
    """Position of (i, j, k) in the pivot-slab layout starting at pivot jb."""
    i, j, k = (np.asarray(x, dtype=np.int64) for x in (i, j, k))
    F = lambda x: (nv - 1) * (x * (x - 1) // 2) - (x - 1) * x * (2 * x - 1) // 6  # noqa: E731
    return F(j) - F(np.int64(jb)) + i * (nv - 1 - j) + (k - j - 1)


def threshold_3way(ps, handle, V, tau, capacity, use_proposal=0, on_host=False):
    """Returns (status, count, triples as (n,3) int array, values float32)."""
    torch = _torch()
    X = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    m = ps.matrix(X)
    if on_host:
        out = (ps.ps_triple * max(capacity, 1))()
        cnt = ctypes.c_int64(-1)
        st = ps.ps_threshold_3way(handle.h, ctypes.byref(m), float(tau), use_proposal,
                                  ctypes.addressof(out), capacity, ctypes.addressof(cnt), 0)
        raw = np.frombuffer(out, dtype=np.int32).reshape(-1, 4)
        count = cnt.value
    else:
        out = torch.empty((max(capacity, 1), 4), dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = ps.ps_threshold_3way(handle.h, ctypes.byref(m), float(tau), use_proposal, out.data_ptr(),
                                  capacity, cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        raw = out.cpu().numpy()
        count = int(cnt.item())
    n = min(count, capacity) if count >= 0 else 0
    trip = raw[:n, :3].astype(np.int64)
    vals = raw[:n, 3].copy().view(np.float32)
    return st, count, trip, vals


def threshold_2way(ps, handle, V, tau, capacity, on_host=False):
    """Returns (status, count, pairs as (n,2) int array, values float32)."""
    torch = _torch()
    X = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    m = ps.matrix(X)
    if on_host:
        out = (ps.ps_pair * max(capacity, 1))()
        cnt = ctypes.c_int64(-1)
        st = ps.ps_threshold_2way(handle.h, ctypes.byref(m), float(tau), ctypes.addressof(out), capacity,
                                  ctypes.addressof(cnt), 0)
        raw = np.frombuffer(out, dtype=np.int32).reshape(-1, 3)
        count = cnt.value
    else:
        out = torch.empty((max(capacity, 1), 3), dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = ps.ps_threshold_2way(handle.h, ctypes.byref(m), float(tau), out.data_ptr(), capacity,
                                  cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        raw = out.cpu().numpy()
        count = int(cnt.item())
    n = min(count, capacity) if count >= 0 else 0
    return st, count, raw[:n, :2].astype(np.int64), raw[:n, 2].copy().view(np.float32)
