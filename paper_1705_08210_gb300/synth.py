"""Seeded synthetic inputs shaped like GWAS/PheWAS association matrices.

This module only draws random numbers; it holds none of the similarity
arithmetic.  Both the CUDA path and the CPU oracle consume what it returns.

All matrices are returned FIELD-MAJOR: a C-contiguous numpy array of shape
(nf, nv) whose element [q, i] is field q of vector i.  That is the library's
layout 0 ("column-major nv x nf"): element (i, q) at offset i + q*nv.

Value recipe (stands in for association matrices whose entries are
-log10 p-values; the paper's poplar PheWAS data are not available):
  * each entry is 0 with probability p_zero (0.85),
  * otherwise -log10(U) with U ~ Uniform(0, 1], i.e. Exponential(1)/ln 10.
One uniform r ~ U[0,1) is drawn per entry: r < p_zero gives 0, else
U = (1 - r) / (1 - p_zero).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 170508210

# Named workloads: (nv, nf).  Seeds are SEED_BASE + workload number.
WORKLOADS = {
    "2way_1024x512_f64": dict(nv=1024, nf=512, dtype=np.float64, number=1),
    "2way_32768x8192_f32": dict(nv=32768, nf=8192, dtype=np.float32, number=2),
    "3way_2048x4096_f32": dict(nv=2048, nf=4096, dtype=np.float32, number=3),
    "batched_64_uneven": dict(number=4),
    "threshold3_8192x2048_f32": dict(nv=8192, nf=2048, dtype=np.float32, number=5),
}


def seed_for(number: int, sub: int = 0) -> int:
    return SEED_BASE + int(number) + 1000 * int(sub)


def zero_inflated(nv: int, nf: int, seed: int, p_zero: float = 0.85,
                  dtype=np.float32, chunk_rows: int = 256) -> np.ndarray:
    """(nf, nv) field-major matrix of zero-inflated -log10(U) values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((nf, nv), dtype=dtype)
    for q0 in range(0, nf, chunk_rows):
        q1 = min(nf, q0 + chunk_rows)
        r = rng.random((q1 - q0, nv))
        val = np.zeros_like(r)
        nz = r >= p_zero
        val[nz] = -np.log10((1.0 - r[nz]) / (1.0 - p_zero))
        out[q0:q1] = val.astype(dtype, copy=False)
    return out


def integer_levels(nv: int, nf: int, seed: int, levels: int = 16,
                   p_zero: float = 0.85, dtype=np.float32) -> np.ndarray:
    """(nf, nv) field-major matrix of integer values in 0..levels-1
    (0 with probability p_zero, else uniform in 1..levels-1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.random((nf, nv))
    v = rng.integers(1, levels, size=(nf, nv))
    return np.where(r < p_zero, 0, v).astype(dtype)


def latent_profiles(nv: int, nf: int, seed: int, n_profiles: int = 64,
                    sigma: float = 0.25, p_zero: float = 0.85,
                    dtype=np.float32, profile_seed: int | None = None):
    """(nf, nv) field-major matrix v_i = a_i * P[z_i] + sigma * N_i.

    P holds n_profiles zero-inflated profiles, z_i ~ U{0..n_profiles-1},
    a_i ~ U[0.5, 1.5], N_i zero-inflated noise of the same distribution.
    P is drawn from profile_seed (default: seed), z, a and N from seed, so
    calls with the same profile_seed and different seeds draw fresh vectors
    from one population.  Returns (V, z) where z is the latent profile index
    of each vector."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pseed = seed if profile_seed is None else profile_seed
    P = zero_inflated(n_profiles, nf, pseed + 7, p_zero=p_zero, dtype=np.float64)
    z = rng.integers(0, n_profiles, size=nv)
    a = rng.uniform(0.5, 1.5, size=nv)
    N = zero_inflated(nv, nf, seed + 11, p_zero=p_zero, dtype=np.float64)
    V = P[:, z] * a[None, :] + sigma * N
    return np.ascontiguousarray(V, dtype=dtype), z


def batched_shapes(seed: int, n_instances: int = 64, n_2way: int = 48):
    """Shapes of the batched uneven workload: list of (way, nv, nf).

    2-way instances: nv ~ U[256, 4096], nf ~ U[512, 8192];
    3-way instances: nv ~ U[256, 1024], nf ~ U[512, 8192]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = []
    for t in range(n_instances):
        if t < n_2way:
            nv = int(rng.integers(256, 4097))
        else:
            nv = int(rng.integers(256, 1025))
        nf = int(rng.integers(512, 8193))
        shapes.append((2 if t < n_2way else 3, nv, nf))
    return shapes


def sample_pairs(nv: int, n: int, seed: int) -> np.ndarray:
    """n distinct-ish random pairs (i, j) with i < j."""
    rng = np.random.Generator(np.random.PCG64(seed))
    i = rng.integers(0, nv, size=n)
    j = rng.integers(0, nv - 1, size=n)
    j = np.where(j >= i, j + 1, j)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return np.stack([lo, hi], axis=1).astype(np.int64)


def sample_triples(nv: int, n: int, seed: int) -> np.ndarray:
    """n random triples (i, j, k) with i < j < k."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n, 3), dtype=np.int64)
    c = 0
    while c < n:
        t = np.sort(rng.integers(0, nv, size=(2 * (n - c) + 8, 3)), axis=1)
        ok = (t[:, 0] < t[:, 1]) & (t[:, 1] < t[:, 2])
        t = t[ok][: n - c]
        out[c:c + len(t)] = t
        c += len(t)
    return out


def binary_bits(nv: int, nf: int, seed: int, p_one: float = 0.15, ld_words: int | None = None,
                junk_tail: bool = True):
    """0/1 vectors (each field 1 with probability p_one), returned twice:
    as the (nf, nv) field-major float32 matrix the oracle reads, and packed
    for the library's PS_B1 input: an (nv, ld_words) uint32 array, field q
    of vector i in bit q % 32 of word [i, q // 32].  With junk_tail the bits
    at q >= nf (and the words past ceil(nf/32)) are filled with random bits,
    which the library must ignore."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dense = (rng.random((nf, nv)) < p_one).astype(np.float32)
    nw = (nf + 31) // 32
    ld = nw if ld_words is None else int(ld_words)
    words = rng.integers(0, 2**32, size=(nv, max(ld, 1)), dtype=np.uint64).astype(np.uint32) \
        if junk_tail else np.zeros((nv, max(ld, 1)), dtype=np.uint32)
    bits = np.zeros((nv, nw * 32), dtype=np.uint8)
    bits[:, :nf] = dense.T.astype(np.uint8)
    if junk_tail and nf % 32:
        bits[:, nf:] = rng.integers(0, 2, size=(nv, nw * 32 - nf), dtype=np.uint8)
    packed = np.packbits(bits.reshape(nv, nw, 32)[:, :, ::-1], axis=2).reshape(nv, nw, 4)
    words[:, :nw] = (packed[:, :, 0].astype(np.uint32) << 24 | packed[:, :, 1].astype(np.uint32) << 16
                     | packed[:, :, 2].astype(np.uint32) << 8 | packed[:, :, 3].astype(np.uint32))
    return dense, words
