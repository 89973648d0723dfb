"""Pins for the CPU oracle against facts that do not restate its code.

Every check here comes from somewhere other than the oracle's own formula:
a library routine (scipy's Bray-Curtis distance), an independent closed form
(the max-form of the 3-way numerator, sorting identities behind the
presorting remark of Section 2.1), set arithmetic (Dice/Sorenson, Section
2.3), analytic families, invariants, and hand-worked values.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1705_08210_gb300 import synth


def _rand_nonneg(n, nf, seed, p_zero=0.5):
    rng = np.random.default_rng(seed)
    V = rng.exponential(1.0, size=(n, nf))
    V[rng.random((n, nf)) < p_zero] = 0.0
    return V


# --------------------------------------------------------------------------
# hand-worked example (values derived by hand from Section 2.1 / 2.2)
#   u=(1,0,2) v=(2,1,0) w=(0,3,1); S = 3, 3, 4
#   n2(u,v)=1+0+0=1 -> c2=2/6=1/3 ; n2(u,w)=0+0+1=1 -> c2=2/7
#   n2(v,w)=0+1+0=1 -> c2=2/7 ; n3'=0+0+0=0 ; n3=3 ; d3=10 ; c3=9/20
# --------------------------------------------------------------------------
def test_hand_worked_example():
    V = np.array([[1, 0, 2], [2, 1, 0], [0, 3, 1]], dtype=np.float64)
    c2 = oracle.c2_packed(V)
    assert c2[0] == pytest.approx(1 / 3, rel=1e-15)
    assert c2[1] == pytest.approx(2 / 7, rel=1e-15)
    assert c2[2] == pytest.approx(2 / 7, rel=1e-15)
    assert oracle.n3prime(V, 0, 1, 2) == 0.0
    assert oracle.c3_triples(V, [[0, 1, 2]])[0] == pytest.approx(0.45, rel=1e-15)


def test_hand_worked_example_with_shared_minimum():
    #   a=(2,1,3,0) b=(1,1,4,2) c=(3,0,2,2); S = 6, 8, 7
    #   n2(a,b)=1+1+3+0=5 ; n2(a,c)=2+0+2+0=4 ; n2(b,c)=1+0+2+2=5
    #   n3'=1+0+2+0=3 ; n3=5+4+5-3=11 ; d3=21 ; c3=1.5*11/21=11/14
    V = np.array([[2, 1, 3, 0], [1, 1, 4, 2], [3, 0, 2, 2]], dtype=np.float64)
    assert oracle.c2_packed(V) == pytest.approx([10 / 14, 8 / 13, 10 / 15], rel=1e-15)
    assert oracle.n3prime(V, 0, 1, 2) == 3.0
    assert oracle.c3_triples(V, [[0, 1, 2]])[0] == pytest.approx(11 / 14, rel=1e-15)


# --------------------------------------------------------------------------
# library special case: c2 = 1 - Bray-Curtis distance (min(a,b)=(a+b-|a-b|)/2)
# --------------------------------------------------------------------------
def test_c2_is_one_minus_braycurtis():
    from scipy.spatial.distance import braycurtis
    V = _rand_nonneg(20, 37, seed=1)
    c2 = oracle.c2_packed(V)
    for i in range(20):
        for j in range(i + 1, 20):
            ref = 1.0 - braycurtis(V[i], V[j])
            assert c2[oracle.pair_index(20, i, j)] == pytest.approx(ref, rel=1e-13, abs=1e-15)


# --------------------------------------------------------------------------
# independent closed form of eq. (1): per element, min-sum of the three pairs
# minus the triple min equals the sum of the two smallest values,
# = u+v+w-max(u,v,w).  Hence c3 = 1.5*(1 - sum max / sum(u+v+w)).
# --------------------------------------------------------------------------
def test_c3_matches_max_form():
    V = _rand_nonneg(9, 41, seed=2)
    trip = np.array(list(itertools.combinations(range(9), 3)))
    got = oracle.c3_triples(V, trip)
    for t, g in zip(trip, got):
        X = V[t]
        ref = 1.5 * (1.0 - X.max(axis=0).sum() / X.sum())
        assert g == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_n3prime_against_numpy_min_reduce():
    V = _rand_nonneg(7, 29, seed=3)
    trip = np.array(list(itertools.combinations(range(7), 3)))
    got = oracle.n3prime_triples(V, trip)
    ref = np.minimum.reduce([V[trip[:, 0]], V[trip[:, 1]], V[trip[:, 2]]]).sum(axis=1)
    np.testing.assert_allclose(got, ref, rtol=1e-13)


# --------------------------------------------------------------------------
# analytic families (the paper's "verifiable analytically" synthetic cases)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [0.25, 0.5, 1.0, 2.0, 7.5])
def test_scaled_copy_2way(alpha):
    u = _rand_nonneg(1, 50, seed=4, p_zero=0.3)[0] + 0.0
    V = np.stack([u, alpha * u])
    ref = 2 * min(1.0, alpha) / (1 + alpha)
    assert oracle.c2_packed(V)[0] == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (1.5, 2.0), (2.0, 5.0), (3.0, 3.0)])
def test_scaled_copies_3way(alpha, beta):
    u = _rand_nonneg(1, 50, seed=5, p_zero=0.3)[0]
    V = np.stack([u, alpha * u, beta * u])
    ref = 1.5 * (1 + alpha) / (1 + alpha + beta)
    for perm in itertools.permutations(range(3)):
        assert oracle.c3_triples(V[list(perm)], [[0, 1, 2]])[0] == pytest.approx(ref, rel=1e-13)


def test_disjoint_supports_give_zero():
    V = np.zeros((3, 12))
    V[0, 0:4] = [1, 2, 3, 4]
    V[1, 4:8] = [5, 1, 1, 2]
    V[2, 8:12] = [0.5, 0.5, 9, 1]
    assert np.all(oracle.c2_packed(V) == 0.0)
    # c3 with pairwise-disjoint supports: every n2 and n3' vanish
    assert oracle.c3_triples(V, [[0, 1, 2]])[0] == 0.0


# --------------------------------------------------------------------------
# Section 2.3: on 0/1 data the metric is the Sorenson (Dice) coefficient
# --------------------------------------------------------------------------
def test_sorenson_dice_on_sets():
    rng = np.random.default_rng(6)
    n, nf = 8, 40
    B = (rng.random((n, nf)) < 0.4).astype(np.float64)
    sets = [set(np.flatnonzero(B[i]).tolist()) for i in range(n)]
    c2 = oracle.c2_packed(B)
    for i in range(n):
        for j in range(i + 1, n):
            A, C = sets[i], sets[j]
            ref = Fraction(2 * len(A & C), len(A) + len(C)) if (A or C) else Fraction(0)
            assert c2[oracle.pair_index(n, i, j)] == pytest.approx(float(ref), rel=1e-15)
    trip = list(itertools.combinations(range(n), 3))
    c3 = oracle.c3_triples(B, trip)
    for (i, j, k), g in zip(trip, c3):
        A, Bs, C = sets[i], sets[j], sets[k]
        num = len(A & Bs) + len(A & C) + len(Bs & C) - len(A & Bs & C)
        ref = Fraction(3 * num, 2 * (len(A) + len(Bs) + len(C)))
        assert g == pytest.approx(float(ref), rel=1e-15)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def test_self_similarity_is_one():
    V = _rand_nonneg(6, 30, seed=7, p_zero=0.6)
    V[:, 0] += 1.0  # make every vector nonzero
    for i in range(6):
        W = np.stack([V[i], V[i], V[i]])
        assert oracle.c2_packed(W[:2])[0] == pytest.approx(1.0, rel=1e-15)
        assert oracle.c3_triples(W, [[0, 1, 2]])[0] == pytest.approx(1.0, rel=1e-15)


def test_symmetry_under_permutation():
    V = _rand_nonneg(3, 64, seed=8)
    base2 = oracle.c2_packed(V[:2])[0]
    assert oracle.c2_packed(V[[1, 0]])[0] == base2
    vals = [oracle.c3_triples(V[list(p)], [[0, 1, 2]])[0] for p in itertools.permutations(range(3))]
    assert max(vals) - min(vals) <= 4e-16 * max(vals)


def test_range_zero_one():
    V = _rand_nonneg(14, 25, seed=9, p_zero=0.7)
    c2 = oracle.c2_packed(V)
    assert np.all(c2 >= 0) and np.all(c2 <= 1 + 1e-15)
    c3 = oracle.c3_slab(V, 0, 14)
    assert np.all(c3 >= 0) and np.all(c3 <= 1 + 1e-15)


def test_pair_with_zero_vector_three_quarters():
    # c3(u, u, 0) = 1.5 * (S + S + S - S) / (2S) = 0.75 for any u != 0
    u = _rand_nonneg(1, 33, seed=10, p_zero=0.2)[0]
    V = np.stack([u, u, np.zeros_like(u)])
    assert oracle.c3_triples(V, [[0, 1, 2]])[0] == pytest.approx(0.75, rel=1e-15)


def test_all_zero_vectors_read_as_zero():
    V = np.zeros((3, 5))
    assert np.all(oracle.c2_packed(V) == 0.0)
    assert oracle.c3_triples(V, [[0, 1, 2]])[0] == 0.0


# --------------------------------------------------------------------------
# sorting identities (Section 2.1 presorting remark): for one field with
# values sorted ascending x_(1) <= ... <= x_(n),
#   sum_{i<j} min(x_i, x_j)       = sum_r x_(r) * (n - r)
#   sum_{i<j<k} min(x_i,x_j,x_k)  = sum_r x_(r) * C(n - r, 2)
# Exact on integer data.
# --------------------------------------------------------------------------
def test_pair_sum_sorting_identity_exact():
    V = synth.integer_levels(nv=30, nf=17, seed=11).T.astype(np.float64)  # (nv, nf)
    n = V.shape[0]
    total = oracle.n2_packed(V).sum()
    ref = 0
    for q in range(V.shape[1]):
        xs = sorted(int(x) for x in V[:, q])
        ref += sum(x * (n - r) for r, x in enumerate(xs, start=1))
    assert total == ref


def test_triple_sum_sorting_identity_exact():
    V = synth.integer_levels(nv=16, nf=11, seed=12, p_zero=0.3).T.astype(np.float64)
    n = V.shape[0]
    trip = np.array(list(itertools.combinations(range(n), 3)))
    total = oracle.n3prime_triples(V, trip).sum()
    ref = 0
    for q in range(V.shape[1]):
        xs = sorted(int(x) for x in V[:, q])
        ref += sum(x * math.comb(n - r, 2) for r, x in enumerate(xs, start=1))
    assert total == ref


# --------------------------------------------------------------------------
# enumeration / layouts: brute force over all tuples
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nv", [2, 3, 5, 12])
def test_packed_pairs_cover_each_pair_once(nv):
    V = _rand_nonneg(nv, 9, seed=13)
    pairs = np.array([(i, j) for i in range(nv) for j in range(i + 1, nv)])
    idx = oracle.pair_index(nv, pairs[:, 0], pairs[:, 1])
    assert sorted(idx.tolist()) == list(range(nv * (nv - 1) // 2))
    packed = oracle.c2_packed(V)
    np.testing.assert_array_equal(packed[idx], oracle.c2_pairs(V, pairs))


@pytest.mark.parametrize("nv", [3, 4, 9])
def test_slab_layout_brute_force(nv):
    V = _rand_nonneg(nv, 8, seed=14)
    order = [(i, j, k) for j in range(nv) for i in range(j) for k in range(j + 1, nv)]
    assert len(order) == nv * (nv - 1) * (nv - 2) // 6
    full = oracle.c3_slab(V, 0, nv)
    np.testing.assert_array_equal(full, oracle.c3_triples(V, order))
    # slabs concatenate
    parts = [oracle.c3_slab(V, a, b) for a, b in [(0, 1), (1, nv // 2), (nv // 2, nv)]]
    np.testing.assert_array_equal(np.concatenate(parts), full)
    assert oracle.slab_size(nv, 0, nv) == len(order)


def test_threshold_matches_enumeration_and_overflow():
    V = synth.latent_profiles(24, 16, seed=15, n_profiles=3, sigma=0.2)[0].T.astype(np.float64)
    nv = V.shape[0]
    tau = 0.6
    ijk, val, total = oracle.threshold_3way(V, tau)
    trip = list(itertools.combinations(range(nv), 3))  # lexicographic
    c3 = oracle.c3_triples(V, trip)
    ref = [(t, c) for t, c in zip(trip, c3) if c >= tau]
    assert total == len(ref) and total > 10
    assert [tuple(r) for r in ijk.tolist()] == [t for t, _ in ref]
    np.testing.assert_array_equal(val, [c for _, c in ref])
    ijk2, val2, total2 = oracle.threshold_3way(V, tau, capacity=5)
    assert total2 == total and len(ijk2) == 5
    np.testing.assert_array_equal(ijk2, ijk[:5])


# --------------------------------------------------------------------------
# quantizer and thermometer identity (not in the paper; reading documented)
# --------------------------------------------------------------------------
def test_percentile_nearest_rank():
    x = synth.zero_inflated(50, 40, seed=16).ravel()
    nz = np.sort(x[x != 0])
    r = math.ceil(0.999 * nz.size)
    assert oracle.percentile_nonzero(x) == nz[r - 1]
    assert oracle.percentile_nonzero(np.zeros(10, np.float32)) == 0.0


def test_quantizer_rounds_to_nearest_level():
    L = 16
    x = synth.zero_inflated(64, 64, seed=17).ravel()
    P = oracle.percentile_nonzero(x)
    q = oracle.quantize(x, L, P)
    assert q.min() >= 0 and q.max() == L - 1
    assert np.all(q[x == 0] == 0)
    step = P / (L - 1)
    inside = x <= P
    # round-to-nearest: reconstruction error at most half a step (+ fp32 slack)
    err = np.abs(x[inside] - q[inside] * step)
    assert np.all(err <= 0.5 * step * (1 + 1e-5))
    # monotone in x
    o = np.argsort(x, kind="stable")
    assert np.all(np.diff(q[o]) >= 0)
    # values above the percentile saturate at the top level
    assert np.all(q[x >= P] == L - 1)


def test_thermometer_identity_matches_min_sum():
    # min(a, b) = sum_{t=1}^{L-1} [a >= t][b >= t] for integer levels a, b
    L = 16
    Q = synth.integer_levels(nv=10, nf=23, seed=18, levels=L).T.astype(np.int64)  # (nv, nf)
    T = np.concatenate([(Q >= t) for t in range(1, L)], axis=1).astype(np.float64)
    via_matmul = T @ T.T
    n2 = oracle.n2_packed(Q.astype(np.float64))
    for i in range(10):
        for j in range(i + 1, 10):
            assert via_matmul[i, j] == n2[oracle.pair_index(10, i, j)]


def test_metric_code_grid_and_rounding():
    # the 256 exact grid points k/255 encode to k; points 0.3/255 either side
    # still round to k (a floor or ceiling instead of rounding fails here), and
    # the ends map to 0 and 255 (a missing or wrong 255 scale fails here)
    k = np.arange(256)
    np.testing.assert_array_equal(oracle.metric_code(k / 255.0), k)
    kk = np.arange(1, 255)
    np.testing.assert_array_equal(oracle.metric_code((kk - 0.3) / 255.0), kk)
    np.testing.assert_array_equal(oracle.metric_code((kk + 0.3) / 255.0), kk)
    assert oracle.metric_code([0.0])[0] == 0 and oracle.metric_code([1.0])[0] == 255
    # clamp above 1 (FP32 metrics may exceed 1 by an ulp)
    assert oracle.metric_code([1.0 + 1e-7, 1.01])[1] == 255


def test_metric_code_error_bound_and_monotone():
    # |code/255 - c| <= 1/510 (+ FP32 rounding of c) on [0, 1]; non-decreasing
    rng = np.random.default_rng(7)
    c = np.sort(rng.random(200_000))
    q = oracle.metric_code(c).astype(np.int64)
    assert np.all(np.diff(q) >= 0)
    assert np.max(np.abs(q / 255.0 - c)) <= 1.0 / 510.0 + 1e-6
    # about 2.4 significant figures near 1: relative error at c >= 0.5 below 0.4%
    hi = c >= 0.5
    assert np.max(np.abs(q[hi] / 255.0 - c[hi]) / c[hi]) < 0.004


def test_threshold_2way_hand_example():
    # identical vectors give c2 = 1, disjoint supports 0, half overlap
    # 2*1/(2+2) = 0.5; tau is inclusive; output sorted by (i, j)
    V = np.array([[1.0, 1.0, 0.0, 0.0],
                  [1.0, 1.0, 0.0, 0.0],
                  [0.0, 0.0, 1.0, 1.0],
                  [1.0, 0.0, 1.0, 0.0]])
    pairs, vals = oracle.threshold_2way(V, 0.5)
    np.testing.assert_array_equal(pairs, [[0, 1], [0, 3], [1, 3], [2, 3]])
    np.testing.assert_allclose(vals, [1.0, 0.5, 0.5, 0.5], rtol=0, atol=1e-15)
    pairs, vals = oracle.threshold_2way(V, 0.75)
    np.testing.assert_array_equal(pairs, [[0, 1]])
    assert oracle.threshold_2way(V, 1.5)[0].shape == (0, 2)


def test_sorenson_special_case_set_closed_forms():
    # Section 2.3: for 0/1 vectors the metric is the Sorenson index
    # 2|A & B| / (|A| + |B|); eq. (1) on sets: n3 = |A&B| + |A&C| + |B&C| -
    # |A&B&C| (a field where exactly two vectors are 1 counts once, where all
    # three are 1 twice)
    rng = np.random.default_rng(23)
    V = (rng.random((9, 70)) < 0.3).astype(np.float64)
    sets = [set(np.nonzero(v)[0].tolist()) for v in V]
    pairs = np.array([(i, j) for i in range(9) for j in range(i + 1, 9)])
    want2 = [2 * len(sets[i] & sets[j]) / (len(sets[i]) + len(sets[j])) for i, j in pairs]
    np.testing.assert_allclose(oracle.c2_pairs(V, pairs), want2, rtol=0, atol=1e-15)
    trip = np.array([(i, j, k) for i in range(9) for j in range(i + 1, 9) for k in range(j + 1, 9)])
    want3 = []
    for i, j, k in trip:
        A, B, C = sets[i], sets[j], sets[k]
        n3 = len(A & B) + len(A & C) + len(B & C) - len(A & B & C)
        two = sum(1 for q in range(70) if (q in A) + (q in B) + (q in C) == 2)
        assert n3 == two + 2 * len(A & B & C)
        want3.append(1.5 * n3 / (len(A) + len(B) + len(C)))
    np.testing.assert_allclose(oracle.c3_triples(V, trip), want3, rtol=0, atol=1e-15)
