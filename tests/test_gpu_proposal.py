"""Learned block proposal and lossless bound filter for the thresholded 3-way
search.  The encoder's forward and gradient are checked against the FP64 CPU
re-statement; the proposal's recall is judged by the exhaustive search; the
bound filter must reproduce the exhaustive result exactly."""
import ctypes

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1705_08210_gb300 import synth
from gpu_run import threshold_3way

pytestmark = pytest.mark.gpu


def _dev(V):
    import torch
    return torch.from_numpy(np.ascontiguousarray(V)).cuda()


def _pair_grad_gpu(ps, handle, V, pairs, y, theta):
    import torch
    nv = V.shape[1]
    n = ps.ps_proposal_param_count(handle.h)
    ps.check(ps.ps_proposal_params(handle.h, 1, theta.ctypes.data, n, None), handle.h)
    X = _dev(V)
    m = ps.matrix(X)
    dp, dy = _dev(pairs.astype(np.int32)), _dev(y.astype(np.float32))
    E = torch.empty(nv * 64, device="cuda")
    g = torch.empty(n, device="cuda")
    loss = ctypes.c_double()
    ps.check(ps.ps_proposal_pair_grad(handle.h, ctypes.byref(m), dp.data_ptr(), dy.data_ptr(), len(y),
                                      E.data_ptr(), g.data_ptr(), ctypes.addressof(loss),
                                      torch.cuda.current_stream().cuda_stream), handle.h)
    return E.cpu().numpy().reshape(nv, 64), loss.value, g.cpu().numpy()


@pytest.mark.parametrize("nv,d_in,scale", [(1100, 2048, 0.03), (300, 385, 0.08), (40, 32, 0.15)])
def test_encoder_within_derived_bounds(ps, handle, nv, d_in, scale):
    # the encoder at the width of the searched 8192 x 2048 workload (d_in =
    # 2048, 256 hidden, 64 outputs) on 1100 vectors (not a multiple of the
    # 128-row tensor-core tiles), and two narrow cases (ragged 64-element K
    # blocks): embeddings, loss and every gradient block against the FP64
    # oracle with the same BF16 weights, each element within the a-priori
    # rounding-error bound of the arithmetic (tests/mlp_bounds.py)
    from mlp_bounds import encoder_bounds
    ps.check(ps.ps_proposal_init(handle.h, d_in, 4321), handle.h)
    n = ps.ps_proposal_param_count(handle.h)
    rng = np.random.default_rng(d_in)
    theta = rng.normal(0, scale, size=n).astype(np.float32)
    V, _ = synth.latent_profiles(nv, d_in, synth.seed_for(5, 400 + d_in), n_profiles=16, sigma=0.4)
    npair = 3000
    pairs = np.stack([rng.integers(0, nv, npair), rng.integers(0, nv, npair)], axis=1)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    y = (rng.random(len(pairs)) < 0.3).astype(np.float64)
    gE, gloss, gg = _pair_grad_gpu(ps, handle, V, pairs, y, theta)
    th = theta.astype(np.float64)
    n1 = 256 * d_in
    th[:n1] = mo.bf16_round(theta[:n1])
    o = n1 + 256
    th[o:o + 64 * 256] = mo.bf16_round(theta[o:o + 64 * 256])
    ref_loss, ref_g, ref_E = mo.pair_loss_and_grad(th, V, pairs, y)
    B = encoder_bounds(th, V, pairs, y)
    errE = np.abs(gE - ref_E)
    assert np.all(errE <= B["E"]), (errE.max(), float((errE / B["E"]).max()))
    assert abs(gloss - ref_loss) <= B["loss"], (gloss, ref_loss, B["loss"])
    worst = {}
    for lo, hi, name in [(0, n1, "W1"), (n1, n1 + 256, "b1"), (o, o + 64 * 256, "W2"), (o + 64 * 256, n, "b2")]:
        err = np.abs(gg[lo:hi] - ref_g[lo:hi])
        ratio = err / np.maximum(B[name], 1e-300)
        worst[name] = float(ratio.max())
        assert np.all(err <= B[name]), (name, float(err.max()), worst[name])
    print(f"encoder d_in={d_in} nv={nv}: max error / bound: E {float((errE / B['E']).max()):.3f}, "
          + ", ".join(f"{k} {v:.3f}" for k, v in worst.items()))


def _train_on_subsets(ps, handle, V, n_sub, size, steps=300, seed=5):
    """Train the encoder on the exact results of small random subsets of V."""
    import torch
    rng = np.random.default_rng(seed)
    mats, keep = (ps.ps_matrix * n_sub)(), []
    for t in range(n_sub):
        cols = np.sort(rng.choice(V.shape[1], size, replace=False))
        X = _dev(V[:, cols])
        keep.append(X)
        mats[t] = ps.matrix(X)
    loss = ctypes.c_double()
    ps.check(ps.ps_proposal_train(handle.h, mats, n_sub, 0.7, steps, 1e-3, 0.999, 99,
                                  ctypes.addressof(loss), torch.cuda.current_stream().cuda_stream), handle.h)
    return loss.value


def test_learned_proposal_recall_and_gain(ps, handle):
    nf = 256
    V, _ = synth.latent_profiles(2048, nf, synth.seed_for(5, 200), n_profiles=16, sigma=0.4)
    loss = _train_on_subsets(ps, handle, V, 3, 512)
    assert np.isfinite(loss)
    st0, c0, t0, v0 = threshold_3way(ps, handle, V, 0.7, capacity=4_000_000, use_proposal=0)
    assert st0 == ps.PS_OK and c0 > 1000
    st1, c1, t1, v1 = threshold_3way(ps, handle, V, 0.7, capacity=4_000_000, use_proposal=1)
    kept = ctypes.c_double()
    nb = ctypes.c_int64()
    ps.check(ps.ps_proposal_last_stats(handle.h, ctypes.byref(kept), ctypes.byref(nb)), handle.h)
    assert st1 == ps.PS_OK
    ref = {tuple(x): v for x, v in zip(t0.tolist(), v0)}
    got = {tuple(x): v for x, v in zip(t1.tolist(), v1)}
    assert set(got) <= set(ref)                        # no false triples
    assert all(got[k] == ref[k] for k in got)          # bit-identical values
    recall = len(got) / len(ref)
    print(f"learned proposal: recall {recall:.5f}, blocks searched {kept.value:.4f} ({nb.value})")
    assert recall >= 0.99
    assert kept.value < 0.5                            # the encoder prunes most blocks
    # the lossless bound filter on the encoder's ordering finds everything
    st2, c2, t2, v2 = threshold_3way(ps, handle, V, 0.7, capacity=4_000_000, use_proposal=2)
    assert st2 == ps.PS_OK and c2 == c0
    np.testing.assert_array_equal(t2, t0)
    np.testing.assert_array_equal(v2, v0)


def test_bound_filter_is_lossless(ps, handle):
    V, _ = synth.latent_profiles(700, 128, synth.seed_for(5, 300), n_profiles=8, sigma=0.3)
    st0, c0, t0, v0 = threshold_3way(ps, handle, V, 0.7, capacity=2_000_000, use_proposal=0)
    st2, c2, t2, v2 = threshold_3way(ps, handle, V, 0.7, capacity=2_000_000, use_proposal=2)
    assert st0 == st2 == ps.PS_OK and c0 == c2 > 0
    np.testing.assert_array_equal(t0, t2)
    np.testing.assert_array_equal(v0, v2)


def test_proposal_requires_trained_encoder(ps):
    h2 = ps.Handle(0)
    V = synth.zero_inflated(50, 16, 1)
    st, _, _, _ = threshold_3way(ps, h2, V, 0.7, capacity=10, use_proposal=1)
    assert st == ps.PS_ERR_INVALID_ARG
    h2.close()
