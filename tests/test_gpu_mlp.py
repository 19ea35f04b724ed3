"""GPU predictor (through the C ABI) against the FP64 MLP oracle, and the
learned join prologue against the plans it must reduce to."""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()


def test_loss_and_gradient_match_fp64_oracle():
    from oracle import mlp as omlp
    rng = np.random.default_rng(1)
    din, h1, h2, n = 20, 48, 40, 70
    m = vj.MLP(din, h1, h2, seed=3)
    flat = (rng.standard_normal(m.num_params()) * 0.3).astype(np.float32)
    m.set_params(flat)
    x = rng.standard_normal((n, din)).astype(np.float32)
    tr = rng.standard_normal(n).astype(np.float32)
    tc = (rng.random(n) < 0.4).astype(np.float32)
    loss, g = m.loss_grad(x, tr, tc)
    lref, gref = omlp.loss_grad(flat.astype(np.float64), x.astype(np.float64), tr, tc, din, h1, h2)
    assert loss == pytest.approx(lref, rel=1e-5)
    err = np.linalg.norm(g.astype(np.float64) - gref) / np.linalg.norm(gref)
    assert err < 1e-5, err
    np.testing.assert_allclose(g, gref, rtol=1e-3, atol=1e-5 * np.abs(gref).max())
    m.free()


def test_training_learns_and_predict_matches_oracle_forward():
    from oracle import mlp as omlp
    rng = np.random.default_rng(2)
    din, n = 12, 4000
    x = (rng.standard_normal((n, din)) * 3 + 5).astype(np.float32)
    tc = (x[:, 0] > 5).astype(np.float32)
    tr = (0.5 * (x[:, 1] - 5)).astype(np.float32)
    m = vj.MLP(din, 64, 64, seed=4)
    l0, _ = m.loss_grad((x - x.mean(0)) / x.std(0), tr, tc)
    lf = m.train(x, tr, tc, epochs=15, batch=128, lr=3e-3, seed=5)
    assert lf < 0.25 * l0, (l0, lf)
    flat, mu, sd = m.get_params()
    y = m.predict(x[:300])
    yref, _ = omlp.forward(flat.astype(np.float64), (x[:300].astype(np.float64) - mu) / sd, din, 64, 64)
    np.testing.assert_allclose(y, yref, rtol=1e-4, atol=1e-4)
    acc = ((y[:, 1] > 0) == (tc[:300] > 0.5)).mean()
    assert acc > 0.9
    m.free()


def test_features_match_definitions(oracle):
    w = inputs.gauss_small(seed=31, nx=2000, nq=200, d=16, k=8, ood_frac=0.2, shift=10.0)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=12, knn_k=24))
    adj, entry, _, _, _ = vj.vj_export_graph(ix)
    eps = 3.0
    F = vj.vj_features(ix, eps)
    assert F.shape == (w.nq, vj.NFEAT + w.d)
    np.testing.assert_array_equal(F[:, vj.NFEAT:], w.Q)
    for q in range(0, w.nq, 7):
        node = w.nx + q
        flag, d1, d2 = oracle.ood(w.X, w.Q, adj, node)
        nb = [int(v) for v in adj[node] if 0 <= v < w.nx]
        dists = [oracle.dist(w.X[v], w.Q[q]) for v in nb]
        if nb:
            assert F[q, 0] == pytest.approx(min(d1 / eps, 100), rel=1e-4)
            assert F[q, 4] == pytest.approx(min(min(dists) / eps, 100), rel=1e-4)
            if not np.isnan(d2):
                assert F[q, 1] == pytest.approx(min(d2 / eps, 100), rel=1e-4)
                assert F[q, 2] == pytest.approx(min(d1 / d2, 100), rel=1e-4)
        assert F[q, 5] == pytest.approx(len(nb) / 12)
        assert F[q, 6] == pytest.approx(sum(dd < eps for dd in dists) / 12)
        de = oracle.dist(w.X[entry] if entry < w.nx else w.Q[entry - w.nx], w.Q[q])
        assert F[q, 3] == pytest.approx(min(de / eps, 100), rel=1e-4)
    ix.free()


def test_learned_join_reduces_to_route_all_and_bfs():
    """A predictor whose route logit is +large routes every query (the join
    then equals the exact join); one with a very negative route logit and a
    budget output of 1 (b = 2^1 - 2 = 0) runs BFS everywhere (the join equals
    the planless join without the rule); with a very negative budget output
    (b clamps to 2^0 - 2 = -1) no query expands (the join equals a plan of -1
    for every query)."""
    w = inputs.gauss_small(seed=32, nx=3000, nq=300, d=16, k=8)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=16, knn_k=32))
    din = vj.NFEAT + w.d
    m = vj.MLP(din, 16, 16, seed=0)
    n = m.num_params()
    eps = 2.5
    ex = vj.vj_join_exact(ix, eps)
    vj.vj_attach_predictor(ix, m, 0.5, 64)
    for route_bias, budget_head, expect in ((50.0, 1.0, "exact"), (-50.0, 1.0, "bfs"), (-50.0, -50.0, "none")):
        flat = np.zeros(n, np.float32)
        flat[-2] = budget_head    # 2^1 - 2 = 0: BFS; 2^0 - 2 = -1 (clamped): no expansion
        flat[-1] = route_bias     # route head
        m.set_params(flat)
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1, learned=1)
        r = vj.vj_join(ix, eps)
        assert r.stats["ms_prologue"] > 0
        if expect == "exact":
            assert np.array_equal(r.offsets, ex.offsets) and np.array_equal(r.ids, ex.ids)
            assert np.all(r.hybrid == 2)
        elif expect == "none":
            assert np.all(r.hybrid == 3)
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, learned=0)
            vj.vj_set_plan(ix, None, np.full(w.nq, -1, np.int32))
            b = vj.vj_join(ix, eps)
            vj.vj_set_plan(ix, None, None)
            assert np.array_equal(r.offsets, b.offsets) and np.array_equal(r.ids, b.ids)
            assert np.array_equal(r.steps, b.steps)
        else:
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, learned=0)
            b = vj.vj_join(ix, eps)
            assert np.array_equal(r.offsets, b.offsets) and np.array_equal(r.ids, b.ids)
            assert np.array_equal(r.steps, b.steps)
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    ix.free()
    m.free()


@pytest.mark.parametrize("h1,h2", [(256, 256), (64, 48), (16, 16)])
def test_prologue_forward_matches_fp64_oracle(oracle, h1, h2):
    """The join prologue's predictor forward (BF16 tensor cores for h1 % 64 ==
    0 and h2 % 16 == 0, FP32 otherwise) against the FP64 MLP oracle on the
    same features.  BF16 rounds inputs and weights to 2^-8 relative; with FP32
    accumulation the outputs stay within a few 2^-8 of the layer scales."""
    from oracle import mlp as omlp
    w = inputs.gauss_small(seed=33, nx=3000, nq=700, d=32, k=8, ood_frac=0.1, shift=8.0)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=16, knn_k=32))
    eps = 2.5
    F = vj.vj_features(ix, eps)
    din = F.shape[1]
    m = vj.MLP(din, h1, h2, seed=7)
    rng = np.random.default_rng(5)
    flat, _, _ = m.get_params()
    flat = flat + (rng.standard_normal(flat.size) * 0.02).astype(np.float32)  # non-zero biases
    mu = F.mean(0).astype(np.float32)
    sd = (F.std(0) + 1e-3).astype(np.float32)
    m.set_params(flat, mu, sd)
    vj.vj_attach_predictor(ix, m, 0.5, 64)
    y = vj.vj_predictor_outputs(ix, eps)
    xs = (F.astype(np.float32) - mu) / sd
    yref, _ = omlp.forward(flat.astype(np.float64), xs.astype(np.float64), din, h1, h2)
    scale = np.abs(yref).mean(0) + 1e-3
    if h1 % 64 == 0 and h2 % 16 == 0:
        # the same network with BF16-rounded inputs, weights and layer-1
        # activations (the tensor-core operands), evaluated in FP64: only the
        # FP32 accumulation order separates it from the GPU
        W1, b1, W2, b2, W3, b3 = omlp.unpack(flat, din, h1, h2)
        a1 = np.maximum(_bf16(xs) @ _bf16(W1).T + b1, 0.0)
        a2 = np.maximum(_bf16(a1) @ _bf16(W2).T + b2, 0.0)
        ybf = a2 @ W3.T + b3
        assert (np.abs(y - ybf) / scale).max() < 1e-3
        # and BF16 rounding itself stays within a few 2^-8 of the FP64 network
        assert (np.abs(y - yref) / scale).max() < 0.1
    else:
        assert (np.abs(y - yref) / scale).max() < 1e-4
    np.testing.assert_array_equal(y, vj.vj_predictor_outputs(ix, eps))  # deterministic
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    ix.free()
    m.free()


@pytest.mark.parametrize("epochs", [1, 2])
def test_adam_steps_match_fp64_oracle(epochs):
    """vj_mlp_train with one batch of all n rows takes one full-batch Adam step
    per epoch; each must equal the FP64 oracle's step (standardisation from the
    rows' mean and population std, gradient by the chain rule, Adam with bias
    correction) to FP32 rounding."""
    from oracle import mlp as omlp
    rng = np.random.default_rng(11)
    din, h1, h2, n = 9, 32, 24, 50
    x = (rng.standard_normal((n, din)) * 2 + 1).astype(np.float32)
    tr = rng.standard_normal(n).astype(np.float32)
    tc = (rng.random(n) < 0.5).astype(np.float32)
    m = vj.MLP(din, h1, h2, seed=6)
    th, _, _ = m.get_params()
    th = th.astype(np.float64)
    lr = 1e-2
    m.train(x, tr, tc, epochs=epochs, batch=n, lr=lr, seed=1)
    got, mu, sd = m.get_params()
    m.free()
    mu_o, sd_o, xs = omlp.standardise(x)
    np.testing.assert_allclose(mu, mu_o, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sd, sd_o, rtol=1e-6)
    mo = np.zeros_like(th)
    vo = np.zeros_like(th)
    grads = []
    for t in range(1, epochs + 1):
        _, g = omlp.loss_grad(th, xs, tr, tc, din, h1, h2)
        grads.append(g)
        th, mo, vo = omlp.adam_step(th, mo, vo, g, t, lr)
    # Where the gradient is far from zero the step is lr * sign-like and FP32
    # only rounds it; a gradient within FP32 noise of zero may take either
    # direction, so those entries are only checked to move at most epochs * lr.
    firm = np.all([np.abs(g) > 1e-4 * np.abs(g).max() for g in grads], axis=0)
    assert firm.mean() > 0.8
    np.testing.assert_allclose(got[firm], th[firm], rtol=0, atol=2e-6)


def test_forward_on_hand_worked_network():
    """The hand-worked 2-3-3-2 network of tests/golden/mlp_hand.json through
    the library's FP32 forward (vj_mlp_predict, no standardisation): the
    values are small integers and halves, exact in FP32."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mlp_hand.json")))
    flat = np.concatenate([np.ravel(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)
    m = vj.MLP(g["din"], g["h1"], g["h2"], seed=0)
    m.set_params(flat)
    y = m.predict(np.array(g["x"], np.float32))
    m.free()
    np.testing.assert_array_equal(y, np.array(g["y"], np.float32))
