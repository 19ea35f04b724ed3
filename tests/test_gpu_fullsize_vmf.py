"""Parity at the full size of the learned-predictor workload, in the launch
configuration bench.py times.

Workload: vmf_like, 10M data x 1M evaluated + 100K held-out queries, d = 768
BF16-exact unit vectors, cosine, degree 32, K = 64, eps for about 10 matches per
query.  The index is built from device inputs, as the bench builds it.  The
CPU oracle checks outputs it can compute one by one:
  * kNN lists of sampled nodes (ids bit-exact, keys within 1e-5): the streamed
    tensor-core sweeps, the approximate-key prefilter and the FP64 prefix;
  * the join rows of whole MST subtrees in the learned step's configuration
    (every query planned with no expansion, BF16 gathers, soft sharing) and in
    the plain arm's (the d1/d2 rule, FP32 gathers), with visited counts, soft
    caches and flags equal;
  * exact-join rows of sampled queries against the nested-loop join (pair ids
    equal outside the |dist - eps| <= 1e-4 eps band, distances within 1e-5).
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu

BAND = 1e-4


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()
    w = inputs.vmf_like(device="cuda")
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    # eps for about 10 matches per query on 50 queries (any threshold would do:
    # the checks decide near-eps pairs in FP64 themselves)
    qs = w.Q[:50].double()
    qs = qs / qs.norm(dim=1, keepdim=True)
    best = []
    for a in range(0, w.nx, 1 << 20):
        xs = w.X[a:a + (1 << 20)].double()
        xs = xs / xs.norm(dim=1, keepdim=True)
        best.append(torch.topk(qs @ xs.T, 20, dim=1).values)
    sims = torch.topk(torch.cat(best, 1).flatten(), 10 * 50).values
    eps = float(np.float32(1.0 - float(sims[-1])))
    Xh, Qh = w.X.cpu().numpy(), w.Q.cpu().numpy()
    yield w, ix, eps, Xh, Qh
    ix.free()


def _d64(Xh, Qh, q, x):
    a = Qh[q].astype(np.float64)
    b = Xh[x].astype(np.float64)
    return float(1.0 - a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _row_diff_outside_band(Xh, Qh, q, got, exp, eps):
    diff = set(int(i) for i in got) ^ set(int(i) for i in exp)
    return [x for x in diff if abs(_d64(Xh, Qh, q, x) - eps) > BAND * eps]


def test_full_size_vmf_knn_rows_sampled(full, oracle):
    w, ix, eps, Xh, Qh = full
    info = ix.build_info()
    assert info["knn_tensor_cores"] and info["knn_uncertified"] == 0, info
    ids, keys = vj.vj_export_knn(ix)
    n, K = ids.shape
    rng = np.random.default_rng(7)
    rows = np.sort(np.concatenate([rng.choice(w.nx, 2, replace=False), w.nx + rng.choice(w.nq, 2, replace=False)]))
    o_ids, o_d = oracle.knn_rows(Xh, Qh, K, rows, w.metric)
    np.testing.assert_array_equal(ids[rows], o_ids)
    np.testing.assert_allclose(keys[rows], o_d, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("arm", ["learned", "plain"])
def test_full_size_vmf_join_subtrees_match_oracle(full, oracle, arm):
    import bench
    w, ix, eps, Xh, Qh = full
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    sub = bench.sample_subtrees(parent, order, 300)
    assert 300 <= len(sub) <= 20000
    if arm == "learned":
        plan = np.full(w.nq, -1, np.int32)
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, gather=vj.VJ_PREC_BF16)
        vj.vj_set_plan(ix, None, plan)
        kw = dict(beam=plan)
    else:
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1, gather=vj.VJ_PREC_FP32)
        kw = dict(adapt_hybrid=True)
    try:
        r = vj.vj_join(ix, eps)
    finally:
        vj.vj_set_plan(ix, None, None)
    o = oracle.join(Xh, Qh, adj, entry, np.float32(eps), metric=w.metric, work_sharing=oracle.WS_SOFT,
                    order=sub, parent=parent, queries=sub, **kw)
    for q in sub:
        bad = _row_diff_outside_band(Xh, Qh, int(q), r.row(q), o.row(q), eps)
        assert not bad, f"{arm}, query {q}: pairs {bad[:5]} differ"
    np.testing.assert_array_equal(r.steps[sub], o.steps[sub])
    np.testing.assert_array_equal(r.cache[sub], o.cache[sub])
    np.testing.assert_array_equal(r.hybrid[sub], o.hybrid[sub])
    assert sum(len(r.row(q)) for q in sub) > 0


def test_full_size_vmf_exact_rows_match_nlj(full, oracle):
    w, ix, eps, Xh, Qh = full
    rng = np.random.default_rng(8)
    sample = np.sort(rng.choice(w.nq - w.nh, 4, replace=False))
    off, ids, _ = oracle.nlj(Xh, Qh[sample], float(np.float32(eps)), w.metric)
    ex = vj.vj_join_exact(ix, eps)
    nonempty, worst = 0, 0.0
    for k, q in enumerate(sample):
        exp = ids[off[k]:off[k + 1]]
        nonempty += len(exp) > 0
        bad = _row_diff_outside_band(Xh, Qh, int(q), ex.row(q), exp, eps)
        assert not bad, f"exact join, query {q}: pairs {bad[:5]} differ"
        lo, hi = ex.offsets[q], ex.offsets[q + 1]
        for x, dv in zip(ex.ids[lo:hi], ex.dists[lo:hi]):
            ref = _d64(Xh, Qh, int(q), int(x))
            worst = max(worst, abs(float(dv) - ref) / max(ref, 1e-30))
    assert nonempty >= 2
    assert worst <= 1e-5, worst
