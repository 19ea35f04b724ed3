"""Parity at the full benchmark size, in the launch configuration bench.py times.

Workload: sift_like, 1M data x 100K queries, d = 128 integers, degree 32,
K = 64, eps for a mean of 20 matches per query.  The CPU oracle cannot redo
the whole join at this size, so it checks outputs it can compute one by one:
  * kNN lists of sampled nodes (bit-exact ids, keys within 1e-5);
  * the MI+SWS join rows of whole MST subtrees (a query's result depends only
    on its MST ancestors and the graph), with visited counts, soft caches and
    hybrid flags equal;
  * exact-join rows and brute-force-routed rows of sampled queries against
    the nested-loop join (pair ids equal outside the |dist - eps| <= 1e-4 eps
    band).
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
    w = inputs.sift_like()
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    # eps for about 20 matches per query on 50 queries (any threshold would do:
    # the checks decide near-eps pairs in FP64 themselves)
    qs = w.Q[:50]
    d2 = (qs ** 2).sum(1)[:, None] + (w.X ** 2).sum(1)[None, :] - 2.0 * qs @ w.X.T
    k = int(w.target_matches * len(qs))
    eps = float(np.float32(np.sqrt(max(float(np.partition(d2.ravel(), k)[k]), 0.0))))
    yield w, ix, eps
    ix.free()


def _d64(w, q, x):
    a = w.Q[q].astype(np.float64)
    b = w.X[x].astype(np.float64)
    return float(np.sqrt(((a - b) ** 2).sum()))


def _row_diff_outside_band(w, q, got, exp, eps):
    diff = set(int(i) for i in got) ^ set(int(i) for i in exp)
    return [x for x in diff if abs(_d64(w, q, x) - eps) > BAND * eps]


def test_full_size_knn_rows_sampled(full, oracle):
    w, ix, eps = full
    ids, keys = vj.vj_export_knn(ix)
    n, K = ids.shape
    rng = np.random.default_rng(5)
    rows = np.sort(np.concatenate([rng.choice(w.nx, 16, replace=False), w.nx + rng.choice(w.nq, 8, replace=False)]))
    o_ids, o_d = oracle.knn_rows(w.X, w.Q, K, rows, w.metric)
    np.testing.assert_array_equal(ids[rows], o_ids)
    np.testing.assert_allclose(keys[rows], o_d ** 2, rtol=1e-5, atol=1e-6)


def test_full_size_join_subtrees_match_oracle(full, oracle):
    import bench
    w, ix, eps = full
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1)
    r = vj.vj_join(ix, eps)
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    sub = bench.sample_subtrees(parent, order, 300)
    assert 300 <= len(sub) <= 5000
    o = oracle.join(w.X, w.Q, adj, entry, np.float32(eps), metric=w.metric, work_sharing=oracle.WS_SOFT,
                    adapt_hybrid=True, order=sub, parent=parent, queries=sub)
    for q in sub:
        bad = _row_diff_outside_band(w, int(q), r.row(q), o.row(q), eps)
        assert not bad, f"query {q}: pairs {bad[:5]} differ"
    np.testing.assert_array_equal(r.steps[sub], o.steps[sub])
    np.testing.assert_array_equal(r.cache[sub], o.cache[sub])
    np.testing.assert_array_equal(r.hybrid[sub], o.hybrid[sub])


def test_full_size_exact_and_routed_rows_match_nlj(full, oracle):
    w, ix, eps = full
    rng = np.random.default_rng(6)
    sample = np.sort(rng.choice(w.nq, 40, replace=False))
    off, ids, _ = oracle.nlj(w.X, w.Q[sample], float(np.float32(eps)), w.metric)
    ex = vj.vj_join_exact(ix, eps)
    # the brute-force route as the learned step runs it: about 10 % of the queries
    route = (rng.random(w.nq) < 0.1).astype(np.uint8)
    route[sample] = 1
    vj.vj_set_plan(ix, route=route)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1)
    r = vj.vj_join(ix, eps)
    vj.vj_set_plan(ix, route=np.zeros(w.nq, np.uint8))
    assert int((r.hybrid == 2).sum()) == int(route.sum())
    nonempty = 0
    worst = 0.0
    for k, q in enumerate(sample):
        exp = ids[off[k]:off[k + 1]]
        nonempty += len(exp) > 0
        bad = _row_diff_outside_band(w, int(q), ex.row(q), exp, eps)
        assert not bad, f"exact join, query {q}: pairs {bad[:5]} differ"
        bad = _row_diff_outside_band(w, int(q), r.row(q), exp, eps)
        assert not bad, f"routed row, query {q}: pairs {bad[:5]} differ"
        assert np.all(np.diff(r.row(q)) > 0)  # ascending data ids
        # returned distances against FP64
        for res in (ex, r):
            lo, hi = res.offsets[q], res.offsets[q + 1]
            for x, dv in zip(res.ids[lo:hi], res.dists[lo:hi]):
                ref = _d64(w, int(q), int(x))
                worst = max(worst, abs(float(dv) - ref) / max(ref, 1e-30))
    assert nonempty >= 20
    assert worst <= 1e-5, worst
