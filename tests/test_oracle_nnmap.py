"""Pins of the NN-Map oracle (the next design of the paper, Sec. NN-Map) against
facts it must satisfy, each computed by independent code: the C oracle's
nested-loop join, connected components of the in-range subgraph (scipy), and
the complete graph.  Both the plain Python oracle and its C twin (for larger
inputs) are pinned, and they agree on every output."""
import numpy as np
import pytest

from oracle import nnmap

scipy_sparse = pytest.importorskip("scipy.sparse")


@pytest.fixture(params=["py", "c"])
def impl(request, oracle):
    if request.param == "py":
        return nnmap.nnmap_build, nnmap.nnmap_join
    return oracle.nnmap_build_c, oracle.nnmap_join_c


@pytest.fixture(scope="module")
def case(oracle):
    rng = np.random.default_rng(21)
    centres = rng.standard_normal((6, 12)) * 3.0
    X = (centres[rng.integers(0, 6, 600)] + rng.standard_normal((600, 12))).astype(np.float32)
    Qi = centres[rng.integers(0, 6, 70)] + rng.standard_normal((70, 12))
    Qo = centres[rng.integers(0, 6, 10)] + 6.0 + rng.standard_normal((10, 12))  # far from the data
    Q = np.concatenate([Qi, Qo]).astype(np.float32)
    adj_x, entry, _ = oracle.build_graph(X, np.zeros((0, 12), np.float32), 10, 20)
    return X, Q, adj_x, nnmap.nnmap_build(X, Q, adj_x)


def test_witness_property_for_every_threshold(case, oracle):
    """(i) dist[q] >= eps: the exact row is empty; (ii) otherwise w[q] is in the
    exact row and is its closest member (ties by id): the nested-loop join."""
    X, Q, adj_x, nm = case
    for eps in np.quantile(nm.wdist, [0.1, 0.4, 0.7, 0.95]) * np.array([1.0, 1.05, 1.2, 1.5]):
        off, ids, dd = oracle.nlj(X, Q, float(eps))
        for q in range(len(Q)):
            row, rd = ids[off[q]:off[q + 1]], dd[off[q]:off[q + 1]]
            if nm.wdist[q] >= eps:
                assert len(row) == 0
            else:
                assert nm.witness[q] in row
                k = int(np.argmin(rd))
                assert rd[k] == pytest.approx(nm.wdist[q], rel=1e-12)
                assert nm.witness[q] == min(int(row[j]) for j in range(len(row)) if rd[j] == rd[k])


def test_certified_empty_queries_compute_nothing(case, impl):
    X, Q, adj_x, nm = case
    eps = float(np.quantile(nm.wdist, 0.5))
    r = impl[1](X, Q, adj_x, nm, eps)
    empty = nm.wdist >= eps
    assert empty.any() and (~empty).any()
    assert np.all(r.steps[empty] == 0)
    assert all(len(r.row(q)) == 0 for q in np.nonzero(empty)[0])


def test_bfs_join_is_the_in_range_component_of_the_witness(case, impl):
    """Non-hybrid: the result is the connected component of w[q] in the
    subgraph of G_X induced by the in-range data nodes (order-independent)."""
    from scipy.sparse.csgraph import connected_components
    X, Q, adj_x, nm = case
    eps = float(np.quantile(nm.wdist, 0.6)) * 1.6
    r = impl[1](X, Q, adj_x, nm, eps, hybrid="off")
    nx, R = adj_x.shape
    src = np.repeat(np.arange(nx), R)
    dst = adj_x.ravel()
    ok = dst >= 0
    for q in range(len(Q)):
        d = np.sqrt(((X.astype(np.float64) - Q[q].astype(np.float64)) ** 2).sum(1))
        inr = d < eps
        keep = ok & inr[src] & inr[np.where(ok, dst, 0)]
        g = scipy_sparse.csr_matrix((np.ones(keep.sum()), (src[keep], dst[keep])), shape=(nx, nx))
        _, lab = connected_components(g, directed=True, connection="weak")
        if nm.wdist[q] >= eps:
            assert len(r.row(q)) == 0
            continue
        comp = np.nonzero((lab == lab[nm.witness[q]]) & inr)[0]
        # directed edges: the closure follows out-edges only; weak components
        # bound it from above, and the reachable set is checked exactly
        reach = {int(nm.witness[q])}
        stack = [int(nm.witness[q])]
        while stack:
            u = stack.pop()
            for v in adj_x[u]:
                if v >= 0 and inr[v] and int(v) not in reach:
                    reach.add(int(v))
                    stack.append(int(v))
        assert set(int(v) for v in r.row(q)) == reach
        assert reach <= set(int(v) for v in comp)


def test_complete_graph_join_equals_nested_loop_join(oracle, impl):
    rng = np.random.default_rng(22)
    X = rng.standard_normal((60, 6)).astype(np.float32)
    Q = rng.standard_normal((15, 6)).astype(np.float32)
    adj = np.array([[v for v in range(60) if v != u] for u in range(60)], np.int32)
    nm = impl[0](X, Q, adj)
    eps = float(np.quantile(nm.wdist, 0.8)) * 1.3
    r = impl[1](X, Q, adj, nm, eps, hybrid="off")
    off, ids, dd = oracle.nlj(X, Q, eps)
    for q in range(len(Q)):
        assert set(r.row(q).tolist()) == set(ids[off[q]:off[q + 1]].tolist())
    np.testing.assert_allclose(r.dists, dd, rtol=1e-12)


def test_hybrid_contains_bfs_and_rows_grow_with_eps(case, impl):
    X, Q, adj_x, nm = case
    e1 = float(np.quantile(nm.wdist, 0.5))
    e2 = e1 * 1.3
    b1 = impl[1](X, Q, adj_x, nm, e1, hybrid="off")
    b2 = impl[1](X, Q, adj_x, nm, e2, hybrid="off")
    h1 = impl[1](X, Q, adj_x, nm, e1, hybrid="force", hybrid_beam_size=16)
    for q in range(len(Q)):
        assert set(b1.row(q).tolist()) <= set(h1.row(q).tolist())
        assert set(b1.row(q).tolist()) <= set(b2.row(q).tolist())  # one build serves every threshold


def test_ood_bit_flags_far_queries(case):
    """The far-shifted queries (the last ten) are flagged far more often than
    the in-distribution ones, and the rule matches a hand computation."""
    X, Q, adj_x, nm = case
    assert nm.ood[70:].mean() > 0.5 and nm.ood[:70].mean() < 0.2
    q = 75
    d = np.sqrt(((X.astype(np.float64) - Q[q].astype(np.float64)) ** 2).sum(1))
    n1 = list(np.lexsort((np.arange(len(d)), d))[:adj_x.shape[1]])
    d1 = d[n1].mean()
    pairs = [np.sqrt(((X[v].astype(np.float64) - X[u].astype(np.float64)) ** 2).sum())
             for v in n1 for u in adj_x[v] if u >= 0 and u not in n1]
    assert nm.ood[q] == int(d1 / np.mean(pairs) > 1.5)


@pytest.mark.parametrize("metric", [0, 1])
def test_python_and_c_oracles_agree(oracle, metric):
    rng = np.random.default_rng(23 + metric)
    centres = rng.standard_normal((5, 10)) * 2.5
    X = (centres[rng.integers(0, 5, 400)] + rng.standard_normal((400, 10))).astype(np.float32)
    Q = np.concatenate([centres[rng.integers(0, 5, 40)] + rng.standard_normal((40, 10)),
                        centres[rng.integers(0, 5, 8)] + 5.0 + rng.standard_normal((8, 10))]).astype(np.float32)
    if metric == 1:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    adj_x, _, _ = oracle.build_graph(X, np.zeros((0, 10), np.float32), 8, 16, metric)
    a = nnmap.nnmap_build(X, Q, adj_x, metric)
    b = oracle.nnmap_build_c(X, Q, adj_x, metric)
    np.testing.assert_array_equal(a.witness, b.witness)
    np.testing.assert_allclose(a.wdist, b.wdist, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(a.ood, b.ood)
    eps = float(np.quantile(a.wdist, 0.7)) * 1.4
    for hyb, beam in (("off", 256), ("adapt", 256), ("force", 8)):
        ra = nnmap.nnmap_join(X, Q, adj_x, a, eps, metric=metric, hybrid=hyb, hybrid_beam_size=beam)
        rb = oracle.nnmap_join_c(X, Q, adj_x, b, eps, metric=metric, hybrid=hyb, hybrid_beam_size=beam)
        np.testing.assert_array_equal(ra.offsets, rb.offsets)
        np.testing.assert_array_equal(ra.ids, rb.ids)
        np.testing.assert_allclose(ra.dists, rb.dists, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(ra.steps, rb.steps)
        np.testing.assert_array_equal(ra.hybrid, rb.hybrid)
