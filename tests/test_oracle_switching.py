"""Query-data switching (the paper's discussion of large thresholds): the join
is symmetric, so it can run with the two sets' roles swapped and the pair list
transposed.  Pins: the transpose itself, the nested-loop join's symmetry, and
the switched approximate join's precision and its equality with the
nested-loop join on a complete graph."""
import numpy as np


def _pairs(off, ids):
    return {(q, int(x)) for q in range(len(off) - 1) for x in ids[off[q]:off[q + 1]]}


def test_transpose_round_trip(oracle):
    rng = np.random.default_rng(41)
    rows = [np.sort(rng.choice(30, rng.integers(0, 8), replace=False)) for _ in range(12)]
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    ids = np.concatenate(rows).astype(np.int32)
    d = rng.random(len(ids))
    t_off, t_ids, t_d = oracle.transpose_csr(off, ids, d, 30)
    assert _pairs(t_off, t_ids) == {(x, q) for q, x in _pairs(off, ids)}
    b_off, b_ids, b_d = oracle.transpose_csr(t_off, t_ids, t_d, 12)
    np.testing.assert_array_equal(b_off, off)
    np.testing.assert_array_equal(b_ids, ids)
    np.testing.assert_array_equal(b_d, d)


def test_nested_loop_join_is_symmetric(oracle):
    rng = np.random.default_rng(42)
    X = rng.standard_normal((300, 6)).astype(np.float32)
    Q = rng.standard_normal((40, 6)).astype(np.float32)
    off, ids, dd = oracle.nlj(X, Q, 1.5)
    off2, ids2, dd2 = oracle.nlj(Q, X, 1.5)
    t_off, t_ids, t_d = oracle.transpose_csr(off2, ids2, dd2, 40)
    np.testing.assert_array_equal(t_off, off)
    np.testing.assert_array_equal(t_ids, ids)
    np.testing.assert_allclose(t_d, dd, rtol=1e-12)


def test_switched_join_precision_and_complete_graph(oracle):
    rng = np.random.default_rng(43)
    centres = rng.standard_normal((4, 8)) * 2
    X = (centres[rng.integers(0, 4, 400)] + rng.standard_normal((400, 8))).astype(np.float32)
    Q = (centres[rng.integers(0, 4, 30)] + rng.standard_normal((30, 8))).astype(np.float32)
    eps = 2.2  # a large threshold: many pairs per query
    off, ids, _ = oracle.nlj(X, Q, eps)
    exact = _pairs(off, ids)
    s_off, s_ids, _ = oracle.join_switched(X, Q, eps, degree=12, knn_k=24, work_sharing=oracle.WS_SELF)
    got = _pairs(s_off, s_ids)
    assert got <= exact and len(got) > 0.5 * len(exact)
    # on a complete merged graph the switched join finds every pair
    n = 430
    adj = np.array([[v for v in range(n) if v != u] for u in range(n)], np.int32)
    r = oracle.join(Q, X, adj, 0, eps, work_sharing=oracle.WS_SELF)
    t_off, t_ids, _ = oracle.transpose_csr(r.offsets, r.ids, r.dists, 30)
    assert _pairs(t_off, t_ids) == exact
