"""Pins of the CPU oracle against facts other than itself.

Each test checks the oracle against one of: an independent library routine
(scipy/numpy distance matrices, scipy's MST), a closed form of what the method
must return (the in-range closure of a non-hybrid merged-index join, exactness
on a complete graph), a theorem (App. C: RNG pruning keeps a node's nearest
neighbour; the RNG is contained in the pruned graph when every node is a
candidate), invariants (symmetry, zero self-distance, monotonicity in eps, the
strict `<` of Def. 1), or hand-traced tiny cases (tests/golden/).
"""
import json
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import minimum_spanning_tree
from scipy.spatial.distance import cdist

from paper_2603_16360_b300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_traced.json")


def _pairs(offsets, ids):
    return {(q, int(i)) for q in range(len(offsets) - 1) for i in ids[offsets[q]:offsets[q + 1]]}


# ---------------------------------------------------------------- distances
@pytest.mark.parametrize("metric,name", [(0, "euclidean"), (1, "cosine")])
def test_dist_matches_scipy(oracle, metric, name):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((20, 17)).astype(np.float32)
    B = rng.standard_normal((15, 17)).astype(np.float32)
    ref = cdist(A.astype(np.float64), B.astype(np.float64), name)
    got = np.array([[oracle.dist(a, b, metric) for b in B] for a in A])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    # symmetry and zero self-distance
    for a in A[:5]:
        assert oracle.dist(a, a, metric) == pytest.approx(0.0, abs=1e-12)
        for b in B[:5]:
            assert oracle.dist(a, b, metric) == oracle.dist(b, a, metric)


# ---------------------------------------------------------------- NLJ
@pytest.mark.parametrize("metric,name", [(0, "euclidean"), (1, "cosine")])
def test_nlj_brute_force(oracle, metric, name):
    w = inputs.uniform_small(3, 200, 30, 9, metric=metric)
    D = cdist(w.Q.astype(np.float64), w.X.astype(np.float64), name)
    eps = float(np.quantile(D, 0.05))
    off, ids, dd = oracle.nlj(w.X, w.Q, eps, metric)
    exp = {(q, x) for q in range(w.nq) for x in range(w.nx) if D[q, x] < eps}
    assert _pairs(off, ids) == exp
    np.testing.assert_allclose(dd, D[np.repeat(np.arange(w.nq), np.diff(off)), ids], rtol=1e-12)
    # ids ascending within each row
    for q in range(w.nq):
        r = ids[off[q]:off[q + 1]]
        assert np.all(np.diff(r) > 0)


def test_nlj_strict_less_than(oracle):
    # 3-4-5 triangle: dist exactly 5; Def. 1 uses a strict inequality
    X = np.array([[3.0, 4.0], [0.0, 1.0]], np.float32)
    Q = np.array([[0.0, 0.0]], np.float32)
    off, ids, _ = oracle.nlj(X, Q, 5.0)
    assert list(ids) == [1]
    off, ids, _ = oracle.nlj(X, Q, 5.0000001)
    assert list(ids) == [0, 1]


def test_nlj_monotone_in_eps(oracle):
    w = inputs.gauss_small(seed=7, nx=400, nq=40, d=8)
    prev = set()
    for eps in [0.5, 1.0, 1.5, 2.0, 3.0]:
        off, ids, _ = oracle.nlj(w.X, w.Q, eps)
        cur = _pairs(off, ids)
        assert prev <= cur
        prev = cur


def test_recall_exact_is_one(oracle):
    w = inputs.gauss_small(seed=8, nx=300, nq=30, d=8)
    off, ids, _ = oracle.nlj(w.X, w.Q, 2.0)
    assert oracle.recall(off, ids, off, ids) == (1.0, 1.0)


# ---------------------------------------------------------------- kNN
def test_knn_brute_force_with_id_ties(oracle):
    rng = np.random.default_rng(4)
    X = rng.integers(0, 3, size=(60, 3)).astype(np.float32)  # many exact ties
    Q = rng.integers(0, 3, size=(20, 3)).astype(np.float32)
    V = np.concatenate([X, Q]).astype(np.float64)
    D = cdist(V, V)
    K = 7
    rows = np.arange(len(V))
    ids, dd = oracle.knn_rows(X, Q, K, rows)
    for u in rows:
        cand = [v for v in range(len(V)) if v != u]
        exp = sorted(cand, key=lambda v: (D[u, v], v))[:K]
        assert list(ids[u]) == exp
        np.testing.assert_allclose(dd[u], D[u, exp], rtol=1e-12)


# ---------------------------------------------------------------- graph build
def test_rng_prune_keeps_nearest_app_c(oracle):
    """App. C: under RNG pruning a node's nearest node stays its neighbour."""
    w = inputs.uniform_small(5, 150, 30, 6)
    K, R = 16, 8
    n = w.nx + w.nq
    knn, _ = oracle.knn_rows(w.X, w.Q, K, np.arange(n))
    adj, entry, pruned = oracle.build_graph(w.X, w.Q, R, K, knn_ids=knn)
    assert np.all(pruned[:, 0] == knn[:, 0])
    assert np.all(adj[:, 0] == knn[:, 0])


def test_rng_contained_in_full_candidate_prune(oracle):
    """With every node a candidate and no degree cap, the pruned lists contain
    every relative-neighbourhood-graph edge (brute-force lune test)."""
    w = inputs.uniform_small(6, 40, 10, 3)
    n = w.nx + w.nq
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(V, V)
    adj, entry, pruned = oracle.build_graph(w.X, w.Q, R=n - 1, K=n - 1)
    for u in range(n):
        kept = set(int(v) for v in pruned[u] if v >= 0)
        for v in range(n):
            if v == u:
                continue
            in_lune = any(D[u, x] < D[u, v] and D[v, x] < D[u, v] for x in range(n) if x not in (u, v))
            if not in_lune:
                assert v in kept, (u, v)


def test_pruned_lists_obey_rule(oracle):
    """Every kept pair respects the rule; every rejected candidate (before the
    cap) has a kept witness closer to it than the node is."""
    w = inputs.uniform_small(9, 120, 20, 5)
    K, R = 12, 6
    n = w.nx + w.nq
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(V, V)
    knn, _ = oracle.knn_rows(w.X, w.Q, K, np.arange(n))
    _, _, pruned = oracle.build_graph(w.X, w.Q, R, K, knn_ids=knn)
    for u in range(n):
        kept = [int(v) for v in pruned[u] if v >= 0]
        for i, v in enumerate(kept):
            for wv in kept[:i]:
                assert not D[wv, v] < D[u, v]
        if len(kept) < R:
            for v in knn[u]:
                if v in kept:
                    continue
                assert any(D[wv, v] < D[u, v] for wv in kept)


def test_graph_lists_sorted_and_reverse_edges(oracle):
    w = inputs.uniform_small(10, 150, 30, 6)
    K, R = 16, 8
    n = w.nx + w.nq
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(V, V)
    adj, entry, pruned = oracle.build_graph(w.X, w.Q, R, K)
    for u in range(n):
        lst = [int(v) for v in adj[u] if v >= 0]
        keys = [(D[u, v], v) for v in lst]
        assert keys == sorted(keys)
        assert len(set(lst)) == len(lst) and u not in lst
        # adj(u) is drawn from pruned(u) U reverse offers
        offers = set(int(v) for v in pruned[u] if v >= 0) | {x for x in range(n) if u in pruned[x]}
        assert set(lst) <= offers
        if len(offers) <= R:
            assert set(lst) == offers
    # entry = node closest to the centroid
    c = V.mean(axis=0)
    dc = np.linalg.norm(V - c, axis=1)
    assert entry == int(np.lexsort((np.arange(n), dc))[0])


# ---------------------------------------------------------------- MST
def _query_graph(w, adj, entry):
    nx, nq = w.nx, w.nq
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    edges = {}
    for qi in range(nq):
        u = nx + qi
        for v in adj[u]:
            if v >= nx and v != u:
                a, b = sorted((u, int(v)))
                edges[(a, b)] = np.linalg.norm(V[a] - V[b])
        if u != entry:
            a, b = sorted((u, entry))
            edges[(a, b)] = np.linalg.norm(V[a] - V[b])
    return edges


@pytest.mark.parametrize("seed", [11, 12])
def test_mst_matches_scipy_and_is_topological(oracle, seed):
    w = inputs.gauss_small(seed=seed, nx=300, nq=120, d=6, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    parent, order, depth, total = oracle.mst(w.X, w.Q, adj, entry)
    edges = _query_graph(w, adj, entry)
    nodes = sorted({entry} | {w.nx + q for q in range(w.nq)})
    idx = {v: i for i, v in enumerate(nodes)}
    r = [idx[a] for a, b in edges]
    c = [idx[b] for a, b in edges]
    m = coo_matrix((list(edges.values()), (r, c)), shape=(len(nodes), len(nodes))).tocsr()
    ref = minimum_spanning_tree(m).sum()
    assert total == pytest.approx(ref, rel=1e-12)
    # every query placed once; parent placed before child; tree edges exist
    assert sorted(order) == list(range(w.nq))
    pos = {int(q): i for i, q in enumerate(order)}
    for q in range(w.nq):
        p = int(parent[q])
        u = w.nx + q
        if p >= 0:
            assert pos[p] < pos[q]
            assert tuple(sorted((u, w.nx + p))) in edges
            assert depth[q] == depth[p] + 1
        elif u != entry:
            assert depth[q] == 1 and tuple(sorted((u, entry))) in edges


# ---------------------------------------------------------------- OOD rule
def test_ood_hand_computed(oracle):
    g = json.load(open(GOLD))["ood"]
    X = np.array(g["X"], np.float32)
    Q = np.array(g["Q"], np.float32)
    adj = np.array(g["adj"], np.int32)
    for e in g["expect"]:
        f, d1, d2 = oracle.ood(X, Q, adj, e["node"])
        assert f == e["ood"], e
        if e["d1"] is None:
            assert np.isnan(d1)
        else:
            assert d1 == pytest.approx(e["d1"], rel=1e-7)
        if e["d2"] is None:
            assert np.isnan(d2)
        else:
            assert d2 == pytest.approx(e["d2"], rel=1e-7)


# ---------------------------------------------------------------- join
@pytest.mark.parametrize("case", json.load(open(GOLD))["cases"], ids=lambda c: c["name"])
def test_join_hand_traced(oracle, case):
    X = np.array(case["X"], np.float32)
    Q = np.array(case["Q"], np.float32)
    adj = np.array(case["adj"], np.int32)
    for run in case["runs"]:
        r = oracle.join(X, Q, adj, case["entry"], case["eps"], work_sharing=oracle.WS_SELF,
                        force_hybrid=bool(run["force_hybrid"]), hybrid_beam_size=run["hybrid_beam_size"])
        assert list(r.row(0)) == run["ids"], run
        assert int(r.steps[0]) == run["steps"], run
        assert int(r.expansions[0]) == run["expansions"], run
        assert int(r.cache[0]) == run["cache"], run


def _closure_expected(w, adj, entry, eps, D, seeds_of):
    """Closed form of the non-hybrid merged-index join for one query.

    I0 = in-range data nodes among the seeds and q's neighbours; the result is
    every data node reachable from I0 along graph edges whose endpoints are all
    in-range data nodes; V = seeds U N(q) U data neighbours of result nodes.
    """
    nx = w.nx
    out = {}
    for qi, seeds in seeds_of:
        u = nx + qi
        dq = D[qi]
        probe = set(seeds) | {u} | {int(v) for v in adj[u] if v >= 0}
        res = {v for v in probe if v < nx and dq[v] < eps}
        stack = list(res)
        while stack:
            a = stack.pop()
            for v in adj[a]:
                v = int(v)
                if 0 <= v < nx and dq[v] < eps and v not in res:
                    res.add(v)
                    stack.append(v)
        visited = set(probe)
        for a in res:
            visited |= {int(v) for v in adj[a] if 0 <= v < nx}
        data_vis = [v for v in visited if v < nx]
        best = min(data_vis, key=lambda v: (dq[v], v)) if data_vis else -1
        out[qi] = (res, len(visited), best)
    return out


@pytest.mark.parametrize("metric", [0, 1])
def test_mi_self_join_equals_closed_form(oracle, metric):
    w = inputs.uniform_small(13, 400, 60, 5, metric=metric) if metric else inputs.gauss_small(seed=13, nx=400, nq=60, d=5, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16, metric=metric)
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(w.Q.astype(np.float64), V, "euclidean" if metric == 0 else "cosine")
    eps = float(np.quantile(D[:, :w.nx], 0.03))
    r = oracle.join(w.X, w.Q, adj, entry, eps, metric=metric, work_sharing=oracle.WS_SELF)
    exp = _closure_expected(w, adj, entry, eps, D, [(q, [entry]) for q in range(w.nq)])
    for q in range(w.nq):
        res, nvis, best = exp[q]
        assert set(int(i) for i in r.row(q)) == res
        assert int(r.steps[q]) == nvis
        assert int(r.cache[q]) == best


@pytest.mark.parametrize("metric", [0, 1])
def test_no_expansion_plan_equals_probe_closed_form(oracle, metric):
    """Plan -1 (an expansion budget of zero): the row is I after the greedy
    phase, i.e. the in-range data nodes among {entry, q} U N(q), the visited
    count is |{entry, q} U N(q)| and the cache the closest of those data
    nodes; plan 0 queries in the same join keep the full closure."""
    w = inputs.uniform_small(15, 400, 60, 5, metric=metric) if metric else inputs.gauss_small(seed=15, nx=400, nq=60, d=5, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16, metric=metric)
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(w.Q.astype(np.float64), V, "euclidean" if metric == 0 else "cosine")
    eps = float(np.quantile(D[:, :w.nx], 0.03))
    beam = np.where(np.arange(w.nq) % 2 == 0, -1, 0).astype(np.int32)
    r = oracle.join(w.X, w.Q, adj, entry, eps, metric=metric, work_sharing=oracle.WS_SELF, beam=beam)
    full = _closure_expected(w, adj, entry, eps, D, [(q, [entry]) for q in range(w.nq)])
    grew = 0
    for q in range(w.nq):
        if beam[q] == 0:
            res, nvis, best = full[q]
            assert int(r.hybrid[q]) == 0
        else:
            u = w.nx + q
            probe = {entry, u} | {int(v) for v in adj[u] if v >= 0}
            res = {v for v in probe if v < w.nx and D[q][v] < eps}
            nvis = len(probe)
            data = [v for v in probe if v < w.nx]
            best = min(data, key=lambda v: (D[q][v], v)) if data else -1
            assert int(r.hybrid[q]) == 3
            grew += len(full[q][0]) > len(res)
        assert set(int(i) for i in r.row(q)) == res
        assert int(r.steps[q]) == nvis
        assert int(r.cache[q]) == best
    assert grew > 0  # the closure adds points on some of these queries


def test_mi_sws_join_equals_closed_form(oracle):
    w = inputs.gauss_small(seed=14, nx=500, nq=80, d=5, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    parent, order, depth, _ = oracle.mst(w.X, w.Q, adj, entry)
    V = np.concatenate([w.X, w.Q]).astype(np.float64)
    D = cdist(w.Q.astype(np.float64), V)
    eps = float(np.quantile(D[:, :w.nx], 0.02))
    r = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SOFT, order=order, parent=parent)
    # walk the tree in order, feeding each parent's closed-form cache to its children
    cache = {}
    for q in order:
        q = int(q)
        p = int(parent[q])
        seeds = [entry] + ([cache[p]] if p >= 0 and cache[p] >= 0 else [])
        res, nvis, best = _closure_expected(w, adj, entry, eps, D, [(q, seeds)])[q]
        cache[q] = best
        assert set(int(i) for i in r.row(q)) == res, q
        assert int(r.steps[q]) == nvis
        assert int(r.cache[q]) == best
    assert depth.max() >= 1


def test_complete_graph_join_is_exact(oracle):
    """On the complete graph every in-range point is a neighbour of q, so the
    merged-index join must return the exact NLJ result."""
    w = inputs.uniform_small(15, 60, 12, 4)
    n = w.nx + w.nq
    adj = np.array([[v for v in range(n) if v != u] for u in range(n)], np.int32)
    off, ids, _ = oracle.nlj(w.X, w.Q, 1.5)
    for hyb in (False, True):
        r = oracle.join(w.X, w.Q, adj, 0, 1.5, work_sharing=oracle.WS_SELF, force_hybrid=hyb)
        assert _pairs(r.offsets, r.ids) == _pairs(off, ids)


def test_mi_self_monotone_in_eps(oracle):
    w = inputs.gauss_small(seed=16, nx=400, nq=50, d=6, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    prev = set()
    for eps in [1.0, 1.5, 2.0, 2.5, 3.0]:
        r = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF)
        cur = _pairs(r.offsets, r.ids)
        assert prev <= cur
        prev = cur


def test_hybrid_superset_of_bfs_and_beam_monotone_on_average(oracle):
    w = inputs.gauss_small(seed=17, nx=600, nq=60, d=6, k=4, ood_frac=0.3, shift=6.0)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    off, ids, _ = oracle.nlj(w.X, w.Q, 2.0)
    base = oracle.join(w.X, w.Q, adj, entry, 2.0, work_sharing=oracle.WS_SELF)
    rec = []
    for beam in [0, 4, 16, 64, 256]:
        r = oracle.join(w.X, w.Q, adj, entry, 2.0, work_sharing=oracle.WS_SELF, force_hybrid=True,
                        hybrid_beam_size=beam)
        # hybrid only adds out-range bridges; the BFS closure is always found
        assert _pairs(base.offsets, base.ids) <= _pairs(r.offsets, r.ids)
        rec.append(oracle.recall(r.offsets, r.ids, off, ids)[0])
        if beam == 0:
            assert _pairs(r.offsets, r.ids) == _pairs(base.offsets, base.ids)
    assert rec[-1] >= rec[0]


def test_ws_none_merged_stops_at_entry(oracle):
    """Merged index without self seeding: StopGreedy's third rule fires on the
    entry at the first check, so only the entry's own in-range closure remains."""
    w = inputs.gauss_small(seed=18, nx=300, nq=30, d=5, k=4)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    r = oracle.join(w.X, w.Q, adj, entry, 2.0, work_sharing=oracle.WS_NONE)
    for q in range(w.nq):
        ds = oracle.dist(w.X[entry] if entry < w.nx else w.Q[entry - w.nx], w.Q[q])
        if not (entry < w.nx and ds < 2.0):
            assert len(r.row(q)) == 0
            assert r.steps[q] == 1


def test_adapt_flags_shifted_queries(oracle):
    """Sec. 4.4 trend: in-distribution queries are rarely flagged OOD, queries
    from a far-shifted mixture mostly are."""
    w = inputs.gauss_small(seed=19, nx=2000, nq=200, d=16, k=8, ood_frac=0.25, shift=12.0)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 12, 24)
    flags = np.array([oracle.ood(w.X, w.Q, adj, w.nx + q)[0] for q in range(w.nq)])
    assert flags[~w.ood].mean() < 0.1
    assert flags[w.ood].mean() > 0.6


# ---------------------------------------------------------------- per-query plan
def test_plan_reduces_to_paper_modes_and_nlj(oracle):
    """A per-query plan (route to brute force / hybrid beam) must reduce to the
    paper's modes: all-zero beams = BFS, all-b beams = forced hybrid with beam b,
    routed rows = the NLJ rows; a mixed plan (self seeding, no cross-query
    dependency) equals each query's uniform-mode row."""
    w = inputs.gauss_small(seed=21, nx=500, nq=60, d=6, k=4, ood_frac=0.3, shift=6.0)
    adj, entry, _ = oracle.build_graph(w.X, w.Q, 8, 16)
    eps = 2.0
    nq = w.nq
    bfs = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF)
    hyb8 = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF, force_hybrid=True, hybrid_beam_size=8)
    off, ids, _ = oracle.nlj(w.X, w.Q, eps)
    p0 = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF, beam=np.zeros(nq, np.int32))
    p8 = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF, beam=np.full(nq, 8, np.int32))
    pr = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF, route=np.ones(nq, np.uint8))
    assert _pairs(p0.offsets, p0.ids) == _pairs(bfs.offsets, bfs.ids)
    assert np.array_equal(p0.steps, bfs.steps)
    assert _pairs(p8.offsets, p8.ids) == _pairs(hyb8.offsets, hyb8.ids)
    assert np.array_equal(p8.steps, hyb8.steps)
    assert _pairs(pr.offsets, pr.ids) == _pairs(off, ids)
    assert np.all(pr.hybrid == 2)
    # routed queries only run the greedy phase: their visited set is the probe
    probe_only = oracle.join(w.X, w.Q, adj, entry, 1e-9, work_sharing=oracle.WS_SELF)
    assert np.array_equal(pr.steps, probe_only.steps)
    rng = np.random.default_rng(3)
    route = (rng.random(nq) < 0.3).astype(np.uint8)
    beam = np.where(rng.random(nq) < 0.5, 8, 0).astype(np.int32)
    mix = oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SELF, route=route, beam=beam)
    for q in range(nq):
        ref = pr if route[q] else (p8 if beam[q] else p0)
        assert list(mix.row(q)) == list(ref.row(q)), q
