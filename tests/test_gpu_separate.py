"""Separate (per-set) indexes (Sec. 3.2: INLJ, HWS and SWS on the data graph
G_Y) on the GPU, through the C ABI, against the oracle on the same seeded
inputs.  Each stage is fed the GPU's output of the stage before:
  * kNN lists rank the row's own set only: ids bit-exact against the
    oracle's exact lists over that set (ties by id), keys within 1e-5;
  * data rows of the graph bit-exact against the oracle's graph build on the
    data set alone, query rows against its build on the query set alone,
    entry s_Y equal; the MST order and parents equal ``oracle.separate_mst``;
  * joins (INLJ, hard and soft sharing; BFS and forced hybrid expansion;
    several greedy queue sizes and convergence thresholds): result rows equal
    outside the |dist - eps| <= 1e-4 eps band, distance evaluations, hybrid
    flags and soft caches equal to ``oracle.join(separate=True)``'s.
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu

BAND = 1e-4


@pytest.fixture(scope="session", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()


CASES = {
    # fewer than 4096 queries: the FP32 SIMT kNN sweep for both sets
    "gauss_d32_simt": lambda: inputs.gauss_small(seed=301, nx=3000, nq=500, d=32),
    # both sets past 4096: BF16 tensor-core kNN, resident tiles, one block per set
    "gauss_d32_tc": lambda: inputs.gauss_small(seed=302, nx=6000, nq=4200, d=32),
    "cosine_d20_tc": lambda: inputs.uniform_small(303, 5000, 4200, 20, metric=1, degree=16, knn_k=32),
    # streamed tiles: a symmetric sweep per set
    "wide_l2_d300": lambda: inputs.uniform_small(304, 4500, 4200, 300, degree=12, knn_k=24),
}


def _build(w):
    p = vj.default_params(degree=w.degree, knn_k=w.knn_k)
    return vj.vj_build(w.X, w.Q, metric=w.metric, params=p, separate=1)


@pytest.fixture(scope="module", params=list(CASES))
def built(request):
    w = CASES[request.param]()
    ix = _build(w)
    yield request.param, w, ix
    ix.free()


def _calib_eps(w, matches, sample=200):
    from scipy.spatial.distance import cdist
    D = cdist(w.Q[:sample].astype(np.float64), w.X.astype(np.float64), "euclidean" if w.metric == 0 else "cosine")
    k = int(matches * min(sample, len(w.Q)))
    return float(np.partition(D.ravel(), k)[k])


def _band_pairs(w, eps):
    from scipy.spatial.distance import cdist
    D = cdist(w.Q.astype(np.float64), w.X.astype(np.float64), "euclidean" if w.metric == 0 else "cosine")
    qs, xs = np.nonzero(np.abs(D - eps) <= BAND * eps)
    return set(zip(qs.tolist(), xs.tolist()))


def _assert_steps(name, r, o):
    """Distance evaluations equal the oracle's.  The known exception is the
    hybrid expansion's pop order (FP32 keys on the GPU, FP64 in the oracle):
    a hybrid search that walks most of the data set (thousands of
    evaluations per query) meets FP32 near-ties, and one flipped pop changes
    its count.  A hybrid query may then differ, on at most 0.5 % of the
    queries, while its result row and cache still equal the oracle's
    (checked by the caller)."""
    bad = np.nonzero(r.steps != o.steps)[0]
    if 0 < len(bad) <= max(1, len(r.steps) // 200) and np.all(r.hybrid[bad] == 1):
        return
    # (under soft sharing a differing cache passes the difference to the
    # query's MST descendants, which are hybrid as well and counted above)
    np.testing.assert_array_equal(r.steps, o.steps, err_msg=name)


def _pairs(off, ids):
    return {(q, int(i)) for q in range(len(off) - 1) for i in ids[off[q]:off[q + 1]]}


def _local(a, base):
    return np.where(a >= 0, a - base, -1).astype(np.int32)


def test_knn_lists_rank_own_set(built, oracle):
    name, w, ix = built
    ids, keys = vj.vj_export_knn(ix)
    K = ids.shape[1]
    assert np.all((ids[:w.nx] >= 0) & (ids[:w.nx] < w.nx)), name
    assert np.all(ids[w.nx:] >= w.nx), name
    for base, S, n in ((0, w.X, w.nx), (w.nx, w.Q, w.nq)):
        rows = np.arange(0, n, 5)
        o_ids, o_d = oracle.knn_rows(S, S[:0], K, rows, w.metric)
        got = _local(ids[base + rows], base)
        mism = np.nonzero((got != o_ids).any(axis=1))[0]
        assert len(mism) == 0, f"{name}: {len(mism)} rows of the set at {base} differ, first {rows[mism[:5]]}"
        ref = o_d ** 2 if w.metric == 0 else o_d
        np.testing.assert_allclose(keys[base + rows], ref, rtol=1e-5, atol=1e-6)


def test_graphs_entry_and_mst_match_oracle(built, oracle):
    name, w, ix = built
    kn, _ = vj.vj_export_knn(ix)
    adj, entry, parent, order, depth = vj.vj_export_graph(ix)
    R, K = adj.shape[1], kn.shape[1]
    gy, ey, _ = oracle.build_graph(w.X, w.X[:0], R, K, w.metric, knn_ids=kn[:w.nx])
    assert entry == ey, name
    mism = np.nonzero((adj[:w.nx] != gy).any(axis=1))[0]
    assert len(mism) == 0, f"{name}: {len(mism)} G_Y rows differ, first {mism[:5]}"
    gq, _, _ = oracle.build_graph(w.Q, w.Q[:0], R, K, w.metric, knn_ids=_local(kn[w.nx:], w.nx))
    adj_q = _local(adj[w.nx:], w.nx)
    mism = np.nonzero((adj_q != gq).any(axis=1))[0]
    assert len(mism) == 0, f"{name}: {len(mism)} query-graph rows differ, first {mism[:5]}"
    o_par, _, o_depth, _ = oracle.separate_mst(w.X, w.Q, adj_q, entry, w.metric)
    np.testing.assert_array_equal(parent, o_par)
    np.testing.assert_array_equal(depth, o_depth)
    pos = np.empty(w.nq, np.int64)
    pos[order] = np.arange(w.nq)
    has = parent >= 0
    assert np.all(pos[parent[has]] < pos[np.nonzero(has)[0]])


JOIN_MODES = [
    ("inlj", dict(work_sharing=vj.VJ_WS_NONE)),
    ("inlj_self", dict(work_sharing=vj.VJ_WS_SELF)),
    ("hws", dict(work_sharing=vj.VJ_WS_HARD)),
    ("sws", dict(work_sharing=vj.VJ_WS_SOFT)),
    ("sws_beam8_conv3", dict(work_sharing=vj.VJ_WS_SOFT, greedy_beam=8, conv_threshold=3)),
    ("inlj_conv0", dict(work_sharing=vj.VJ_WS_NONE, conv_threshold=0)),
    ("sws_force_hybrid_8", dict(work_sharing=vj.VJ_WS_SOFT, force_hybrid=1, hybrid_beam=8)),
    ("hws_force_hybrid_64", dict(work_sharing=vj.VJ_WS_HARD, force_hybrid=1, hybrid_beam=64)),
]
OWS = {vj.VJ_WS_NONE: 0, vj.VJ_WS_HARD: 1, vj.VJ_WS_SOFT: 2, vj.VJ_WS_SELF: 3}


@pytest.mark.parametrize("mode,kw", JOIN_MODES, ids=[m for m, _ in JOIN_MODES])
def test_separate_join_matches_oracle(built, oracle, mode, kw):
    name, w, ix = built
    eps = float(np.float32(_calib_eps(w, 10)))
    full = dict(greedy_beam=256, conv_threshold=10, hybrid_beam=256, adapt_hybrid=1, force_hybrid=0)
    full.update(kw)
    vj.vj_set_join_params(ix, **full)
    r = vj.vj_join(ix, eps)
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    o = oracle.join(w.X, w.Q, adj[:w.nx], entry, np.float32(eps), metric=w.metric,
                    work_sharing=OWS[full["work_sharing"]], force_hybrid=bool(full["force_hybrid"]),
                    adapt_hybrid=True, greedy_beam_size=full["greedy_beam"],
                    conv_threshold=full["conv_threshold"], hybrid_beam_size=full["hybrid_beam"],
                    order=order, parent=parent, separate=True)
    band = _band_pairs(w, float(np.float32(eps)))
    g, e = _pairs(r.offsets, r.ids), _pairs(o.offsets, o.ids)
    diff = (g ^ e) - band
    np.testing.assert_array_equal(r.hybrid, o.hybrid)
    # the hybrid search's FP32 pop order (see _assert_steps): with a queue of a
    # few entries one flipped pop can also change what the search reaches
    dq = sorted({q for q, _ in diff})
    slack = full["force_hybrid"] and len(dq) <= max(1, w.nq // 1000) and np.all(r.hybrid[dq] == 1)
    assert not diff or slack, f"{name}/{mode}: {len(diff)} pairs differ, e.g. {sorted(diff)[:5]}"
    if full["work_sharing"] == vj.VJ_WS_SOFT:
        # a soft cache is the closest visited node: FP64 among near-ties, so
        # it equals the oracle's wherever the visited set does
        bad = np.nonzero((r.cache != o.cache) & (r.steps == o.steps))[0]
        assert len(bad) == 0, f"{name}/{mode}: caches differ at {bad[:5]}"
    _assert_steps(name, r, o)
    assert r.stats["dist_computations"] == int(r.steps.sum())
    for q in range(0, w.nq, 11):
        a, b = r.row(q), o.row(q)
        _, ia, ib = np.intersect1d(a, b, return_indices=True)
        np.testing.assert_allclose(r.dists[r.offsets[q] + ia], o.dists[o.offsets[q] + ib], rtol=1e-5, atol=1e-6)


def test_hard_sharing_needs_separate_indexes():
    w = CASES["gauss_d32_simt"]()
    p = vj.default_params(degree=w.degree, knn_k=w.knn_k)
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=p)
    with pytest.raises(vj.VjError):
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_HARD)
    ix.free()
    with pytest.raises(vj.VjError):
        vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k),
                    separate=1, nnmap=1)


def test_separate_wait_timeout_is_reported():
    """A query that never publishes: its children's bounded waits run out and
    the join returns VJ_ERR_TIMEOUT; the index stays usable."""
    w = CASES["gauss_d32_simt"]()
    ix = _build(w)
    _, _, parent, order, _ = vj.vj_export_graph(ix)
    held = int(parent[parent >= 0][0])
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT)
    vj.vj_set_wait_test(ix, 2000, held)
    with pytest.raises(vj.VjError) as e:
        vj.vj_join(ix, 1.0)
    assert e.value.status == vj.VJ_ERR_TIMEOUT
    vj.vj_set_wait_test(ix, 0, -1)
    r = vj.vj_join(ix, 1.0)
    assert r.offsets[-1] == len(r.ids)
    ix.free()
