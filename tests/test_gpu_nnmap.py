"""NN-Map index (the paper's closing design, "NN-Map") on the GPU, through the
C ABI, against the oracle on the same seeded inputs.

Bars, stage by stage (each stage fed the GPU's output of the stage before,
so a difference is pinned to one stage):
  * kNN lists of an NN-Map index rank data vectors only: ids bit-exact
    against the oracle's exact lists over the data set (ties by id), keys
    within 1e-5 relative;
  * the graph is G_X: data rows bit-exact against the oracle's graph build on
    the data set alone (same kNN lists), entry equal, query rows empty;
  * witness ids and OOD bits bit-exact, witness distances within 1e-12
    relative of the oracle's FP64 values (``oracle.nnmap_build_c`` on G_X);
  * joins (BFS, adaptive and forced hybrid expansion): result rows equal
    outside the |dist - eps| <= 1e-4 eps band, distance evaluations and hybrid
    flags equal to ``oracle.nnmap_join_c``'s.
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
    # fewer than 4096 data vectors: the FP32 SIMT kNN sweep
    "gauss_d32_simt": lambda: inputs.gauss_small(seed=201, nx=3000, nq=400, d=32),
    # BF16 tensor-core kNN, resident tiles (queries and data in one sweep)
    "sift_like_tc": lambda: inputs.sift_like(seed=202, scale=0.005),  # 5000 x 128 integers, 500 queries
    "cosine_d20_tc": lambda: inputs.uniform_small(203, 5000, 300, 20, metric=1, degree=16, knn_k=32),
    # streamed tiles: the symmetric data sweep plus the query rows' own launch
    "wide_l2_d300": lambda: inputs.uniform_small(204, 4500, 300, 300, degree=12, knn_k=24),
    "vmf_cos_d768": lambda: inputs.vmf_like(seed=205, scale=0.00045),  # 4500 x 768 cosine, 495 queries
}


def _build(w):
    p = vj.default_params(degree=w.degree, knn_k=w.knn_k)
    return vj.vj_build(w.X, w.Q, metric=w.metric, params=p, nnmap=1)


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
    """Distance evaluations equal the oracle's.  The one known exception is
    the hybrid expansion's pop order: the GPU orders its out-range queue by
    FP32 keys, the oracle by FP64 distances, and where the distances crowd
    within a few percent of each other (the d = 768 cosine case) an FP32
    near-tie can flip one pop.  There a hybrid query may differ in its count,
    at most 0.5 % of the queries, while its result row still equals the
    oracle's (checked by the caller)."""
    bad = np.nonzero(r.steps != o.steps)[0]
    if name == "vmf_cos_d768" and len(bad) <= max(1, len(r.steps) // 200):
        assert np.all(r.hybrid[bad] == 1), bad
        return
    np.testing.assert_array_equal(r.steps, o.steps)


def _pairs(off, ids):
    return {(q, int(i)) for q in range(len(off) - 1) for i in ids[off[q]:off[q + 1]]}


def test_knn_lists_rank_data_only(built, oracle):
    name, w, ix = built
    ids, keys = vj.vj_export_knn(ix)
    K = ids.shape[1]
    assert np.all((ids >= 0) & (ids < w.nx)), name
    empty = w.Q[:0]
    drows = np.arange(0, w.nx, 7)
    o_ids, o_d = oracle.knn_rows(w.X, empty, K, drows, w.metric)
    mism = np.nonzero((ids[drows] != o_ids).any(axis=1))[0]
    assert len(mism) == 0, f"{name}: {len(mism)} data rows differ, first {drows[mism[:5]]}"
    ref = o_d ** 2 if w.metric == 0 else o_d
    np.testing.assert_allclose(keys[drows], ref, rtol=1e-5, atol=1e-6)
    # a query's list: its K nearest data vectors (the merged set X + {q})
    for qi in range(0, w.nq, 5):
        q_ids, q_d = oracle.knn_rows(w.X, w.Q[qi:qi + 1], K, [w.nx], w.metric)
        np.testing.assert_array_equal(ids[w.nx + qi], q_ids[0], err_msg=f"{name}: query {qi}")
        r = q_d[0] ** 2 if w.metric == 0 else q_d[0]
        np.testing.assert_allclose(keys[w.nx + qi], r, rtol=1e-5, atol=1e-6)


def test_graph_is_the_data_graph(built, oracle):
    name, w, ix = built
    kn, _ = vj.vj_export_knn(ix)
    adj, entry, parent, order, depth = vj.vj_export_graph(ix)
    R, K = adj.shape[1], kn.shape[1]
    assert np.all(adj[w.nx:] == -1), name
    o_adj, o_entry, _ = oracle.build_graph(w.X, w.Q[:0], R, K, w.metric, knn_ids=kn[:w.nx])
    assert entry == o_entry, name
    mism = np.nonzero((adj[:w.nx] != o_adj).any(axis=1))[0]
    assert len(mism) == 0, f"{name}: {len(mism)} G_X rows differ, first {mism[:5]}"
    np.testing.assert_array_equal(order, np.arange(w.nq))
    assert np.all(parent == -1)


def test_witness_and_ood_match_oracle(built, oracle):
    name, w, ix = built
    adj = vj.vj_export_graph(ix)[0][:w.nx]
    wg, wdg, oodg = vj.vj_export_nnmap(ix)
    o = oracle.nnmap_build_c(w.X, w.Q, adj, w.metric)
    np.testing.assert_array_equal(wg, o.witness, err_msg=name)
    np.testing.assert_allclose(wdg, o.wdist, rtol=1e-12, atol=1e-15, err_msg=name)
    np.testing.assert_array_equal(oodg, o.ood, err_msg=name)


def test_ood_bit_follows_far_queries(oracle):
    """The generator marks a fifth of the queries as drawn away from the data's
    clusters; the d1/d2 rule flags those more often than the others."""
    w = CASES["gauss_d32_simt"]()
    ix = _build(w)
    _, _, ood = vj.vj_export_nnmap(ix)
    ix.free()
    far = np.asarray(w.ood, bool)
    assert far.any() and (~far).any()
    assert ood[far].mean() > ood[~far].mean() + 0.2, (ood[far].mean(), ood[~far].mean())


JOIN_MODES = [
    ("bfs", "off", dict(adapt_hybrid=0, force_hybrid=0)),
    ("adapt", "adapt", dict(adapt_hybrid=1, force_hybrid=0, hybrid_beam=64)),
    ("force_64", "force", dict(adapt_hybrid=0, force_hybrid=1, hybrid_beam=64)),
    ("force_8", "force", dict(adapt_hybrid=0, force_hybrid=1, hybrid_beam=8)),
]


@pytest.mark.parametrize("matches", [0.3, 10])
@pytest.mark.parametrize("mode,omode,kw", JOIN_MODES, ids=[m for m, _, _ in JOIN_MODES])
def test_nnmap_join_matches_oracle(built, oracle, mode, omode, kw, matches):
    name, w, ix = built
    eps = float(np.float32(_calib_eps(w, matches)))
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_NONE, **kw)
    r = vj.vj_join(ix, eps)
    adj = vj.vj_export_graph(ix)[0][:w.nx]
    nm = oracle.nnmap_build_c(w.X, w.Q, adj, w.metric)
    o = oracle.nnmap_join_c(w.X, w.Q, adj, nm, eps, metric=w.metric, hybrid=omode,
                            hybrid_beam_size=kw.get("hybrid_beam", 256))
    band = _band_pairs(w, eps)
    g, e = _pairs(r.offsets, r.ids), _pairs(o.offsets, o.ids)
    diff = (g ^ e) - band
    assert not diff, f"{name}/{mode}: {len(diff)} pairs differ, e.g. {sorted(diff)[:5]}"
    np.testing.assert_array_equal(r.hybrid, o.hybrid)
    _assert_steps(name, r, o)
    # certified-empty rows computed nothing
    empty = nm.wdist >= eps
    assert np.all(r.steps[empty] == 0) and np.all(np.diff(r.offsets)[empty] == 0)
    assert r.stats["dist_computations"] == int(r.steps.sum())
    for q in range(0, w.nq, 7):
        a, b = r.row(q), o.row(q)
        common, ia, ib = np.intersect1d(a, b, return_indices=True)
        np.testing.assert_allclose(r.dists[r.offsets[q] + ia], o.dists[o.offsets[q] + ib], rtol=1e-5, atol=1e-6)


def test_nnmap_refuses_plans_and_features():
    w = CASES["gauss_d32_simt"]()
    ix = _build(w)
    with pytest.raises(vj.VjError):
        vj.vj_set_plan(ix, beam=np.zeros(w.nq, np.int32))
    with pytest.raises(vj.VjError):
        vj.vj_features(ix, 1.0)
    vj.vj_set_plan(ix)  # clearing a plan is allowed
    ix.free()
    # an index built without nnmap has no NN-Map outputs
    p = vj.default_params(degree=w.degree, knn_k=w.knn_k)
    ix2 = vj.vj_build(w.X, w.Q, metric=w.metric, params=p)
    with pytest.raises(vj.VjError):
        vj.vj_export_nnmap(ix2)
    ix2.free()
    with pytest.raises(vj.VjError):
        vj.vj_build(w.X[:1], w.Q, metric=w.metric, params=vj.default_params(degree=1, knn_k=1), nnmap=1)
