"""Joins of a collection of instances (vj_join_batch) against single joins and the oracle.

The traversal passes of every instance in a batch run fused (one launch per
pass over all instances of a kernel class).  Each instance's result must equal
what vj_join gives for that instance alone (pairs, distances, visited counts,
soft caches, hybrid flags), and one instance is also checked against the CPU
oracle's MI+SWS join on the same graph.
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu

SMALL = dict(nx_range=(1500, 12000), nq_range=(150, 2000))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()


def _eps(w, sample=200):
    """eps with about target_matches exact pairs per query on a query sample (FP64, cdist)."""
    from scipy.spatial.distance import cdist
    Qs = w.Q[:sample].astype(np.float64)
    D = cdist(Qs, w.X.astype(np.float64), "euclidean" if w.metric == 0 else "cosine")
    k = int(w.target_matches * len(Qs))
    return float(np.float32(np.partition(D.ravel(), k)[k]))


def _build(w):
    return vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))


def _same(a, b, tag):
    np.testing.assert_array_equal(a.offsets, b.offsets, err_msg=tag)
    np.testing.assert_array_equal(a.ids, b.ids, err_msg=tag)
    np.testing.assert_array_equal(a.dists, b.dists, err_msg=tag)
    np.testing.assert_array_equal(a.steps, b.steps, err_msg=tag)
    np.testing.assert_array_equal(a.cache, b.cache, err_msg=tag)
    np.testing.assert_array_equal(a.hybrid, b.hybrid, err_msg=tag)


@pytest.fixture(scope="module")
def collection():
    ws = list(inputs.angular_collection(seed=501, n=6, **SMALL))
    # a second kernel class (d = 32, L2) in the same batch
    ws.append(inputs.gauss_small(seed=502, nx=4000, nq=500, d=32))
    ixs = [_build(w) for w in ws]
    eps = [_eps(w) for w in ws]
    # per-instance join modes: soft sharing (default), self-only, forced hybrid,
    # and a plan that routes every 7th query to the brute-force scan
    vj.vj_set_join_params(ixs[1], work_sharing=vj.VJ_WS_SELF, adapt_hybrid=1)
    vj.vj_set_join_params(ixs[2], work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=1, hybrid_beam=16)
    route = np.zeros(ws[3].nq, np.uint8)
    route[::7] = 1
    vj.vj_set_plan(ixs[3], route=route)
    yield ws, ixs, eps
    for ix in ixs:
        ix.free()


def test_batch_equals_single_joins(collection):
    ws, ixs, eps = collection
    single = [vj.vj_join(ix, e) for ix, e in zip(ixs, eps)]
    batch = vj.vj_join_batch(ixs, eps)
    assert len(batch) == len(ixs)
    for i, (a, b) in enumerate(zip(batch, single)):
        _same(a, b, f"instance {i}")
        assert a.nnz == len(a.ids) == a.offsets[-1]
        assert a.stats["dist_computations"] == b.stats["dist_computations"]
    # the collection really is uneven (targets of 8 to 49 matches per query)
    counts = [b.nnz / w.nq for b, w in zip(batch, ws)]
    assert max(counts) > 2 * min(counts)


def test_batch_repeated_and_reordered(collection):
    """A second batch (longest-first dispatch from the first) and a reversed
    batch give the same results."""
    ws, ixs, eps = collection
    first = vj.vj_join_batch(ixs, eps)
    again = vj.vj_join_batch(ixs, eps)
    rev = vj.vj_join_batch(ixs[::-1], eps[::-1])[::-1]
    for i in range(len(ixs)):
        _same(first[i], again[i], f"repeat {i}")
        _same(first[i], rev[i], f"reversed {i}")


def test_batch_instance_matches_oracle(collection, oracle):
    ws, ixs, eps = collection
    i = int(np.argmin([w.nx for w in ws[:6]]))
    w, ix = ws[i], ixs[i]
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1)
    r = vj.vj_join_batch([ix], [eps[i]])[0]
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    o = oracle.join(w.X, w.Q, adj, entry, np.float32(eps[i]), metric=w.metric, work_sharing=oracle.WS_SOFT,
                    adapt_hybrid=True, order=order, parent=parent)
    from scipy.spatial.distance import cdist
    D = cdist(w.Q.astype(np.float64), w.X.astype(np.float64), "cosine")
    qs, xs = np.nonzero(np.abs(D - eps[i]) <= 1e-4 * eps[i])
    band = set(zip(qs.tolist(), xs.tolist()))

    def pairs(off, ids):
        return {(q, int(x)) for q in range(len(off) - 1) for x in ids[off[q]:off[q + 1]]}

    diff = (pairs(r.offsets, r.ids) ^ pairs(o.offsets, o.ids)) - band
    assert not diff, f"{len(diff)} pairs differ"
    np.testing.assert_array_equal(r.steps, o.steps)
    np.testing.assert_array_equal(r.cache, o.cache)
    np.testing.assert_array_equal(r.hybrid, o.hybrid)


def test_batch_shared_predictor_and_errors(collection):
    ws, ixs, eps = collection
    # one predictor attached to two indexes of the same dimension
    m = vj.MLP(ws[0].d + vj.NFEAT, 64, 32, seed=3)
    vj.vj_attach_predictor(ixs[4], m, route_threshold=0.9, beam_cap=64)
    vj.vj_attach_predictor(ixs[5], m, route_threshold=0.9, beam_cap=64)
    for ix in (ixs[4], ixs[5]):
        vj.vj_set_join_params(ix, learned=1)
    single = [vj.vj_join(ixs[k], eps[k]) for k in (4, 5)]
    batch = vj.vj_join_batch([ixs[4], ixs[5]], [eps[4], eps[5]])
    for a, b, k in zip(batch, single, (4, 5)):
        _same(a, b, f"learned instance {k}")
    for ix in (ixs[4], ixs[5]):
        vj.vj_set_join_params(ix, learned=0)
        vj.vj_attach_predictor(ix, None, route_threshold=0.5)
    # all or nothing
    with pytest.raises(vj.VjError) as e:
        vj.vj_join_batch([ixs[0], ixs[0]], [eps[0], eps[0]])
    assert e.value.status == vj.VJ_ERR_ARG
    with pytest.raises(vj.VjError) as e:
        vj.vj_join_batch([ixs[0], ixs[1]], [eps[0], -1.0])
    assert e.value.status == vj.VJ_ERR_ARG
    assert vj.vj_join_batch([], []) == []


def test_batch_beyond_one_launch():
    """More instances than one fused launch takes (64): the batch is split
    into several launches per pass and still equals the single joins."""
    rng = np.random.default_rng(77)
    ixs, eps, single = [], [], []
    for k in range(70):
        nx, nq = int(rng.integers(300, 900)), int(rng.integers(20, 120))
        X = rng.standard_normal((nx, 16)).astype(np.float32)
        Q = (X[rng.integers(0, nx, nq)] + 0.3 * rng.standard_normal((nq, 16))).astype(np.float32)
        ix = vj.vj_build(X, Q, params=vj.default_params(degree=8, knn_k=16))
        ixs.append(ix)
        eps.append(2.0 + 0.01 * k)
    single = [vj.vj_join(ix, e) for ix, e in zip(ixs, eps)]
    batch = vj.vj_join_batch(ixs, eps)
    for i, (a, b) in enumerate(zip(batch, single)):
        _same(a, b, f"instance {i}")
    assert sum(r.nnz for r in batch) > 0
    for ix in ixs:
        ix.free()


def test_concurrent_joins_on_host_threads():
    """Joins of different indexes from concurrent host threads each borrow
    their own traversal workspace and give the single-thread results."""
    import threading
    ws = [inputs.angular_instance(601, k, nx_range=(3000, 6000), nq_range=(300, 600)) for k in range(4)]
    ixs = [_build(w) for w in ws]
    eps = [_eps(w) for w in ws]
    ref = [vj.vj_join(ix, e) for ix, e in zip(ixs, eps)]
    out = [None] * len(ixs)
    errs = []

    def run(k):
        try:
            for _ in range(3):
                out[k] = vj.vj_join(ixs[k], eps[k])
        except Exception as e:  # reported below
            errs.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in range(len(ixs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for k in range(len(ixs)):
        _same(out[k], ref[k], f"thread {k}")
    for ix in ixs:
        ix.free()
    # a rebuilt index borrows a cached workspace and joins the same
    w = ws[0]
    ix = _build(w)
    r = vj.vj_join(ix, eps[0])
    _same(r, ref[0], "after the cache was emptied")
    ix.free()
