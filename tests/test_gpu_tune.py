"""Traversal tuning: every setting the tuner may choose computes the same join.

A setting is the gather layout of the traversal (lanes per row, 16-byte
slots per lane, rows in flight), the persistent grid, the probe ring and the
probe's copy (16-byte copies per lane, or one bulk copy per row).
In-range decisions near eps are re-decided in FP64 and cache ties too, so
the pairs, visited counts and soft caches equal the default setting's and
the oracle's; a pair's FP32 distance may differ in its last bits (the
summation order of a key follows the layout).
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()


def _eps(w, matches):
    from scipy.spatial.distance import cdist
    D = cdist(w.Q[:100].astype(np.float64), w.X.astype(np.float64), "euclidean" if w.metric == 0 else "cosine")
    return float(np.float32(np.partition(D.ravel(), matches * 100)[matches * 100]))


def _same_join(a, b):
    np.testing.assert_array_equal(a.offsets, b.offsets)
    np.testing.assert_array_equal(a.ids, b.ids)
    np.testing.assert_allclose(a.dists, b.dists, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(a.steps, b.steps)
    np.testing.assert_array_equal(a.cache, b.cache)
    np.testing.assert_array_equal(a.hybrid, b.hybrid)


CASES = {
    "gauss_d32": lambda: inputs.gauss_small(seed=301, nx=4000, nq=400, d=32),
    "angular_d100": lambda: inputs.uniform_small(302, 4000, 400, 100, metric=1, degree=16, knn_k=32),
    "vmf_d768": lambda: inputs.vmf_like(seed=303, scale=0.0003),
}


@pytest.mark.parametrize("case", list(CASES))
def test_autotune_keeps_the_join(case, oracle):
    w = CASES[case]()
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    try:
        eps = _eps(w, 10)
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1)
        base = vj.vj_join(ix, eps)
        rep = vj.vj_autotune(ix, eps, reps=1)
        rows = rep["settings"]
        assert len(rows) >= 3
        assert all(r["valid"] for r in rows), rows
        assert all(r["ms"] > 0 for r in rows)
        ch = rows[rep["chosen"]]
        assert ch["lanes"] * ch["slots"] * 4 >= w.d
        tuned = vj.vj_join(ix, eps)
        _same_join(base, tuned)
        # every class the tuner tried, set explicitly, gives the same join
        for r in rows:
            vj.vj_set_tuning(ix, r["lanes"], r["slots"], r["inflight"], r["blocks"], r["probe_ring"],
                             r["probe_bulk"])
            _same_join(base, vj.vj_join(ix, eps))
        # and the join equals the oracle's on the same graph
        adj, entry, parent, order, _ = vj.vj_export_graph(ix)
        o = oracle.join(w.X, w.Q, adj, entry, np.float32(eps), metric=w.metric, work_sharing=oracle.WS_SOFT,
                        adapt_hybrid=True, order=order, parent=parent)
        assert {(q, int(i)) for q in range(w.nq) for i in base.row(q)} == \
               {(q, int(i)) for q in range(w.nq) for i in o.row(q)}
    finally:
        ix.free()


def test_tuning_applies_to_batched_joins():
    """A setting set on every index of a batch: vj_join_batch equals one join per index."""
    ws = [inputs.uniform_small(310 + i, 2500 + 500 * i, 250, 100, metric=1, degree=16, knn_k=32) for i in range(3)]
    ixs = [vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
           for w in ws]
    try:
        eps = [_eps(w, 8) for w in ws]
        for ix in ixs:
            vj.vj_set_tuning(ix, 16, 4, 2, 0, 4, 1)  # a larger class than the default for d = 100, bulk probe
        batch = vj.vj_join_batch(ixs, eps)
        for ix, e, b in zip(ixs, eps, batch):
            _same_join(vj.vj_join(ix, e), b)
    finally:
        for ix in ixs:
            ix.free()


def test_tuning_arguments_are_checked():
    w = inputs.uniform_small(320, 1500, 100, 300, degree=12, knn_k=24)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    try:
        for bad in [(8, 4, 2, 0, 0),    # 128 floats per row: too small for d = 300
                    (8, 3, 2, 0, 0),    # no such class
                    (0, 0, 0, -1, 0),   # negative grid
                    (0, 0, 0, 0, 1),    # probe ring below 2
                    (0, 0, 0, 0, 0, 2)]:  # probe_bulk not 0/1
            with pytest.raises(vj.VjError) as e:
                vj.vj_set_tuning(ix, *bad)
            assert e.value.status == vj.VJ_ERR_ARG
        with pytest.raises(vj.VjError) as e:
            vj.vj_autotune(ix, 1.0, reps=0)
        assert e.value.status == vj.VJ_ERR_ARG
        vj.vj_set_tuning(ix)  # defaults
        assert vj.vj_join(ix, 1.0).offsets.shape == (w.nq + 1,)
    finally:
        ix.free()
