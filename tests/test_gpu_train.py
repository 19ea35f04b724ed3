"""The predictor's labels and training inside the library (vj_predictor_labels,
vj_train_predictor) against the oracle, and the bounded dependency wait of
soft work sharing (vj_set_wait_test)."""
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


def _eps(w, matches, metric=0):
    from scipy.spatial.distance import cdist
    D = cdist(w.Q[:200].astype(np.float64), w.X.astype(np.float64), "euclidean" if metric == 0 else "cosine")
    k = int(matches * 200)
    return float(np.float32(np.partition(D.ravel(), k)[k]))


@pytest.mark.parametrize("ws", [vj.VJ_WS_SELF, vj.VJ_WS_SOFT], ids=["self", "sws"])
def test_labels_equal_oracle_labels(oracle, ws):
    """Budget and route labels made on the GPU (exact rows from the scan,
    planned joins per ladder budget) equal those the oracle's nested-loop join
    and planned joins give by the same rules, on the same graph and with the
    same scan-row cost."""
    from oracle import labels as olab
    w = inputs.gauss_small(seed=41, nx=3000, nq=400, d=16, k=8, ood_frac=0.1, shift=8.0)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=16, knn_k=32))
    eps = _eps(w, 10)
    vj.vj_set_join_params(ix, work_sharing=ws, adapt_hybrid=1)
    rows = np.arange(0, w.nq, 2, dtype=np.int32)
    kw = dict(ladder=[-1, 0, 8], query_recall=0.95, pooled_recall=0.97, scan_row_cost=120.0)
    b, r, rep = vj.vj_predictor_labels(ix, eps, rows, **kw)
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    ob, orr = olab.predictor_labels(oracle, w.X, w.Q, adj, entry, np.float32(eps), rows, kw["ladder"],
                                    kw["query_recall"], kw["pooled_recall"], kw["scan_row_cost"],
                                    work_sharing={vj.VJ_WS_SELF: oracle.WS_SELF, vj.VJ_WS_SOFT: oracle.WS_SOFT}[ws],
                                    order=order, parent=parent)
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(r, orr)
    assert rep["n"] == len(rows) and rep["ladder_run"] == 3 and rep["routed"] == int(r.sum())
    assert sum(rep["per_budget"][:3]) == len(rows)
    assert len(set(b.tolist())) >= 2 and 0 < r.sum() < len(rows)  # the labels are not all alike
    # the join parameters and the (empty) plan are restored
    a = vj.vj_join(ix, eps)
    vj.vj_set_join_params(ix, work_sharing=ws, adapt_hybrid=1)
    c = vj.vj_join(ix, eps)
    assert np.array_equal(a.ids, c.ids) and np.array_equal(a.steps, c.steps)
    ix.free()


def test_train_predictor_end_to_end():
    """vj_train_predictor: labels, features of the training rows, Adam; the
    returned predictor attaches and plans a join (routed queries get exact
    rows)."""
    w = inputs.gauss_small(seed=42, nx=3000, nq=500, d=16, k=8, ood_frac=0.1, shift=8.0)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=16, knn_k=32))
    eps = _eps(w, 10)
    rows = np.arange(0, w.nq, 2, dtype=np.int32)
    m, rep = vj.vj_train_predictor(ix, eps, rows, ladder=[-1, 0, 8], h1=64, h2=64, epochs=20, batch=64)
    assert m.din == vj.NFEAT + w.d
    assert rep["final_loss"] > 0 and rep["ms_train"] > 0 and rep["scan_row_cost"] > 0
    vj.vj_attach_predictor(ix, m, 0.5, 64)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, learned=1)
    r = vj.vj_join(ix, eps)
    ex = vj.vj_join_exact(ix, eps)
    for q in np.nonzero(r.hybrid == 2)[0]:
        assert np.array_equal(r.row(q), ex.row(q))
    vj.vj_set_join_params(ix, learned=0)
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    m.free()
    ix.free()


def test_dependency_wait_times_out_and_index_stays_usable():
    """A query that never publishes its cache (a test knob) makes its MST
    children's bounded waits run out: the join returns VJ_ERR_TIMEOUT, and
    with the knob cleared the next join equals a join that never timed out."""
    w = inputs.gauss_small(seed=43, nx=2000, nq=300, d=16, k=8)
    ix = vj.vj_build(w.X, w.Q, params=vj.default_params(degree=16, knn_k=32))
    eps = _eps(w, 10)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1)
    ref = vj.vj_join(ix, eps)
    _, _, parent, _, _ = vj.vj_export_graph(ix)
    kids = np.bincount(parent[parent >= 0], minlength=w.nq)
    held = int(np.argmax(kids))
    assert kids[held] > 0
    vj.vj_set_wait_test(ix, max_polls=2000, hold_q=held)
    with pytest.raises(vj.VjError) as e:
        vj.vj_join(ix, eps)
    assert e.value.status == vj.VJ_ERR_TIMEOUT
    vj.vj_set_wait_test(ix, 0, -1)
    r = vj.vj_join(ix, eps)
    assert np.array_equal(r.offsets, ref.offsets) and np.array_equal(r.ids, ref.ids)
    assert np.array_equal(r.steps, ref.steps) and np.array_equal(r.cache, ref.cache)
    with pytest.raises(vj.VjError):
        vj.vj_set_wait_test(ix, 0, w.nq)  # out of range
    ix.free()


def _recall_rows(r, ex, lo, hi):
    hit = tot = 0
    for q in range(lo, hi):
        a = set(r.row(q).tolist())
        b = set(ex.row(q).tolist())
        hit += len(a & b)
        tot += len(b)
    return hit / max(tot, 1)


def test_learned_route_gains_over_the_rule():
    """What the trained network gains over the method without it.  On the
    learned-predictor recipe (vMF embeddings, BF16, cosine), a predictor trained
    on held-out queries of the index (vj_train_predictor) plans the evaluated
    queries.  It must reach recall 0.95 against the exact join, and cost at most
    half as much as the paper's d1/d2 rule (Sec. 4.4), alone or with its OOD
    queries sent to the brute-force scan.  Cost: distance evaluations plus
    routed queries times the cost of a scan row in distance evaluations."""
    w = inputs.vmf_like(seed=44, scale=0.01)  # 100K x 768 data, 10K evaluated + 1K held-out queries
    ne = w.nq - w.nh
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=32, knn_k=64))
    from scipy.spatial.distance import cdist
    D = cdist(w.Q[:200].astype(np.float64), w.X.astype(np.float64), "cosine")
    eps = float(np.float32(np.partition(D.ravel(), 2000)[2000]))
    ex = vj.vj_join_exact(ix, eps)
    rows = np.arange(ne, w.nq, dtype=np.int32)
    m, rep = vj.vj_train_predictor(ix, eps, rows, ladder=[-1, 0], h1=64, h2=64, epochs=20, batch=64)
    c_scan = rep["scan_row_cost"]

    def cost(r):
        s = r.steps[:ne].astype(np.float64)
        return float(s.sum() + (r.hybrid[:ne] == 2).sum() * c_scan)

    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1, learned=0)
    rule = vj.vj_join(ix, eps)
    route = (rule.hybrid == 1).astype(np.uint8)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, learned=0)
    vj.vj_set_plan(ix, route, np.zeros(w.nq, np.int32))
    rule_routed = vj.vj_join(ix, eps)
    vj.vj_set_plan(ix, None, None)
    vj.vj_attach_predictor(ix, m, 0.5, 0)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, learned=1, gather=vj.VJ_PREC_BF16)
    lr = vj.vj_join(ix, eps)
    rec = {k: _recall_rows(r, ex, 0, ne) for k, r in (("rule", rule), ("rule_routed", rule_routed), ("learned", lr))}
    c = {k: cost(r) for k, r in (("rule", rule), ("rule_routed", rule_routed), ("learned", lr))}
    assert rec["learned"] >= 0.95, (rec, c)
    assert c["learned"] <= 0.5 * min(c["rule"], c["rule_routed"]), (rec, c)
    vj.vj_set_join_params(ix, learned=0, gather=vj.VJ_PREC_FP32)
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    m.free()
    ix.free()
