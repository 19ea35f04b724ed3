"""Labels of the learned route / budget predictor, restated plainly on top of
the oracle's joins (test infrastructure only; nothing in the library imports
this module).

The paper has no predictor: its route is the d1/d2 > 1.5 rule of Sec. 4.4.
The labels are the library's own rules, written here from their definition:

  exact row       the nested-loop join (Sec. 3.2) of each training query;
  ladder          one oracle join (Alg. 1 on the merged index) per budget, every
                  query planned with that budget (-1: no expansion phase, 0: the
                  BFS expansion, > 0: hybrid queue size); a query's recall is
                  |row n exact| / |exact| (1 for an empty exact row) and its
                  cost the distance evaluations it made;
  budget label    the first budget whose recall reaches query_recall, else the
                  last budget;
  route label     1 when the query's cost at its budget is at least
                  scan_row_cost; then, while the training queries' pooled
                  recall is below pooled_recall, the query with the largest
                  missed / (scan_row_cost - cost), ties by smaller query index.

Recall comparisons are taken in float32 and the route arithmetic in float64,
the precisions the library decides in.
"""
from __future__ import annotations

import numpy as np


def predictor_labels(oracle, X, Q, adj, entry, eps, rows, ladder, query_recall, pooled_recall, scan_row_cost, *,
                     metric=0, work_sharing=None, order=None, parent=None):
    """(budget [n], route [n]) of the training queries `rows` (query indices)."""
    rows = np.asarray(rows, np.int64)
    nq = len(Q)
    off, ids, _ = oracle.nlj(X, Q, eps, metric)
    exact = [set(ids[off[q]:off[q + 1]].tolist()) for q in rows]
    ws = oracle.WS_SOFT if work_sharing is None else work_sharing
    rec, miss, cost = [], [], []
    for b in ladder:
        r = oracle.join(X, Q, adj, entry, eps, metric=metric, work_sharing=ws, order=order, parent=parent,
                        beam=np.full(nq, b, np.int32))
        rk, mk, ck = [], [], []
        for i, q in enumerate(rows):
            got = set(r.row(int(q)).tolist())
            tot = len(exact[i])
            hit = len(got & exact[i])
            rk.append(np.float32(hit / tot) if tot > 0 else np.float32(1.0))
            mk.append(float(tot - hit))
            ck.append(int(r.steps[q]))
        rec.append(rk)
        miss.append(mk)
        cost.append(ck)
    n = len(rows)
    qr = np.float32(query_recall)
    pick = [len(ladder) - 1] * n
    for i in range(n):
        for k in range(len(ladder)):
            if rec[k][i] >= qr:
                pick[i] = k
                break
    budget = np.array([ladder[pick[i]] for i in range(n)], np.int32)
    c_scan = float(np.float32(scan_row_cost))
    route = np.zeros(n, np.uint8)
    tot_all = float(sum(len(e) for e in exact))
    missed = 0.0
    gain = [0.0] * n
    for i in range(n):
        c, m = float(cost[pick[i]][i]), miss[pick[i]][i]
        if c >= c_scan:
            route[i] = 1
        else:
            missed += m
            gain[i] = m / max(c_scan - c, 1e-9)
    allowed = (1.0 - float(np.float32(pooled_recall))) * tot_all
    if missed > allowed:
        cand = [i for i in range(n) if not route[i] and miss[pick[i]][i] > 0]
        cand.sort(key=lambda i: (-gain[i], int(rows[i])))
        for i in cand:
            if missed <= allowed:
                break
            route[i] = 1
            missed -= miss[pick[i]][i]
    return budget, route
