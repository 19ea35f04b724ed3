"""Pins of oracle/labels.py, the plain restatement of the predictor's label
rules, on a hand-worked case: a stub stands in for the nested-loop join and
the planned joins, so every recall, cost and route decision below is known by
hand."""
import numpy as np

from oracle import labels


class _Row:
    def __init__(self, rows, steps):
        self.rows, self.steps = rows, np.array(steps)

    def row(self, q):
        return np.array(self.rows[q], np.int32)


class _Stub:
    WS_SOFT = 2

    # exact rows of queries 0..3: sizes 4, 2, 0, 10
    EXACT = [[1, 2, 3, 4], [5, 6], [], list(range(10))]
    # per budget (-1, 0): rows found and distance evaluations
    ROWS = {-1: ([[1, 2, 3], [5, 6], [], [0, 1, 2, 3]], [30, 40, 20, 50]),
            0: ([[1, 2, 3, 4], [5, 6], [], [0, 1, 2, 3, 4, 5]], [90, 60, 25, 500])}

    def nlj(self, X, Q, eps, metric):
        off = np.cumsum([0] + [len(r) for r in self.EXACT])
        ids = np.array(sum(self.EXACT, []), np.int32)
        return off, ids, None

    def join(self, X, Q, adj, entry, eps, *, beam, **kw):
        b = int(beam[0])
        rows, steps = self.ROWS[b]
        return _Row(rows, steps)


def test_budget_and_route_labels_by_hand():
    """query_recall 0.95: q0 (3/4 at -1, 4/4 at 0) -> 0; q1 (2/2 at -1) -> -1;
    q2 (empty exact row: recall 1) -> -1; q3 (4/10, 6/10) -> the last budget, 0.
    scan_row_cost 400: q3's cost at budget 0 is 500 >= 400 -> routed.  The
    rest miss nothing, so pooled recall is already 1 -> no other route."""
    Q = np.zeros((4, 2), np.float32)
    b, r = labels.predictor_labels(_Stub(), None, Q, None, 0, 1.0, [0, 1, 2, 3], [-1, 0], 0.95, 0.955, 400.0)
    assert b.tolist() == [0, -1, -1, 0]
    assert r.tolist() == [0, 0, 0, 1]


def test_knapsack_routes_by_missed_pairs_per_extra_cost():
    """scan_row_cost 1000: nobody is dearer than a scan.  Budgets as above;
    missed at the chosen budget: q0 0, q1 0, q2 0, q3 4 (cost 500).  Pooled:
    exact pairs 16, found 12 -> recall 0.75 < 0.955, allowed misses 0.72:
    q3 (the only one missing pairs) is routed; pooled misses drop to 0."""
    Q = np.zeros((4, 2), np.float32)
    b, r = labels.predictor_labels(_Stub(), None, Q, None, 0, 1.0, [0, 1, 2, 3], [-1, 0], 0.95, 0.955, 1000.0)
    assert b.tolist() == [0, -1, -1, 0]
    assert r.tolist() == [0, 0, 0, 1]


def test_knapsack_order_and_stop():
    """Query recall target 0.7 keeps q0 at -1 (3/4 = 0.75 missing 1 pair at
    cost 30) and labels q3 with the last budget 0 (6/10, missing 4 at cost
    500).  scan_row_cost 1000: gains q0 1/970 = 0.00103, q3 4/500 = 0.008.
    Pooled: 16 exact, 5 missed; pooled_recall 0.75 allows 4 misses: q3 alone
    (the larger gain) brings the misses to 1 <= 4, so q0 stays."""
    Q = np.zeros((4, 2), np.float32)
    b, r = labels.predictor_labels(_Stub(), None, Q, None, 0, 1.0, [0, 1, 2, 3], [-1, 0], 0.7, 0.75, 1000.0)
    assert b.tolist() == [-1, -1, -1, 0]
    assert r.tolist() == [0, 0, 0, 1]
    # a stricter pooled target (misses must fall to 0) routes q0 too, after q3
    b, r = labels.predictor_labels(_Stub(), None, Q, None, 0, 1.0, [0, 1, 2, 3], [-1, 0], 0.7, 1.0, 1000.0)
    assert r.tolist() == [1, 0, 0, 1]
