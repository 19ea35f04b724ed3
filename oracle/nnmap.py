"""NN-Map join (Sec. NN-Map), plain Python in FP64: test infrastructure only.

The paper closes with a design in which the merged index is replaced by a
materialised top-1 join index.  Each query keeps the id of its nearest data
vector (the witness), that distance, and an OOD bit, and the data set keeps
its own graph G_X.  A join at threshold eps then needs no greedy phase:
  * dist[q] >= eps: the row is certainly empty, and no distance is computed;
  * otherwise the expansion phase of Alg. 7 starts from the in-range seed w[q]
    on G_X, as the BFS closure, or as the hybrid search when the OOD bit is
    set (or forced).

This module is the oracle of that design.  It is written for the small inputs
of the tests (Python loops over nodes, numpy only for the distance rows), and
it shares no code with the CUDA library.  Like the rest of ``oracle``, only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.

Readings (the design is sketched, not fully specified):
  * witness: the nearest data vector by FP64 distance, ties by smaller id;
  * OOD bit: the d1/d2 rule of Alg. 6 with N1 = the query's R nearest data
    vectors (the neighbourhood a merged-index insertion would start from),
    d2 = mean length of the G_X edges from N1 to data nodes outside N1;
    OOD iff d1/d2 > 1.5, and no such edge means not OOD (parity unpinned
    against the paper beyond the far-query trend);
  * distance computations ("steps"): the witness distance is stored, so the
    seed costs none; every other node the expansion evaluates costs one.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np

L2, COSINE = 0, 1


def _dist_row(X, q, metric):
    """FP64 distances from one query vector to every data vector (Def. 1)."""
    Xd = np.asarray(X, np.float64)
    qd = np.asarray(q, np.float64)
    if metric == L2:
        return np.sqrt(((Xd - qd) ** 2).sum(axis=1))
    nx = np.linalg.norm(Xd, axis=1)
    nq = np.linalg.norm(qd)
    return 1.0 - (Xd @ qd) / (nx * nq)


def _dist(a, b, metric):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if metric == L2:
        return float(np.sqrt(((a - b) ** 2).sum()))
    return float(1.0 - (a @ b) / (np.linalg.norm(a) * np.linalg.norm(b)))


@dataclass
class NNMap:
    witness: np.ndarray  # [nq] int32: nearest data vector
    wdist: np.ndarray    # [nq] float64: its distance
    ood: np.ndarray      # [nq] uint8


@dataclass
class NNMapResult:
    offsets: np.ndarray
    ids: np.ndarray
    dists: np.ndarray
    steps: np.ndarray
    hybrid: np.ndarray

    def row(self, q):
        return self.ids[self.offsets[q]:self.offsets[q + 1]]


def nnmap_build(X, Q, adj_x, metric: int = L2) -> NNMap:
    """Witness, witness distance and OOD bit of every query against X, whose own
    graph is adj_x ([nx][R] data ids, -1 padded)."""
    X = np.asarray(X, np.float32)
    Q = np.asarray(Q, np.float32)
    adj_x = np.asarray(adj_x, np.int32)
    nq, R = Q.shape[0], adj_x.shape[1]
    w = np.zeros(nq, np.int32)
    wd = np.zeros(nq, np.float64)
    ood = np.zeros(nq, np.uint8)
    for q in range(nq):
        dr = _dist_row(X, Q[q], metric)
        order = np.lexsort((np.arange(len(dr)), dr))  # ascending (dist, id)
        w[q] = order[0]
        wd[q] = dr[order[0]]
        n1 = [int(v) for v in order[:R]]
        inn1 = set(n1)
        d1 = float(np.mean([dr[v] for v in n1]))
        pairs = []
        for v in n1:
            for u in adj_x[v]:
                if u < 0 or int(u) in inn1:
                    continue
                pairs.append(_dist(X[v], X[u], metric))
        if pairs:
            d2 = float(np.mean(pairs))
            ood[q] = 1 if d2 > 0 and d1 / d2 > 1.5 else 0
    return NNMap(w, wd, ood)


def nnmap_join(X, Q, adj_x, nm: NNMap, eps: float, *, metric: int = L2, hybrid: str = "adapt",
               hybrid_beam_size: int = 256) -> NNMapResult:
    """The join of every query at threshold eps.  hybrid: "adapt" (the OOD
    bit), "force" (every query) or "off" (the BFS closure for every query)."""
    X = np.asarray(X, np.float32)
    Q = np.asarray(Q, np.float32)
    adj_x = np.asarray(adj_x, np.int32)
    nq = Q.shape[0]
    rows, rdists = [], []
    steps = np.zeros(nq, np.int64)
    hyb_out = np.zeros(nq, np.uint8)
    for q in range(nq):
        if nm.wdist[q] >= eps:  # certified empty: no distance computed
            rows.append(np.zeros(0, np.int32))
            rdists.append(np.zeros(0))
            continue
        hyb = {"adapt": bool(nm.ood[q]), "force": True, "off": False}[hybrid]
        hyb_out[q] = 1 if hyb else 0
        s = int(nm.witness[q])
        seen = {s: float(nm.wdist[q])}
        res = [s]
        heap = [(float(nm.wdist[q]), s)]  # min-queue on (dist, id)
        nsteps = 0
        while heap:
            _, u = heapq.heappop(heap)
            for v in adj_x[u]:
                v = int(v)
                if v < 0 or v in seen:
                    continue
                dv = _dist(X[v], Q[q], metric)
                nsteps += 1
                seen[v] = dv
                if dv < eps:
                    heapq.heappush(heap, (dv, v))
                    res.append(v)
                elif hyb:
                    heapq.heappush(heap, (dv, v))
                    if len(heap) > hybrid_beam_size:
                        # drop the largest (dist, id): out of range, never a result
                        heap.remove(max(heap))
                        heapq.heapify(heap)
        res = np.array(sorted(res), np.int32)
        rows.append(res)
        rdists.append(np.array([seen[int(v)] for v in res]))
        steps[q] = nsteps
    offsets = np.zeros(nq + 1, np.int64)
    offsets[1:] = np.cumsum([len(r) for r in rows])
    ids = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    dists = np.concatenate(rdists) if rdists else np.zeros(0)
    return NNMapResult(offsets, ids.astype(np.int32), dists, steps, hyb_out)
