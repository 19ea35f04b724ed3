"""Plain FP64 CPU oracle of the vector epsilon-join (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and it shares no code
with that path: the arithmetic lives in ``vj_oracle.c`` (plain single-threaded
loops, FP64 accumulation) and this module only marshals numpy arrays into it.
``nnmap.py`` holds the oracle of the NN-Map design in plain Python (small
inputs only).

Naming follows the build's convention: ``X`` = data vectors (node ids
``0..nx-1``), ``Q`` = query vectors (node ids ``nx..nx+nq-1``); the paper
calls these Y and X respectively (Def. 1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vj_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libvjoracle.so")

L2, COSINE = 0, 1
WS_NONE, WS_HARD, WS_SOFT, WS_SELF = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compile vj_oracle.c into a shared library beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        p = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.vjo_dist.restype = dbl
        lib.vjo_dist.argtypes = [p, p, i32, i32]
        lib.vjo_nlj.restype = i64
        lib.vjo_nlj.argtypes = [p, i64, p, i64, i32, i32, dbl, p, p, p]
        lib.vjo_knn_rows.restype = None
        lib.vjo_knn_rows.argtypes = [p, i64, p, i64, i32, i32, i32, p, i64, p, p]
        lib.vjo_build_graph.restype = C.c_int32
        lib.vjo_build_graph.argtypes = [p, i64, p, i64, i32, i32, i32, i32, p, p, p]
        lib.vjo_mst.restype = dbl
        lib.vjo_mst.argtypes = [p, i64, p, i64, i32, i32, p, i32, C.c_int32, p, p, p]
        lib.vjo_ood.restype = i32
        lib.vjo_ood.argtypes = [p, i64, p, i32, i32, p, i32, i64, p, p]
        lib.vjo_join.restype = i64
        lib.vjo_join.argtypes = [p, i64, p, i64, i32, i32, p, i32, C.c_int32, p, i64, p, p, dbl, p]
        lib.vjo_nnmap_build.restype = None
        lib.vjo_nnmap_build.argtypes = [p, i64, p, i64, i32, i32, p, i32, p, p, p]
        lib.vjo_nnmap_join.restype = i64
        lib.vjo_nnmap_join.argtypes = [p, i64, p, i64, i32, i32, p, i32, p, p, p, i32, i32, dbl, p, p, p, i64, p, p]
        _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Cfg(C.Structure):
    _fields_ = [
        ("work_sharing", C.c_int),
        ("force_hybrid", C.c_int),
        ("adapt_hybrid", C.c_int),
        ("greedy_beam_size", C.c_int),
        ("conv_threshold", C.c_int),
        ("hybrid_beam_size", C.c_int),
        ("route", C.c_void_p),
        ("beam", C.c_void_p),
        ("separate", C.c_int),
        ("hybrid_seed_best", C.c_int),
    ]


class _Out(C.Structure):
    _fields_ = [
        ("offsets", C.c_void_p),
        ("ids", C.c_void_p),
        ("dists", C.c_void_p),
        ("cap", C.c_int64),
        ("steps", C.c_void_p),
        ("cache", C.c_void_p),
        ("hybrid", C.c_void_p),
        ("expansions", C.c_void_p),
    ]


def dist(a, b, metric: int = L2) -> float:
    """Def. 1 distance of two vectors, FP64."""
    a, b = _f32(a), _f32(b)
    return _load().vjo_dist(_ptr(a), _ptr(b), a.shape[-1], metric)


def nlj(X, Q, eps: float, metric: int = L2):
    """Exact nested-loop join (Sec. 3.2): CSR (offsets[nq+1], ids, dists) by query."""
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    lib = _load()
    offsets = np.zeros(nq + 1, np.int64)
    total = lib.vjo_nlj(_ptr(X), nx, _ptr(Q), nq, d, metric, float(eps), _ptr(offsets), None, None)
    ids = np.zeros(max(total, 1), np.int32)
    dists = np.zeros(max(total, 1), np.float64)
    lib.vjo_nlj(_ptr(X), nx, _ptr(Q), nq, d, metric, float(eps), _ptr(offsets), _ptr(ids), _ptr(dists))
    return offsets, ids[:total], dists[:total]


def knn_rows(X, Q, K: int, rows, metric: int = L2):
    """Exact K nearest other nodes of the merged set for the given node ids."""
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    ids = np.zeros((len(rows), K), np.int32)
    dd = np.zeros((len(rows), K), np.float64)
    _load().vjo_knn_rows(_ptr(X), nx, _ptr(Q), nq, d, metric, K, _ptr(rows), len(rows), _ptr(ids), _ptr(dd))
    return ids, dd


def build_graph(X, Q, R: int, K: int, metric: int = L2, knn_ids=None):
    """Merged-index graph (kNN -> RNG prune -> reverse edges -> entry).

    Returns (adj[n][R] int32 -1 padded, entry, pruned[n][R]).
    """
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    n = nx + nq
    adj = np.zeros((n, R), np.int32)
    pruned = np.zeros((n, R), np.int32)
    kn = None if knn_ids is None else np.ascontiguousarray(knn_ids, dtype=np.int32)
    entry = _load().vjo_build_graph(_ptr(X), nx, _ptr(Q), nq, d, metric, K, R, _ptr(kn), _ptr(pruned), _ptr(adj))
    return adj, int(entry), pruned


def mst(X, Q, adj, entry: int, metric: int = L2):
    """Prim MST over queries + star edges. Returns (parent, order, depth, total_weight)."""
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    R = adj.shape[1]
    parent = np.full(nq, -2, np.int32)
    order = np.full(nq, -1, np.int32)
    depth = np.zeros(nq, np.int32)
    w = _load().vjo_mst(_ptr(X), nx, _ptr(Q), nq, d, metric, _ptr(adj), R, int(entry), _ptr(parent), _ptr(order), _ptr(depth))
    return parent, order, depth, w


def separate_mst(X, Q, adj_q, entry: int, metric: int = L2):
    """Order and parents of separate-index work sharing (Sec. 3.2 WS, Alg. 2):
    the MST over the query graph G_X (adj_q: [nq][R] query ids, -1 padded)
    plus an edge from the data entry s_Y to every query, rooted at s_Y.
    Returns (parent, order, depth, total_weight) as `mst` does."""
    X, Q = _f32(X), _f32(Q)
    nx, nq = X.shape[0], Q.shape[0]
    adj_q = np.asarray(adj_q, np.int32)
    R = adj_q.shape[1]
    # the same Prim routine, on a node set whose query rows hold G_X's edges
    adj_m = np.full((nx + nq, R), -1, np.int32)
    adj_m[nx:] = np.where(adj_q >= 0, adj_q + nx, -1)
    return mst(X, Q, adj_m, entry, metric)


def ood(X, Q, adj, node: int, metric: int = L2):
    """OOD predictor of Sec. 4.4 for merged node id `node`: (flag, d1, d2)."""
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    d1 = C.c_double()
    d2 = C.c_double()
    f = _load().vjo_ood(_ptr(X), nx, _ptr(Q), d, metric, _ptr(adj), adj.shape[1], int(node), C.byref(d1), C.byref(d2))
    return int(f), d1.value, d2.value


@dataclass
class JoinResult:
    offsets: np.ndarray
    ids: np.ndarray
    dists: np.ndarray
    steps: np.ndarray
    cache: np.ndarray
    hybrid: np.ndarray
    expansions: np.ndarray

    def row(self, q):
        return self.ids[self.offsets[q]:self.offsets[q + 1]]


def join(X, Q, adj, entry: int, eps: float, *, metric: int = L2, work_sharing: int = WS_SELF,
         force_hybrid: bool = False, adapt_hybrid: bool = False, greedy_beam_size: int = 256,
         conv_threshold: int = 10, hybrid_beam_size: int = 256, order=None, parent=None,
         queries=None, route=None, beam=None, separate: bool = False,
         hybrid_seed_best: bool = False) -> JoinResult:
    """Alg. 1 VectorJoin on the merged index.

    route/beam (optional, per query) replace Alg. 6's rule with a plan:
    route[q] = 1 sends q to the brute-force scan after its greedy phase
    (hybrid flag 2), beam[q] > 0 runs the hybrid expansion with that queue
    size, beam[q] = 0 the BFS expansion, beam[q] = -1 no expansion phase
    (an expansion budget of zero: the row is I after the greedy phase, flag 3).

    order/parent default to the MST of `mst()` when work sharing is hard/soft,
    else to index order.

    hybrid_seed_best=True starts a hybrid expansion whose greedy phase found no
    in-range point from the closest visited data node (a variant; the literal
    reading returns an empty row).

    separate=True runs the separate-index execution (Sec. 3.2 INLJ, HWS/SWS on
    a per-set index): adj is the data graph G_Y ([nx][R]) with entry s_Y, and
    with hard/soft sharing order/parent must be given (`separate_mst`).  `queries` (optional) restricts the run to that list of
    query indices, processed in the given order; it must be closed under MST
    parents when sharing is on (a set of whole subtrees).
    """
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    R = adj.shape[1]
    if separate and work_sharing in (WS_HARD, WS_SOFT) and (order is None or parent is None):
        raise ValueError("separate-index sharing needs the order and parents of separate_mst()")
    if work_sharing in (WS_HARD, WS_SOFT) and (order is None or parent is None):
        p, o, _, _ = mst(X, Q, adj, entry, metric)
        parent = p if parent is None else parent
        order = o if order is None else order
    if queries is not None:
        order = np.ascontiguousarray(queries, dtype=np.int32)
    route_a = None if route is None else np.ascontiguousarray(route, dtype=np.uint8)
    beam_a = None if beam is None else np.ascontiguousarray(beam, dtype=np.int32)
    cfg = _Cfg(work_sharing, int(force_hybrid), int(adapt_hybrid), greedy_beam_size, conv_threshold, hybrid_beam_size,
               _ptr(route_a), _ptr(beam_a), int(separate), int(hybrid_seed_best))
    lib = _load()
    order_a = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    parent_a = None if parent is None else np.ascontiguousarray(parent, dtype=np.int32)
    nrun = nq if order_a is None else len(order_a)
    offsets = np.zeros(nq + 1, np.int64)
    steps = np.zeros(nq, np.int64)
    cache = np.full(nq, -1, np.int32)
    hyb = np.zeros(nq, np.uint8)
    exps = np.zeros(nq, np.int64)
    cap = 1 << 16
    while True:
        ids = np.zeros(cap, np.int32)
        dists = np.zeros(cap, np.float64)
        out = _Out(_ptr(offsets), _ptr(ids), _ptr(dists), cap, _ptr(steps), _ptr(cache), _ptr(hyb), _ptr(exps))
        total = lib.vjo_join(_ptr(X), nx, _ptr(Q), nq, d, metric, _ptr(adj), R, int(entry), _ptr(order_a),
                             nrun, _ptr(parent_a), C.byref(cfg), float(eps), C.byref(out))
        if total <= cap:
            break
        cap = int(total)
    return JoinResult(offsets, ids[:total], dists[:total], steps, cache, hyb, exps)


def recall(offsets, ids, ex_offsets, ex_ids):
    """Pooled recall |R n E| / |E| over all queries, and the per-query mean.

    An empty exact row counts as recall 1 in the per-query mean (Def. 2 leaves
    it undefined).
    """
    nq = len(ex_offsets) - 1
    hit = 0
    per = np.ones(nq)
    for q in range(nq):
        e = ex_ids[ex_offsets[q]:ex_offsets[q + 1]]
        r = ids[offsets[q]:offsets[q + 1]]
        if len(e) == 0:
            continue
        h = len(np.intersect1d(e, r, assume_unique=True))
        hit += h
        per[q] = h / len(e)
    tot = int(ex_offsets[-1])
    return (hit / tot if tot else 1.0), float(per.mean())


def nnmap_build_c(X, Q, adj_x, metric: int = L2):
    """NN-Map witnesses, witness distances and OOD bits (Sec. NN-Map), in C;
    the same readings as ``nnmap.nnmap_build``."""
    from .nnmap import NNMap
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    adj_x = np.ascontiguousarray(adj_x, dtype=np.int32)
    w = np.zeros(nq, np.int32)
    wd = np.zeros(nq, np.float64)
    ood = np.zeros(nq, np.uint8)
    _load().vjo_nnmap_build(_ptr(X), nx, _ptr(Q), nq, d, metric, _ptr(adj_x), adj_x.shape[1], _ptr(w), _ptr(wd),
                            _ptr(ood))
    return NNMap(w, wd, ood)


def nnmap_join_c(X, Q, adj_x, nm, eps: float, *, metric: int = L2, hybrid: str = "adapt",
                 hybrid_beam_size: int = 256):
    """The NN-Map join (Sec. NN-Map) in C; the same semantics as ``nnmap.nnmap_join``."""
    from .nnmap import NNMapResult
    X, Q = _f32(X), _f32(Q)
    nx, d = X.shape
    nq = Q.shape[0]
    adj_x = np.ascontiguousarray(adj_x, dtype=np.int32)
    mode = {"off": 0, "adapt": 1, "force": 2}[hybrid]
    w = np.ascontiguousarray(nm.witness, np.int32)
    wd = np.ascontiguousarray(nm.wdist, np.float64)
    ood = np.ascontiguousarray(nm.ood, np.uint8)
    offsets = np.zeros(nq + 1, np.int64)
    steps = np.zeros(nq, np.int64)
    hyb = np.zeros(nq, np.uint8)
    cap = 1 << 16
    while True:
        ids = np.zeros(cap, np.int32)
        dists = np.zeros(cap, np.float64)
        total = _load().vjo_nnmap_join(_ptr(X), nx, _ptr(Q), nq, d, metric, _ptr(adj_x), adj_x.shape[1], _ptr(w),
                                       _ptr(wd), _ptr(ood), mode, int(hybrid_beam_size), float(eps), _ptr(offsets),
                                       _ptr(ids), _ptr(dists), cap, _ptr(steps), _ptr(hyb))
        if total <= cap:
            break
        cap = int(total)
    return NNMapResult(offsets, ids[:total], dists[:total], steps, hyb)


def transpose_csr(offsets, ids, dists, n_cols: int):
    """Rows <-> columns of a CSR pair list (pairs ascending by column id per row)."""
    offsets = np.asarray(offsets, np.int64)
    rows = np.repeat(np.arange(len(offsets) - 1, dtype=np.int64), np.diff(offsets))
    cols = np.asarray(ids, np.int64)
    order = np.lexsort((rows, cols))  # by new row (old column), then new column (old row)
    t_off = np.zeros(n_cols + 1, np.int64)
    np.add.at(t_off, cols + 1, 1)
    return np.cumsum(t_off), rows[order].astype(np.int32), np.asarray(dists, np.float64)[order]


def join_switched(X, Q, eps: float, *, degree: int, knn_k: int, metric: int = L2, **kw):
    """Query-data switching (the large-threshold discussion after Sec. 5): the
    join X |><| Q equals Q |><| X, so the merged-index join runs with the roles
    swapped (Q as data, X as queries, on the merged graph of both) and its
    pair list is transposed back to one row per query of Q.  Returns
    (offsets, ids, dists) over Q's queries.  kw: the options of `join`."""
    X, Q = _f32(X), _f32(Q)
    adj, entry, _ = build_graph(Q, X, degree, knn_k, metric)
    r = join(Q, X, adj, entry, eps, metric=metric, **kw)
    return transpose_csr(r.offsets, r.ids, r.dists, Q.shape[0])
