"""Python binding of libvj.so (include/vj.h): argument marshalling only.

Every function here forwards to the C ABI of the CUDA library; no step of a
build or a join runs in Python.  ``load()`` raises ``VjLibraryMissing`` when
the library has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvj.so")

VJ_OK, VJ_ERR_ARG, VJ_ERR_OOM, VJ_ERR_CUDA, VJ_ERR_TIMEOUT, VJ_ERR_STATE = range(6)
VJ_L2, VJ_COSINE = 0, 1
VJ_WS_NONE, VJ_WS_HARD, VJ_WS_SOFT, VJ_WS_SELF = 0, 1, 2, 3
VJ_PREC_FP32, VJ_PREC_BF16, VJ_PREC_FP8 = 0, 1, 2

# every function declared in include/vj.h
EXPORTS = ["vj_mlp_create", "vj_mlp_num_params", "vj_mlp_get_params", "vj_mlp_set_params", "vj_mlp_loss_grad",
           "vj_mlp_train", "vj_mlp_predict", "vj_mlp_free", "vj_features", "vj_attach_predictor",
           "vj_predictor_outputs",
           "vj_default_params", "vj_build", "vj_set_stream", "vj_set_join_params", "vj_set_plan", "vj_join",
           "vj_join_device", "vj_join_batch", "vj_join_exact", "vj_join_exact_noalloc", "vj_export_graph", "vj_export_knn",
           "vj_index_info", "vj_build_info", "vj_result_free", "vj_free", "vj_last_error", "vj_set_wait_test",
           "vj_default_train_params", "vj_predictor_labels", "vj_train_predictor", "vj_join_switched",
           "vj_export_nnmap", "vj_autotune", "vj_set_tuning"]

NOALLOC_MAX_QUERIES = 1 << 20


class VjLibraryMissing(RuntimeError):
    pass


class VjError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"vj status {status}: {msg}")
        self.status = status


VJ_TUNE_MAX = 16


class vj_tune_report(C.Structure):
    _fields_ = [("n", C.c_int), ("lanes", C.c_int * VJ_TUNE_MAX), ("slots", C.c_int * VJ_TUNE_MAX),
                ("inflight", C.c_int * VJ_TUNE_MAX), ("blocks", C.c_int * VJ_TUNE_MAX),
                ("probe_ring", C.c_int * VJ_TUNE_MAX), ("probe_bulk", C.c_int * VJ_TUNE_MAX),
                ("ms", C.c_double * VJ_TUNE_MAX),
                ("valid", C.c_int * VJ_TUNE_MAX), ("chosen", C.c_int)]


class vj_params(C.Structure):
    _fields_ = [("degree", C.c_int), ("knn_k", C.c_int), ("greedy_beam", C.c_int), ("conv_threshold", C.c_int),
                ("hybrid_beam", C.c_int), ("work_sharing", C.c_int), ("adapt_hybrid", C.c_int),
                ("force_hybrid", C.c_int), ("precision", C.c_int), ("learned", C.c_int),
                ("route_bruteforce", C.c_int), ("input_on_device", C.c_int), ("seed", C.c_uint64),
                ("gather", C.c_int), ("hybrid_seed_best", C.c_int), ("nnmap", C.c_int), ("separate", C.c_int),
                ("scan", C.c_int)]


class vj_stats(C.Structure):
    _fields_ = [("dist_computations", C.c_int64), ("expansions", C.c_int64), ("adj_rows_read", C.c_int64),
                ("hybrid_queries", C.c_int64), ("rechecks", C.c_int64), ("spill_queries", C.c_int64),
                ("ms_traverse", C.c_double), ("ms_csr", C.c_double), ("ms_total", C.c_double),
                ("bytes_algorithmic", C.c_int64), ("kernel_launches", C.c_int64), ("ms_scan", C.c_double),
                ("scan_candidates", C.c_int64), ("ms_prologue", C.c_double),
                ("sws_restarts", C.c_int64), ("ms_route", C.c_double), ("ms_sws", C.c_double * 3)]


class vj_train_params(C.Structure):
    _fields_ = [("n_ladder", C.c_int), ("ladder", C.c_int * 8), ("query_recall", C.c_float),
                ("pooled_recall", C.c_float), ("scan_row_cost", C.c_float), ("h1", C.c_int), ("h2", C.c_int),
                ("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("seed", C.c_uint64)]


class vj_train_report(C.Structure):
    _fields_ = [("n", C.c_int64), ("routed", C.c_int64), ("per_budget", C.c_int64 * 8), ("ladder_run", C.c_int),
                ("scan_row_cost", C.c_double), ("final_loss", C.c_double), ("ms_labels", C.c_double),
                ("ms_train", C.c_double)]


class vj_result(C.Structure):
    _fields_ = [("nq", C.c_int64), ("nnz", C.c_int64), ("offsets", C.POINTER(C.c_int64)),
                ("ids", C.POINTER(C.c_int32)), ("dists", C.POINTER(C.c_float)), ("steps", C.POINTER(C.c_int32)),
                ("cache", C.POINTER(C.c_int32)), ("hybrid", C.POINTER(C.c_uint8)), ("on_device", C.c_int),
                ("stats", vj_stats)]


_lib = None


def load():
    """Load libvj.so (raises VjLibraryMissing if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise VjLibraryMissing(f"{LIB_PATH} is missing: run paper_2603_16360_b300/build.py (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    P, I64, I = C.c_void_p, C.c_int64, C.c_int
    lib.vj_default_params.argtypes = [C.POINTER(vj_params)]
    lib.vj_default_params.restype = None
    lib.vj_build.argtypes = [P, I64, P, I64, I, I, C.POINTER(vj_params), C.POINTER(P)]
    lib.vj_build.restype = I
    lib.vj_set_stream.argtypes = [P, P]
    lib.vj_set_stream.restype = I
    lib.vj_set_join_params.argtypes = [P, C.POINTER(vj_params)]
    lib.vj_set_join_params.restype = I
    lib.vj_set_plan.argtypes = [P, P, P]
    lib.vj_set_plan.restype = I
    lib.vj_mlp_create.argtypes = [I, I, I, C.c_uint64, C.POINTER(P)]
    lib.vj_mlp_create.restype = I
    lib.vj_mlp_num_params.argtypes = [P]
    lib.vj_mlp_num_params.restype = I64
    lib.vj_mlp_get_params.argtypes = [P, P, P, P]
    lib.vj_mlp_get_params.restype = I
    lib.vj_mlp_set_params.argtypes = [P, P, P, P]
    lib.vj_mlp_set_params.restype = I
    lib.vj_mlp_loss_grad.argtypes = [P, P, P, P, I64, C.POINTER(C.c_double), P]
    lib.vj_mlp_loss_grad.restype = I
    lib.vj_mlp_train.argtypes = [P, P, P, P, I64, I, I, C.c_float, C.c_uint64, C.POINTER(C.c_double)]
    lib.vj_mlp_train.restype = I
    lib.vj_mlp_predict.argtypes = [P, P, I64, P]
    lib.vj_mlp_predict.restype = I
    lib.vj_mlp_free.argtypes = [P]
    lib.vj_mlp_free.restype = None
    lib.vj_features.argtypes = [P, C.c_float, P]
    lib.vj_features.restype = I
    lib.vj_attach_predictor.argtypes = [P, P, C.c_float, I]
    lib.vj_attach_predictor.restype = I
    lib.vj_predictor_outputs.argtypes = [P, C.c_float, P]
    lib.vj_predictor_outputs.restype = I
    lib.vj_join_switched.argtypes = [P, C.c_float, C.POINTER(C.POINTER(vj_result))]
    lib.vj_join_switched.restype = I
    for fn in ("vj_join", "vj_join_device"):
        getattr(lib, fn).argtypes = [P, C.c_float, I, C.POINTER(C.POINTER(vj_result))]
        getattr(lib, fn).restype = I
    lib.vj_join_batch.argtypes = [P, P, I, P]
    lib.vj_join_batch.restype = I
    lib.vj_join_exact.argtypes = [P, C.c_float, C.POINTER(C.POINTER(vj_result))]
    lib.vj_join_exact.restype = I
    lib.vj_join_exact_noalloc.argtypes = [P, I64, P, I64, I, I, C.c_float, P, P, P, I64, C.POINTER(C.c_int64), P]
    lib.vj_join_exact_noalloc.restype = I
    lib.vj_export_graph.argtypes = [P, P, P, P, P, P]
    lib.vj_export_graph.restype = I
    lib.vj_export_knn.argtypes = [P, P, P]
    lib.vj_export_knn.restype = I
    lib.vj_export_nnmap.argtypes = [P, P, P, P]
    lib.vj_export_nnmap.restype = I
    lib.vj_index_info.argtypes = [P, P, P, P, P, P, P]
    lib.vj_index_info.restype = I
    lib.vj_build_info.argtypes = [P, P, P, P, P]
    lib.vj_build_info.restype = I
    lib.vj_result_free.argtypes = [C.POINTER(vj_result)]
    lib.vj_result_free.restype = None
    lib.vj_free.argtypes = [P]
    lib.vj_free.restype = None
    lib.vj_default_train_params.argtypes = [C.POINTER(vj_train_params)]
    lib.vj_default_train_params.restype = None
    lib.vj_predictor_labels.argtypes = [P, C.c_float, P, I64, C.POINTER(vj_train_params), P, P,
                                        C.POINTER(vj_train_report)]
    lib.vj_predictor_labels.restype = I
    lib.vj_train_predictor.argtypes = [P, C.c_float, P, I64, C.POINTER(vj_train_params), C.POINTER(P),
                                       C.POINTER(vj_train_report)]
    lib.vj_train_predictor.restype = I
    lib.vj_set_wait_test.argtypes = [P, C.c_longlong, I64]
    lib.vj_set_wait_test.restype = I
    lib.vj_autotune.argtypes = [P, C.c_float, I, C.POINTER(vj_tune_report)]
    lib.vj_autotune.restype = I
    lib.vj_set_tuning.argtypes = [P, I, I, I, I, I, I]
    lib.vj_set_tuning.restype = I
    lib.vj_last_error.argtypes = []
    lib.vj_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(st):
    if st != VJ_OK:
        raise VjError(st, load().vj_last_error().decode(errors="replace"))


def default_params(**kw) -> vj_params:
    p = vj_params()
    load().vj_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@dataclass
class Result:
    """Host copy of a vj_result (CSR by query plus per-query arrays)."""
    offsets: np.ndarray
    ids: np.ndarray
    dists: np.ndarray
    steps: np.ndarray
    cache: np.ndarray
    hybrid: np.ndarray
    stats: dict = field(default_factory=dict)

    def row(self, q):
        return self.ids[self.offsets[q]:self.offsets[q + 1]]

    @property
    def nnz(self) -> int:
        return len(self.ids)


def _stats(s: vj_stats) -> dict:
    out = {}
    for name, _ in vj_stats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


class _ResultOwner:
    """Releases a host vj_result once no array viewing its buffers is left."""

    def __init__(self, rp):
        self.rp = rp

    def __del__(self):
        try:
            load().vj_result_free(self.rp)
        except Exception:
            pass


def _host_result(rp) -> Result:
    """Numpy views of the library's page-locked result arrays (no copy)."""
    r = rp.contents
    nq, nnz = r.nq, r.nnz
    owner = _ResultOwner(rp)

    def arr(ptr, n, ctype, dt):
        if n == 0:
            return np.empty(0, dt)
        buf = (ctype * n).from_address(C.cast(ptr, C.c_void_p).value)
        buf._owner = owner  # the buffer lives while any view of it does
        return np.frombuffer(buf, dtype=dt)

    return Result(arr(r.offsets, nq + 1, C.c_int64, np.int64), arr(r.ids, nnz, C.c_int32, np.int32),
                  arr(r.dists, nnz, C.c_float, np.float32), arr(r.steps, nq, C.c_int32, np.int32),
                  arr(r.cache, nq, C.c_int32, np.int32), arr(r.hybrid, nq, C.c_uint8, np.uint8), _stats(r.stats))


class DeviceResult:
    """A vj_result whose arrays live in device memory; free() releases it."""

    def __init__(self, rp):
        self._rp = rp
        r = rp.contents
        self.nq, self.nnz, self.stats = r.nq, r.nnz, _stats(r.stats)
        self.offsets_ptr = C.cast(r.offsets, C.c_void_p).value
        self.ids_ptr = C.cast(r.ids, C.c_void_p).value
        self.dists_ptr = C.cast(r.dists, C.c_void_p).value

    def free(self):
        if self._rp is not None:
            load().vj_result_free(self._rp)
            self._rp = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Index:
    """An opaque vj_index built by vj_build (offline merged-index build)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self):
        nx, nq = C.c_int64(), C.c_int64()
        d, deg, k, md = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(load().vj_index_info(self._h, C.byref(nx), C.byref(nq), C.byref(d), C.byref(deg), C.byref(k),
                                    C.byref(md)))
        return {"nx": nx.value, "nq": nq.value, "d": d.value, "degree": deg.value, "knn_k": k.value,
                "max_depth": md.value}

    def build_info(self):
        tc, unc, ms, mk = C.c_int(), C.c_int64(), C.c_double(), C.c_double()
        _check(load().vj_build_info(self._h, C.byref(tc), C.byref(unc), C.byref(ms), C.byref(mk)))
        return {"knn_tensor_cores": bool(tc.value), "knn_uncertified": unc.value, "ms_build": ms.value,
                "ms_knn": mk.value}

    def free(self):
        if self._h:
            load().vj_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vj_build(X, Q, metric: int = VJ_L2, params: vj_params | None = None, **kw) -> Index:
    """Build the merged index over data X [nx, d] and queries Q [nq, d].

    X and Q may be numpy arrays (host) or CUDA tensors exposing
    ``data_ptr()`` (device, float32, contiguous).
    """
    lib = load()
    p = params if params is not None else default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    if hasattr(X, "data_ptr"):
        assert X.is_cuda and Q.is_cuda and X.is_contiguous() and Q.is_contiguous()
        p.input_on_device = 1
        xp, qp = X.data_ptr(), Q.data_ptr()
        nx, d = X.shape
        nq = Q.shape[0]
        keep = (X, Q)
    else:
        X = np.ascontiguousarray(X, np.float32)
        Q = np.ascontiguousarray(Q, np.float32)
        p.input_on_device = 0
        xp, qp = X.ctypes.data, Q.ctypes.data
        nx, d = X.shape
        nq = Q.shape[0]
        keep = (X, Q)
    h = C.c_void_p()
    _check(lib.vj_build(xp, nx, qp, nq, d, metric, C.byref(p), C.byref(h)))
    del keep
    return Index(h)


def vj_set_stream(ix: Index, stream_ptr: int):
    _check(load().vj_set_stream(ix.handle, C.c_void_p(stream_ptr)))


def vj_set_join_params(ix: Index, params: vj_params | None = None, **kw):
    p = params if params is not None else default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    _check(load().vj_set_join_params(ix.handle, C.byref(p)))


NFEAT = 7


class MLP:
    """The learned route / budget predictor (vj_mlp in include/vj.h)."""

    def __init__(self, din: int, h1: int = 256, h2: int = 256, seed: int = 0):
        h = C.c_void_p()
        _check(load().vj_mlp_create(din, h1, h2, seed, C.byref(h)))
        self._h, self.din, self.h1, self.h2 = h, din, h1, h2

    @property
    def handle(self):
        return self._h

    @classmethod
    def _adopt(cls, handle, din: int, h1: int, h2: int):
        """Wrap a predictor the library created (vj_train_predictor)."""
        m = cls.__new__(cls)
        m._h, m.din, m.h1, m.h2 = handle, din, h1, h2
        return m

    def num_params(self) -> int:
        return int(load().vj_mlp_num_params(self._h))

    def get_params(self):
        flat = np.zeros(self.num_params(), np.float32)
        mu = np.zeros(self.din, np.float32)
        sd = np.zeros(self.din, np.float32)
        _check(load().vj_mlp_get_params(self._h, flat.ctypes.data, mu.ctypes.data, sd.ctypes.data))
        return flat, mu, sd

    def set_params(self, flat, mu=None, sd=None):
        flat = np.ascontiguousarray(flat, np.float32)
        mu_a = None if mu is None else np.ascontiguousarray(mu, np.float32)
        sd_a = None if sd is None else np.ascontiguousarray(sd, np.float32)
        _check(load().vj_mlp_set_params(self._h, flat.ctypes.data, None if mu_a is None else mu_a.ctypes.data,
                                         None if sd_a is None else sd_a.ctypes.data))

    def loss_grad(self, x, t_reg, t_cls):
        x = np.ascontiguousarray(x, np.float32)
        tr = np.ascontiguousarray(t_reg, np.float32)
        tc = np.ascontiguousarray(t_cls, np.float32)
        loss = C.c_double()
        g = np.zeros(self.num_params(), np.float32)
        _check(load().vj_mlp_loss_grad(self._h, x.ctypes.data, tr.ctypes.data, tc.ctypes.data, len(x),
                                       C.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, x, t_reg, t_cls, epochs=20, batch=256, lr=1e-3, seed=0) -> float:
        x = np.ascontiguousarray(x, np.float32)
        tr = np.ascontiguousarray(t_reg, np.float32)
        tc = np.ascontiguousarray(t_cls, np.float32)
        loss = C.c_double()
        _check(load().vj_mlp_train(self._h, x.ctypes.data, tr.ctypes.data, tc.ctypes.data, len(x), epochs, batch,
                                   float(lr), seed, C.byref(loss)))
        return loss.value

    def predict(self, x):
        x = np.ascontiguousarray(x, np.float32)
        out = np.zeros((len(x), 2), np.float32)
        _check(load().vj_mlp_predict(self._h, x.ctypes.data, len(x), out.ctypes.data))
        return out

    def free(self):
        if self._h:
            load().vj_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vj_features(ix: Index, eps: float):
    inf = ix.info()
    out = np.zeros((inf["nq"], NFEAT + inf["d"]), np.float32)
    _check(load().vj_features(ix.handle, float(eps), out.ctypes.data))
    return out


def vj_attach_predictor(ix: Index, mlp, route_threshold: float = 0.5, beam_cap: int = 256):
    _check(load().vj_attach_predictor(ix.handle, None if mlp is None else mlp.handle, float(route_threshold),
                                      int(beam_cap)))


def vj_predictor_outputs(ix: Index, eps: float) -> np.ndarray:
    """Outputs [nq, 2] of the attached predictor as the learned prologue computes them."""
    out = np.empty((ix.info()["nq"], 2), np.float32)
    _check(load().vj_predictor_outputs(ix.handle, float(eps), out.ctypes.data))
    return out


def train_params(**kw) -> vj_train_params:
    """vj_train_params with the library's defaults, fields overridden by kw
    (ladder may be a sequence: it also sets n_ladder)."""
    tp = vj_train_params()
    load().vj_default_train_params(C.byref(tp))
    for k, v in kw.items():
        if k == "ladder":
            v = list(v)
            if not 1 <= len(v) <= 8:
                raise ValueError("ladder needs 1..8 budgets")
            tp.n_ladder = len(v)
            for i, b in enumerate(v):
                tp.ladder[i] = int(b)
        else:
            setattr(tp, k, v)
    return tp


def _report(rep: vj_train_report) -> dict:
    d = {name: getattr(rep, name) for name, _ in vj_train_report._fields_}
    d["per_budget"] = list(rep.per_budget)
    return d


def vj_predictor_labels(ix: Index, eps: float, rows, **kw):
    """(budget [n] int32, route [n] uint8, report) of the training queries rows."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    tp = train_params(**kw)
    budget = np.zeros(len(r), np.int32)
    route = np.zeros(len(r), np.uint8)
    rep = vj_train_report()
    _check(load().vj_predictor_labels(ix.handle, float(eps), r.ctypes.data, len(r), C.byref(tp), budget.ctypes.data,
                                      route.ctypes.data, C.byref(rep)))
    return budget, route, _report(rep)


def vj_train_predictor(ix: Index, eps: float, rows, **kw):
    """(MLP, report): labels of the training queries rows, then a trained predictor."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    tp = train_params(**kw)
    h = C.c_void_p()
    rep = vj_train_report()
    _check(load().vj_train_predictor(ix.handle, float(eps), r.ctypes.data, len(r), C.byref(tp), C.byref(h),
                                     C.byref(rep)))
    inf = ix.info()
    return MLP._adopt(h, NFEAT + inf["d"], tp.h1, tp.h2), _report(rep)


def vj_set_wait_test(ix: Index, max_polls: int = 0, hold_q: int = -1):
    """Limit the soft-sharing dependency wait (0: default) and hold one query's publication (-1: none)."""
    _check(load().vj_set_wait_test(ix.handle, int(max_polls), int(hold_q)))


def vj_autotune(ix: Index, eps: float, reps: int = 2) -> dict:
    """Time the join at eps under each candidate traversal setting, keep the
    fastest on the index; returns the settings tried and the chosen one."""
    rep = vj_tune_report()
    _check(load().vj_autotune(ix.handle, float(eps), int(reps), C.byref(rep)))
    rows = [{"lanes": rep.lanes[i], "slots": rep.slots[i], "inflight": rep.inflight[i], "blocks": rep.blocks[i],
             "probe_ring": rep.probe_ring[i], "probe_bulk": rep.probe_bulk[i], "ms": rep.ms[i],
             "valid": bool(rep.valid[i])} for i in range(rep.n)]
    return {"settings": rows, "chosen": rep.chosen}


def vj_set_tuning(ix: Index, lanes: int = 0, slots: int = 0, inflight: int = 0, blocks: int = 0,
                  probe_ring: int = 0, probe_bulk: int = 0):
    """Set the traversal setting (0 = default for each field)."""
    _check(load().vj_set_tuning(ix.handle, int(lanes), int(slots), int(inflight), int(blocks), int(probe_ring),
                                int(probe_bulk)))


def vj_set_plan(ix: Index, route=None, beam=None):
    """Per-query plan (route to the brute-force scan, hybrid queue size) for later joins."""
    r = None if route is None else np.ascontiguousarray(route, dtype=np.uint8)
    b = None if beam is None else np.ascontiguousarray(beam, dtype=np.int32)
    _check(load().vj_set_plan(ix.handle, None if r is None else r.ctypes.data, None if b is None else b.ctypes.data))


def vj_join(ix: Index, eps: float, budget: int = 0) -> Result:
    rp = C.POINTER(vj_result)()
    _check(load().vj_join(ix.handle, float(eps), int(budget), C.byref(rp)))
    return _host_result(rp)


def vj_join_switched(ix: Index, eps: float) -> Result:
    """Join on an index built with the roles swapped (vj_build(Q, X)), transposed
    back to one row per original query."""
    rp = C.POINTER(vj_result)()
    _check(load().vj_join_switched(ix.handle, float(eps), C.byref(rp)))
    return _host_result(rp)


def vj_join_device(ix: Index, eps: float, budget: int = 0) -> DeviceResult:
    rp = C.POINTER(vj_result)()
    _check(load().vj_join_device(ix.handle, float(eps), int(budget), C.byref(rp)))
    return DeviceResult(rp)


def vj_join_batch(ixs, eps) -> list:
    """Independent joins of several indexes with fused traversal launches; result i = vj_join(ixs[i], eps[i])."""
    n = len(ixs)
    e = np.ascontiguousarray(eps, dtype=np.float32)
    if e.shape != (n,):
        raise ValueError("eps needs one threshold per index")
    hs = (C.c_void_p * max(n, 1))(*[ix.handle for ix in ixs])
    outs = (C.POINTER(vj_result) * max(n, 1))()
    _check(load().vj_join_batch(C.cast(hs, C.c_void_p), e.ctypes.data, n, C.cast(outs, C.c_void_p)))
    return [_host_result(outs[i]) for i in range(n)]


def vj_join_exact(ix: Index, eps: float) -> Result:
    rp = C.POINTER(vj_result)()
    _check(load().vj_join_exact(ix.handle, float(eps), C.byref(rp)))
    return _host_result(rp)


def vj_join_exact_noalloc(X, Q, eps: float, offsets, ids, dists, metric: int = VJ_L2, stream_ptr: int = 0) -> int:
    """Exact join into caller-owned device buffers, allocating nothing.

    For callers that cannot allocate device memory (a fixed pre-carved memory
    budget, or no tolerance for cudaMalloc/cudaFree locks and syncs).  X, Q,
    offsets (int64, nq+1), ids (int32) and dists (float32) are CUDA tensors the
    caller owns; returns the pair count.  Raises VjError (VJ_ERR_STATE) when the
    pairs exceed len(ids); offsets are complete even then.
    """
    import torch
    ts = {"X": X, "Q": Q, "offsets": offsets, "ids": ids, "dists": dists}
    for name, t in ts.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    devs = {t.device for t in ts.values()}
    if len(devs) != 1 or next(iter(devs)).index != torch.cuda.current_device():
        raise ValueError("every tensor must live on the current CUDA device")
    want = {"X": torch.float32, "Q": torch.float32, "offsets": torch.int64, "ids": torch.int32,
            "dists": torch.float32}
    for name, dt in want.items():
        if ts[name].dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {ts[name].dtype}")
    if X.dim() != 2 or Q.dim() != 2 or X.shape[1] != Q.shape[1]:
        raise ValueError("X and Q must be 2-D with the same number of columns")
    nx, d = X.shape
    nq = Q.shape[0]
    if offsets.dim() != 1 or offsets.numel() < nq + 1:
        raise ValueError(f"offsets needs at least nq + 1 = {nq + 1} entries")
    nnz = C.c_int64(0)
    cap = min(ids.numel(), dists.numel())
    _check(load().vj_join_exact_noalloc(X.data_ptr(), nx, Q.data_ptr(), nq, d, metric, float(eps),
                                        offsets.data_ptr(), ids.data_ptr(), dists.data_ptr(), cap, C.byref(nnz),
                                        C.c_void_p(stream_ptr)))
    return nnz.value


def vj_export_graph(ix: Index):
    """(adj [n, R], entry, parent [nq], order [nq], depth [nq])."""
    inf = ix.info()
    n = inf["nx"] + inf["nq"]
    adj = np.zeros((n, inf["degree"]), np.int32)
    par = np.zeros(inf["nq"], np.int32)
    order = np.zeros(inf["nq"], np.int32)
    depth = np.zeros(inf["nq"], np.int32)
    entry = C.c_int32()
    _check(load().vj_export_graph(ix.handle, adj.ctypes.data, C.addressof(entry), par.ctypes.data,
                                  order.ctypes.data, depth.ctypes.data))
    return adj, entry.value, par, order, depth


def vj_export_knn(ix: Index):
    """(ids [n, K], keys [n, K]); keys are squared distances for L2."""
    inf = ix.info()
    n = inf["nx"] + inf["nq"]
    ids = np.zeros((n, inf["knn_k"]), np.int32)
    keys = np.zeros((n, inf["knn_k"]), np.float32)
    _check(load().vj_export_knn(ix.handle, ids.ctypes.data, keys.ctypes.data))
    return ids, keys


def vj_export_nnmap(ix: Index):
    """(witness [nq] int32, wdist [nq] float64, ood [nq] uint8) of an index
    built with nnmap=1."""
    nq = ix.info()["nq"]
    w = np.zeros(nq, np.int32)
    wd = np.zeros(nq, np.float64)
    ood = np.zeros(nq, np.uint8)
    _check(load().vj_export_nnmap(ix.handle, w.ctypes.data, wd.ctypes.data, ood.ctypes.data))
    return w, wd, ood
