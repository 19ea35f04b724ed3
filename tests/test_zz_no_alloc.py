"""vj_join_exact_noalloc: the exact join for callers that cannot allocate
device memory (services confined to a fixed, pre-carved memory budget, or
paths that cannot take cudaMalloc/cudaFree's locks and device syncs).

The test calls it through the C ABI twice in a row on caller-owned device
buffers and checks both outputs against vj_join_exact, the allocating entry
point, and against the CPU oracle's nested-loop join (FP64), with the
tolerances of the other parity tests: pair ids equal outside the
|dist - eps| <= 1e-4 eps band, distances within 1e-5 relative on every pair
the two results share.  This file sorts last so that a run stopping at its
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu

BAND = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()
    return torch


def _pairs(off, ids):
    return {(q, int(i)) for q in range(len(off) - 1) for i in ids[off[q]:off[q + 1]]}


def _dist_map(off, ids, dists):
    return {(q, int(ids[k])): float(dists[k]) for q in range(len(off) - 1) for k in range(off[q], off[q + 1])}


def _check_shared_dists(got, want, what):
    shared = got.keys() & want.keys()
    assert shared, f"{what}: no shared pair to compare distances on"
    a = np.array([got[k] for k in sorted(shared)])
    b = np.array([want[k] for k in sorted(shared)])
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6, err_msg=what)


@pytest.mark.parametrize("metric", [vj.VJ_L2, vj.VJ_COSINE])
def test_noalloc_matches_allocating_exact_join_twice(torch_cuda, oracle, metric):
    torch = torch_cuda
    w = inputs.uniform_small(201 + metric, 2000, 300, 37, metric=metric)
    from scipy.spatial.distance import cdist
    D = cdist(w.Q.astype(np.float64), w.X.astype(np.float64), "euclidean" if metric == 0 else "cosine")
    eps = float(np.float32(np.partition(D.ravel(), 12 * w.nq)[12 * w.nq]))
    band = set(zip(*[a.tolist() for a in np.nonzero(np.abs(D - eps) <= BAND * eps)]))

    ix = vj.vj_build(w.X, w.Q, metric=metric, params=vj.default_params(degree=12, knn_k=24))
    ref = vj.vj_join_exact(ix, eps)
    ix.free()
    o_off, o_ids, o_d = oracle.nlj(w.X, w.Q, eps, metric)

    X = torch.from_numpy(w.X).cuda()
    Q = torch.from_numpy(w.Q).cuda()
    cap = int(ref.offsets[-1]) + 64
    for call in range(2):
        off = torch.full((w.nq + 1,), -1, dtype=torch.int64, device="cuda")
        ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        dd = torch.zeros(cap, dtype=torch.float32, device="cuda")
        nnz = vj.vj_join_exact_noalloc(X, Q, eps, off, ids, dd, metric=metric)
        torch.cuda.synchronize()
        o = off.cpu().numpy()
        i = ids.cpu().numpy()[:nnz]
        dv = dd.cpu().numpy()[:nnz]
        assert o[-1] == nnz
        diff = (_pairs(o, i) ^ _pairs(ref.offsets, ref.ids)) - band
        assert not diff, f"call {call}: {len(diff)} pairs differ from vj_join_exact"
        diff = (_pairs(o, i) ^ _pairs(o_off, o_ids)) - band
        assert not diff, f"call {call}: {len(diff)} pairs differ from the oracle"
        for q in range(w.nq):
            r = i[o[q]:o[q + 1]]
            assert np.all(np.diff(r) > 0)
        got = _dist_map(o, i, dv)
        _check_shared_dists(got, _dist_map(ref.offsets, ref.ids, ref.dists), f"call {call} vs vj_join_exact")
        _check_shared_dists(got, _dist_map(o_off, o_ids, o_d), f"call {call} vs the oracle")


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    X = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    off = torch.zeros(8, dtype=torch.int64, device="cuda")
    ids = torch.zeros(8, dtype=torch.int32, device="cuda")
    dd = torch.zeros(8, dtype=torch.float32, device="cuda")
    lib = vj.load()
    import ctypes as C
    nnz = C.c_int64(0)
    st = lib.vj_join_exact_noalloc(X.data_ptr(), 4, X.data_ptr(), vj.NOALLOC_MAX_QUERIES + 1, 8, vj.VJ_L2, 1.0,
                                   off.data_ptr(), ids.data_ptr(), dd.data_ptr(), 8, C.byref(nnz), None)
    assert st == vj.VJ_ERR_ARG
    assert b"scratch limit" in lib.vj_last_error()


def test_noalloc_reports_capacity_overflow(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(5)
    Xh = rng.standard_normal((300, 16)).astype(np.float32)
    X = torch.from_numpy(Xh).cuda()
    off = torch.zeros(301, dtype=torch.int64, device="cuda")
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    dd = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(vj.VjError) as e:
        vj.vj_join_exact_noalloc(X, X, 100.0, off, ids, dd)  # every pair matches
    assert e.value.status == vj.VJ_ERR_STATE
    assert int(off[-1].item()) == 300 * 300
