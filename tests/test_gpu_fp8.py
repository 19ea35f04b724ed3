"""FP8 (E4M3) brute-force scan tiles against the FP64 nested-loop join.

The scan's tiles hold E4M3 copies of the rows (a power-of-two scale per data
row, one shared by the scanned query rows) and accumulate the exact products
in FP32 on the tensor cores.  A pair is a candidate when its tile value is
within the measured rounding bound of eps (each row's own rounding error,
Cauchy-Schwarz, plus the accumulation), and every candidate is re-decided from
the FP32 vectors, so the join is exact: pair ids equal the FP64 nested-loop
join (Sec. 3.2) outside the |dist - eps| <= 1e-4 eps band, distances within
1e-5 relative.  The same holds for the BF16 tiles of inputs that are not BF16
values, which take the same measured bound.
"""
import numpy as np
import pytest

from paper_2603_16360_b300 import inputs
from paper_2603_16360_b300 import vj

pytestmark = pytest.mark.gpu

BAND = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16360_b300 import build as b
    b.build()
    vj.load()


def _cdist(w):
    from scipy.spatial.distance import cdist
    return cdist(w.Q.astype(np.float64), w.X.astype(np.float64), "euclidean" if w.metric == 0 else "cosine")


def _eps(D, matches):
    k = int(matches * D.shape[0])
    return float(np.float32(np.partition(D.ravel(), k)[k]))


def _pairs(off, ids):
    return {(q, int(i)) for q in range(len(off) - 1) for i in ids[off[q]:off[q + 1]]}


def _check_exact(w, r, eps, oracle, D):
    off, ids, dd = oracle.nlj(w.X, w.Q, eps, w.metric)
    qs, xs = np.nonzero(np.abs(D - eps) <= BAND * eps)
    band = set(zip(qs.tolist(), xs.tolist()))
    got, exp = _pairs(r.offsets, r.ids), _pairs(off, ids)
    diff = (got ^ exp) - band
    assert not diff, f"{len(diff)} pairs differ, e.g. {sorted(diff)[:5]}"
    # distances on the pairs both hold
    ref = {(q, int(ids[j])): float(dd[j]) for q in range(w.nq) for j in range(off[q], off[q + 1])}
    n = 0
    for q in range(w.nq):
        for j in range(r.offsets[q], r.offsets[q + 1]):
            key = (q, int(r.ids[j]))
            if key in ref:
                assert abs(float(r.dists[j]) - ref[key]) <= 1e-5 * abs(ref[key]) + 1e-6, key
                n += 1
    assert n > 0
    return len(exp)


CASES = {
    # d = 960 Gaussian mixture (sigma 0.3), L2: the precision workload's recipe
    "gauss_wide_d960": lambda: inputs.gauss_wide(seed=207, scale=0.0015),
    # 768-wide unit BF16 vMF rows, cosine
    "vmf_cos_d768": lambda: inputs.vmf_like(seed=208, scale=0.0002),
    # integers 0..255, d = 128 (one K block, no tail)
    "sift_like_d128": lambda: inputs.sift_like(seed=209, scale=0.002),
    # ragged widths: 300 columns (K tail of two steps), 37 columns (rows padded to one box)
    "uniform_l2_d300": lambda: inputs.uniform_small(210, 1500, 170, 300, degree=12, knn_k=24),
    "uniform_cos_d300": lambda: inputs.uniform_small(211, 1500, 170, 300, metric=1, degree=12, knn_k=24),
    "ragged_d37": lambda: inputs.uniform_small(212, 1300, 150, 37, degree=12, knn_k=24),
}


@pytest.fixture(scope="module", params=list(CASES))
def built(request):
    w = CASES[request.param]()
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    yield request.param, w, ix, _cdist(w)
    ix.free()


def test_fp8_exact_join_matches_nlj(built, oracle):
    name, w, ix, D = built
    eps = _eps(D, 10)
    vj.vj_set_join_params(ix, scan=vj.VJ_PREC_FP8)
    try:
        r8 = vj.vj_join_exact(ix, eps)
    finally:
        vj.vj_set_join_params(ix, scan=vj.VJ_PREC_BF16)
    npairs = _check_exact(w, r8, eps, oracle, D)
    assert npairs > 0
    # every result pair was a candidate of the FP8 tiles
    assert r8.stats["scan_candidates"] >= len(r8.ids)


def test_fp8_and_bf16_scans_give_the_same_join(built, oracle):
    """Both precisions re-decide every candidate from the FP32 vectors, so the
    rows are identical; each precision's candidates cover the result."""
    name, w, ix, D = built
    eps = _eps(D, 10)
    rb = vj.vj_join_exact(ix, eps)
    vj.vj_set_join_params(ix, scan=vj.VJ_PREC_FP8)
    try:
        r8 = vj.vj_join_exact(ix, eps)
    finally:
        vj.vj_set_join_params(ix, scan=vj.VJ_PREC_BF16)
    np.testing.assert_array_equal(r8.offsets, rb.offsets)
    np.testing.assert_array_equal(r8.ids, rb.ids)
    np.testing.assert_array_equal(r8.dists, rb.dists)
    assert r8.stats["scan_candidates"] >= len(r8.ids)
    assert rb.stats["scan_candidates"] >= len(rb.ids)
    _check_exact(w, rb, eps, oracle, D)


def test_fp8_routed_rows_are_exact(oracle):
    """Queries routed to the brute-force scan take FP8 tiles when scan = FP8;
    their rows equal the nested-loop join."""
    w = inputs.gauss_wide(seed=213, scale=0.0012)
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    D = _cdist(w)
    eps = _eps(D, 10)
    rng = np.random.default_rng(3)
    route = (rng.random(w.nq) < 0.3).astype(np.uint8)
    vj.vj_set_join_params(ix, scan=vj.VJ_PREC_FP8)
    vj.vj_set_plan(ix, route, None)
    try:
        r = vj.vj_join(ix, eps)
    finally:
        vj.vj_set_plan(ix, None, None)
        ix.free()
    rq = np.nonzero(route)[0]
    off, ids, _ = oracle.nlj(w.X, w.Q[rq], eps, w.metric)
    qs, xs = np.nonzero(np.abs(D[rq] - eps) <= BAND * eps)
    band = {(int(rq[a]), int(b)) for a, b in zip(qs, xs)}
    got = {(int(q), int(x)) for q in rq for x in r.row(int(q))}
    exp = {(int(rq[i]), int(x)) for i in range(len(rq)) for x in ids[off[i]:off[i + 1]]}
    assert exp and not ((got ^ exp) - band)


def test_fp8_rounding_midpoints_and_edge_sizes(oracle):
    """Coordinates at the midpoints between neighbouring E4M3 values (the
    largest rounding error per coordinate), a data count that is not a
    multiple of the 256-row tile, a single query, and a zero data row."""
    rng = np.random.default_rng(5)
    d, nx = 200, 777
    # in [1, 2) E4M3 steps by 1/8: midpoints 1 + (2k + 1) / 16
    base = 1.0 + (2 * rng.integers(0, 8, size=(nx + 1, d)) + 1) / 16.0
    sign = np.where(rng.random((nx + 1, d)) < 0.5, -1.0, 1.0)
    A = (base * sign).astype(np.float32)
    X, Q = A[:nx].copy(), A[nx:].copy()
    X[5] = 0.0
    ix = vj.vj_build(X, Q, params=vj.default_params(degree=8, knn_k=16))
    w = type("W", (), {"X": X, "Q": Q, "nq": 1, "metric": 0})()
    D = _cdist(w)
    eps = float(np.float32(np.sort(D.ravel())[40]))
    vj.vj_set_join_params(ix, scan=vj.VJ_PREC_FP8)
    try:
        r = vj.vj_join_exact(ix, eps)
        r2 = vj.vj_join_exact(ix, eps)  # a second call reuses the data-side rows
    finally:
        ix.free()
    assert _check_exact(w, r, eps, oracle, D) > 0
    np.testing.assert_array_equal(r.ids, r2.ids)


def test_scan_precision_is_validated():
    X = np.random.default_rng(1).standard_normal((300, 16)).astype(np.float32)
    ix = vj.vj_build(X, X[:10].copy(), params=vj.default_params(degree=8, knn_k=16))
    try:
        with pytest.raises(vj.VjError) as e:
            vj.vj_set_join_params(ix, scan=7)
        assert e.value.status == vj.VJ_ERR_ARG
        with pytest.raises(vj.VjError) as e:
            vj.vj_build(X, X[:10].copy(), params=vj.default_params(degree=8, knn_k=16, precision=vj.VJ_PREC_FP8))
        assert e.value.status == vj.VJ_ERR_ARG
    finally:
        ix.free()
