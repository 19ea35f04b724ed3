"""The seeded workload recipes: deterministic, with the stated shapes and value ranges."""
import numpy as np

from paper_2603_16360_b300 import inputs


def test_sift_like_recipe():
    a = inputs.sift_like(scale=0.002)
    b = inputs.sift_like(scale=0.002)
    assert a.X.shape == (2000, 128) and a.Q.shape == (200, 128)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Q, b.Q)
    assert a.X.dtype == np.float32 and a.X.min() >= 0 and a.X.max() <= 255
    assert np.array_equal(a.X, np.rint(a.X))  # integer descriptors stored as FP32
    assert abs(a.ood.mean() - 0.10) < 0.01


def test_angular_instance_recipe():
    w = inputs.angular_instance(7, 3, nx_range=(2000, 5000), nq_range=(300, 800))
    v = inputs.angular_instance(7, 3, nx_range=(2000, 5000), nq_range=(300, 800))
    assert np.array_equal(w.X, v.X) and np.array_equal(w.Q, v.Q) and w.target_matches == v.target_matches
    assert 2000 <= w.nx <= 5000 and 300 <= w.nq <= min(800, w.nx)
    assert w.d == 100 and w.metric == 1 and w.degree == 32 and w.knn_k == 64
    np.testing.assert_allclose(np.linalg.norm(w.X, axis=1), 1.0, atol=1e-5)
    np.testing.assert_allclose(np.linalg.norm(w.Q, axis=1), 1.0, atol=1e-5)
    assert 5 <= w.target_matches <= 50
    assert abs(w.ood.mean() - 0.10) < 0.02
    # another instance index draws another instance
    u = inputs.angular_instance(7, 4, nx_range=(2000, 5000), nq_range=(300, 800))
    assert u.nx != w.nx or not np.array_equal(u.X[:10], w.X[:10])


def test_angular_collection_sizes_log_uniform():
    ws = list(inputs.angular_collection(seed=5, n=64, nx_range=(50, 5000), nq_range=(10, 1000)))
    nx = np.array([w.nx for w in ws])
    nq = np.array([w.nq for w in ws])
    assert nx.min() >= 50 and nx.max() <= 5000 and nq.min() >= 10 and np.all(nq <= np.minimum(nx, 1000))
    # log-uniform: about half of the instances below the geometric midpoint
    assert 20 <= int((nx < np.sqrt(50 * 5000)).sum()) <= 44
    assert len({w.target_matches for w in ws}) > 10
