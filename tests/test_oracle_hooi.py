"""Pins for oracle.hooi (Tucker-ALS, Section 2)."""
import numpy as np

from oracle import hooi, tensor, metrics


def test_clamp_ranks():
    assert hooi.clamp_ranks((4, 30, 20), (5, 5, 5)) == [4, 5, 5]
    assert hooi.clamp_ranks((1, 30, 20), (5, 5, 5)) == [1, 5, 5]
    assert hooi.clamp_ranks((1, 30, 20), (5, 8, 5)) == [1, 5, 5]   # r2 <= r1 * r3
    assert hooi.clamp_ranks((2, 3), (5, 5)) == [2, 2]


def test_matrix_case_is_truncated_svd():
    # p = 2: Tucker of a matrix is the truncated SVD (Eckart-Young)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((40, 25))
    G, U, it, _ = hooi.tucker_als(X, (6, 6), max_iter=30, tol=0)
    s = np.linalg.svd(X, compute_uv=False)
    best = np.sqrt(np.sum(s[6:] ** 2))
    assert abs(metrics.residual_norm(X, G, U) - best) < 1e-9 * np.linalg.norm(X)


def test_full_rank_is_exact():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 5, 4))
    G, U, _, _ = hooi.tucker_als(X, (6, 5, 4), max_iter=3, tol=0)
    assert metrics.residual_norm_dense(X, G, U) < 1e-12 * tensor.frob(X)


def test_exact_low_rank_recovered():
    rng = np.random.default_rng(2)
    core = rng.standard_normal((3, 4, 2))
    F = [np.linalg.qr(rng.standard_normal((d, r)))[0] for d, r in zip((12, 15, 9), (3, 4, 2))]
    X = tensor.multi_mode_product(core, F)
    G, U, _, _ = hooi.tucker_als(X, (3, 4, 2), max_iter=5, tol=0)
    assert metrics.residual_norm_dense(X, G, U) < 1e-12 * tensor.frob(X)
    for u, f in zip(U, F):
        assert metrics.principal_angle_max(f, u) < 1e-10


def test_orthonormal_factors_and_monotone_error():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((10, 9, 8))
    errs = []
    for k in range(1, 6):
        G, U, it, e = hooi.tucker_als(X, (3, 3, 3), max_iter=k, tol=0)
        assert it == k
        for u in U:
            assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < 1e-12
        errs.append(metrics.residual_norm(X, G, U))
        # the stopping quantity is the true residual of the orthogonal model
        assert abs(e[-1] - errs[-1] / tensor.frob(X)) < 1e-10
    assert all(b <= a + 1e-12 for a, b in zip(errs, errs[1:]))


def test_tolerance_stops_early():
    rng = np.random.default_rng(4)
    core = rng.standard_normal((2, 2, 2))
    F = [np.linalg.qr(rng.standard_normal((d, 2)))[0] for d in (8, 7, 6)]
    X = tensor.multi_mode_product(core, F) + 1e-3 * rng.standard_normal((8, 7, 6))
    _, _, it, errs = hooi.tucker_als(X, (2, 2, 2), max_iter=20, tol=0.01)
    assert it == 2 and len(errs) == 2


def test_model_distance_matches_dense_and_resolves_small_gaps():
    rng = np.random.default_rng(9)
    G = rng.standard_normal((3, 2, 2))
    U = [np.linalg.qr(rng.standard_normal((d, r)))[0] for d, r in zip((7, 6, 5), (3, 2, 2))]
    for delta in (1e-1, 1e-6, 1e-11):
        G2 = G + delta * rng.standard_normal(G.shape)
        U2 = [np.linalg.qr(u + delta * rng.standard_normal(u.shape))[0] for u in U]
        dense = tensor.frob(tensor.reconstruct(G, U) - tensor.reconstruct(G2, U2))
        assert abs(metrics.model_distance(G, U, G2, U2) - dense) < 1e-9 * dense + 1e-14
    assert metrics.model_distance(G, U, G, U) < 1e-14


def test_principal_angle_resolves_small_angles():
    for ang in (1e-3, 1e-7, 1e-10):
        A = np.array([[1.0], [0.0]])
        B = np.array([[np.cos(ang)], [np.sin(ang)]])
        assert abs(metrics.principal_angle_max(A, B) - ang) < 1e-3 * ang


def test_residual_formula_matches_dense():
    rng = np.random.default_rng(10)
    X = rng.standard_normal((6, 5, 4))
    G, U, _, _ = hooi.tucker_als(X, (2, 3, 2), max_iter=2, tol=0)
    assert abs(metrics.residual_norm(X, G, U) - metrics.residual_norm_dense(X, G, U)) < 1e-10
