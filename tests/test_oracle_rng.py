"""Pins of the oracle's seeded Stitch start (oracle/rng.py: Algorithm 2's
"randomly initialize U^(2..p)", drawn by splitmix64, Box-Muller and QR).

Pinned against what does not come from the oracle itself:
  * splitmix64's published output for seed 0 (the first three values of the
    reference generator's stream);
  * the distributions: uniforms on (0, 1] and Box-Muller Gaussians against
    their CDFs (Kolmogorov-Smirnov), mean and variance, and the pairing of
    cos and sin (independent normals: no correlation within a pair);
  * the counter property (an element depends only on the seed and its
    index) and the element offsets of the modes;
  * orthonormal factors spanning the Gaussian matrices' column spaces;
  * Algorithm 2 from the random start on noise-free low-rank data stored at
    full rank returns the data exactly, like the HOSVD start.
A mutation of the generator (a constant of splitmix64, the element offsets,
cos and sin swapped, a dropped orthonormalization) breaks one of these.
"""
import numpy as np
import pytest

from oracle import rng, stitch as st, tensor
from oracle.tree import StreamSegmentTree
import synth


def test_splitmix64_reference_values():
    assert [rng.splitmix64(0, k) for k in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                         0x06C45D188009454F]


def test_uniforms_and_gaussians_have_their_distributions():
    scipy_stats = pytest.importorskip("scipy.stats")
    u = np.array([rng.uniform(7, k) for k in range(20000)])
    assert u.min() > 0.0 and u.max() <= 1.0
    assert scipy_stats.kstest(u, "uniform").pvalue > 1e-3
    g = np.array([rng.gaussian(7, e) for e in range(20000)])
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1.0) < 0.04
    assert scipy_stats.kstest(g, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair are independent normals
    assert abs(np.corrcoef(g[0::2], g[1::2])[0, 1]) < 0.03
    # even members use cos, odd ones sin: their squares of a pair sum to -2 ln u1
    for j in range(5):
        u1 = rng.uniform(7, 2 * j)
        assert abs(g[2 * j] ** 2 + g[2 * j + 1] ** 2 + 2 * np.log(u1)) < 1e-12
        assert g[2 * j] * np.sin(2 * np.pi * rng.uniform(7, 2 * j + 1)) == pytest.approx(
            g[2 * j + 1] * np.cos(2 * np.pi * rng.uniform(7, 2 * j + 1)), abs=1e-12)


def test_elements_depend_only_on_seed_and_index():
    full = rng.gaussian_matrix(11, 0, 6, 5)
    assert np.array_equal(rng.gaussian_matrix(11, 10, 2, 5), full[2:4])  # rows 2..3 are elements 10..19
    assert not np.array_equal(rng.gaussian_matrix(12, 0, 6, 5), full)


def test_seeded_factors_are_orthonormal_bases_of_the_gaussian_matrices():
    dims, ranks = (9, 7, 5), (3, 4, 2, 3)
    U = rng.seeded_factors(dims, ranks, 5)
    assert U[0] is None
    off = 0
    for n in range(1, 4):
        D, r = dims[n - 1], ranks[n]
        assert U[n].shape == (D, r)
        assert np.allclose(U[n].T @ U[n], np.eye(r), atol=1e-13)
        G = rng.gaussian_matrix(5, off, D, r)
        off += D * r
        # same column space: the projection of G onto U's span is G
        assert np.allclose(U[n] @ (U[n].T @ G), G, atol=1e-12)


def test_random_start_recovers_noise_free_low_rank_data():
    dims, ranks, B, T = (8, 7), (3, 3, 3), 4, 32
    X = synth.piecewise_tucker(T, dims, ranks, T, 0.0, 77)   # one regime, exact rank (3, 3, 3)
    for init in ("hosvd", "random"):
        o = StreamSegmentTree(dims, ranks, B=B, max_iter=30, tol=0.0, init=init, seed=9)
        o.build(X)
        for ts, te in [(0, 32), (3, 29), (5, 9)]:
            r = o.query(ts, te)
            Y = r["G"]
            for n, u in enumerate(r["U"]):
                Y = tensor.mode_product(Y, u, n)
            assert np.linalg.norm(Y - X[ts:te]) <= 1e-8 * np.linalg.norm(X[ts:te]), (init, ts, te)


def test_random_and_hosvd_starts_differ_only_in_the_start():
    dims, ranks, T = (8, 7), (3, 3, 3), 64
    X = synth.piecewise_tucker(T, dims, ranks, 16, 0.05, 78)
    o1 = StreamSegmentTree(dims, ranks, B=4, max_iter=1, tol=0.0, init="random", seed=3)
    o2 = StreamSegmentTree(dims, ranks, B=4, max_iter=1, tol=0.0, init="hosvd")
    o1.build(X)
    o2.build(X)
    # one iteration from different starts: different models, both within the data's reach
    a, b = o1.query(5, 60), o2.query(5, 60)
    assert not np.allclose(np.abs(a["U"][1]), np.abs(b["U"][1]), atol=1e-6)
    with pytest.raises(ValueError):
        st.stitch([(np.ones((1, 1, 1)), [np.ones((1, 1)), np.ones((8, 1)), np.ones((7, 1))])], [1, 1, 1],
                  init="bogus")


def _mode_product(X, M, n):
    return np.moveaxis(np.tensordot(M, X, axes=(1, n)), 0, n)


def _dense_hooi_from(Y, r, U0, iters):
    """Textbook HOOI (Gauss-Seidel over the modes) on the dense tensor Y from
    the start U0 (U0[0] unused: the temporal factor is updated first),
    written with NumPy's SVD, independently of the oracle's stitch code."""
    p = Y.ndim
    U = list(U0)
    for _ in range(iters):
        for n in range(p):
            Z = Y
            for m in range(p):
                if m != n:
                    Z = _mode_product(Z, U[m].T, m)
            Zn = np.moveaxis(Z, n, 0).reshape(Z.shape[n], -1)
            u, _, _ = np.linalg.svd(Zn, full_matrices=False)
            U[n] = u[:, : r[n]]
    G = Y
    for m in range(p):
        G = _mode_product(G, U[m].T, m)
    return G, U


@pytest.mark.parametrize("iters", [1, 3])
def test_random_start_stitch_equals_dense_hooi_from_the_same_start(iters):
    # Algorithm 2 from the seeded start is HOOI on the stitched tensor Y~ from
    # the same U^(2..p): the literal matricizations of the oracle's Stitch
    # against a dense HOOI loop on the materialized Y~
    rs = np.random.default_rng(5)
    dims, q = (9, 8), (3, 3, 3)
    hits = []
    for ell in (6, 4, 5):
        H = rs.standard_normal(q)
        V = [np.linalg.qr(rs.standard_normal((ell, q[0])))[0]] + \
            [np.linalg.qr(rs.standard_normal((d, k)))[0] for d, k in zip(dims, q[1:])]
        hits.append((H, V))
    Y = st.materialize_stitched(hits)
    r = st.stitched_ranks(hits, dims, (4, 3, 3))
    G, U, it, _ = st.stitch(hits, r, max_iter=iters, tol=0, init="random", seed=21)
    Gd, Ud = _dense_hooi_from(Y, r, rng.seeded_factors(dims, r, 21), iters)
    Ya, Yb = G, Gd
    for m in range(3):
        Ya, Yb = _mode_product(Ya, U[m], m), _mode_product(Yb, Ud[m], m)
    assert it == iters
    assert np.linalg.norm(Ya - Yb) < 1e-10 * np.linalg.norm(Y)
    # and differs from the HOSVD start after one iteration
    if iters == 1:
        Gh, Uh, _, _ = st.stitch(hits, r, max_iter=1, tol=0)
        Yh = Gh
        for m in range(3):
            Yh = _mode_product(Yh, Uh[m], m)
        assert np.linalg.norm(Ya - Yh) > 1e-6 * np.linalg.norm(Y)
