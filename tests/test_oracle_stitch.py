"""Pins for oracle.stitch (Eq. (partial-tucker), Algorithm 2) and the range query:
algebraic identities against the materialized stitched tensor, closed forms,
and the error bound of Proposition (err)."""
import numpy as np
import pytest

import synth
from oracle import tensor, hooi, stitch, metrics
from oracle.tree import StreamSegmentTree


def _rand_orth(rng, m, r):
    return np.linalg.qr(rng.standard_normal((m, r)))[0]


def _rand_hits(seed, lens, dims, q):
    rng = np.random.default_rng(seed)
    hits = []
    for l in lens:
        qq = [min(q[0], l)] + list(q[1:])
        H = rng.standard_normal(tuple(qq))
        V = [_rand_orth(rng, l, qq[0])] + [_rand_orth(rng, d, r) for d, r in zip(dims, qq[1:])]
        hits.append((H, V))
    return hits


def test_matricizations_equal_definition_on_materialized_tensor():
    # Eq. (stitch-temp-2) and Eq. (stitch-nontemp-3) equal Eq. (als-mat) applied to Y~ = [Y~_1; ...].
    rng = np.random.default_rng(0)
    dims, q, r = (7, 6), (3, 3, 2), (4, 3, 2)
    hits = _rand_hits(1, [5, 2, 4], dims, q)
    Y = stitch.materialize_stitched(hits)
    U = [_rand_orth(rng, Y.shape[0], r[0]), _rand_orth(rng, dims[0], r[1]), _rand_orth(rng, dims[1], r[2])]
    Z1 = stitch.temporal_matricization(hits, U)
    ref1 = tensor.unfold(tensor.multi_mode_product(Y, [None, U[1].T, U[2].T]), 0)
    assert np.allclose(Z1, ref1, atol=1e-12)
    offs = np.cumsum([0] + [V[0].shape[0] for _, V in hits])
    for n in (1, 2):
        mats = [u.T for u in U]
        mats[n] = None
        ref = tensor.unfold(tensor.multi_mode_product(Y, mats), n)
        assert np.allclose(stitch.nontemporal_matricization(hits, U, n, offs), ref, atol=1e-12)


def test_init_is_hosvd_of_stitched_tensor():
    hits = _rand_hits(2, [6, 3, 5], (8, 7), (3, 3, 3))
    Y = stitch.materialize_stitched(hits)
    U = stitch.init_factors(hits, [3, 3, 3])
    for n in (1, 2):
        ref = tensor.leading_left_singular_vectors(tensor.unfold(Y, n), 3)
        assert metrics.principal_angle_max(ref, U[n]) < 1e-9


@pytest.mark.parametrize("iters", [1, 3])
def test_stitch_equals_dense_hooi_on_stitched_tensor(iters):
    # Algorithm 2 is Tucker-ALS on the concatenation Y~, rewritten (Section 5.2).
    hits = _rand_hits(3, [6, 4, 5, 3], (9, 8), (3, 3, 3))
    Y = stitch.materialize_stitched(hits)
    r = stitch.stitched_ranks(hits, (9, 8), (4, 3, 3))
    G, U, it, errs = stitch.stitch(hits, r, max_iter=iters, tol=0)
    Gd, Ud, itd, errsd = hooi.tucker_als(Y, r, max_iter=iters, tol=0)
    assert it == itd == iters
    assert metrics.model_distance(G, U, Gd, Ud) < 1e-10 * tensor.frob(Y)
    assert abs(errs[-1] - errsd[-1]) < 1e-12
    # the stopping quantity is the true relative residual against Y~
    assert abs(errs[-1] - metrics.residual_norm_dense(Y, G, U) / tensor.frob(Y)) < 1e-10
    for u in U:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < 1e-12


@pytest.mark.parametrize("p", [4, 5, 6, 7])
def test_more_modes_match_the_materialized_tensor(p):
    # The paper's mode-count experiment reaches p = 7 (Section 8, synthetic
    # tensors); with p >= 4 a wrong Kronecker order of the non-temporal modes
    # in Eq. (stitch-temp-2) / Eq. (stitch-nontemp-3) changes the result.
    rng = np.random.default_rng(40 + p)
    dims = tuple(int(d) for d in rng.integers(3, 6, size=p - 1))
    q = (3,) + (2,) * (p - 1)
    hits = _rand_hits(50 + p, [4, 3, 5], dims, q)
    Y = stitch.materialize_stitched(hits)
    U = [_rand_orth(rng, Y.shape[0], 3)] + [_rand_orth(rng, d, 2) for d in dims]
    ref1 = tensor.unfold(tensor.multi_mode_product(Y, [None] + [u.T for u in U[1:]]), 0)
    assert np.allclose(stitch.temporal_matricization(hits, U), ref1, atol=1e-12)
    offs = np.cumsum([0] + [V[0].shape[0] for _, V in hits])
    for n in range(1, p):
        mats = [u.T for u in U]
        mats[n] = None
        ref = tensor.unfold(tensor.multi_mode_product(Y, mats), n)
        assert np.allclose(stitch.nontemporal_matricization(hits, U, n, offs), ref, atol=1e-12)
    r = stitch.stitched_ranks(hits, dims, (3,) + (2,) * (p - 1))
    G, Us, it, errs = stitch.stitch(hits, r, max_iter=2, tol=0)
    Gd, Ud, itd, errsd = hooi.tucker_als(Y, r, max_iter=2, tol=0)
    assert it == itd == 2
    assert metrics.model_distance(G, Us, Gd, Ud) < 1e-10 * tensor.frob(Y)
    assert abs(errs[-1] - errsd[-1]) < 1e-12


def test_full_rank_stitch_is_exact():
    hits = _rand_hits(4, [3, 2, 4], (4, 3), (2, 2, 2))
    Y = stitch.materialize_stitched(hits)
    r = stitch.stitched_ranks(hits, (4, 3), (9, 4, 3))
    G, U, _, _ = stitch.stitch(hits, r, max_iter=2, tol=0)
    assert metrics.residual_norm_dense(Y, G, U) < 1e-12 * tensor.frob(Y)


def test_partial_hit_qr():
    rng = np.random.default_rng(5)
    H = rng.standard_normal((4, 3, 3))
    V = [_rand_orth(rng, 16, 4), _rand_orth(rng, 7, 3), _rand_orth(rng, 6, 3)]
    H2, V2 = stitch.partial_hit(H, V, 3, 14)
    Q = V2[0]
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-14
    # the restricted tensor equals rows 3..13 of the node tensor exactly (Eq. (partial-tucker) is an identity)
    full = tensor.reconstruct(H, V)
    assert np.allclose(tensor.reconstruct(H2, V2), full[3:14], atol=1e-12)
    # short slice (fewer rows than the rank): still exact
    H3, V3 = stitch.partial_hit(H, V, 5, 7)
    assert V3[0].shape == (2, 2)
    assert np.allclose(tensor.reconstruct(H3, V3), full[5:7], atol=1e-12)


def _single_regime_tree(T, dims, ranks, B, sigma, theta=(7, 10)):
    X = synth.piecewise_tucker(T, dims, ranks, regime=T, sigma=sigma, seed=7)
    t = StreamSegmentTree(dims, ranks, B=B, theta=theta, max_iter=20, tol=0)
    t.build(X)
    return X, t


def test_noise_free_low_rank_queries_are_exact():
    X, t = _single_regime_tree(48, (9, 7), (3, 3, 3), B=4, sigma=0.0)
    for ts, te in [(0, 48), (3, 29), (5, 6), (17, 40), (44, 48)]:
        r = t.query(ts, te, max_iter=4, tol=0)
        res = metrics.residual_norm_dense(X[ts:te], r["G"], r["U"])
        assert res < 1e-10 * tensor.frob(X[ts:te])


def test_query_on_a_node_reproduces_the_node():
    X, t = _single_regime_tree(32, (6, 5), (3, 3, 3), B=4, sigma=0.05)
    v = t.root.left                      # node [0, 16)
    r = t.query(0, 16, max_iter=20, tol=0)
    assert len(r["hits"]) == 1
    for n in range(3):
        assert metrics.principal_angle_max(v.V[n], r["U"][n]) < 1e-8
    assert metrics.model_distance(v.H, v.V, r["G"], r["U"]) < 1e-8 * tensor.frob(v.H)


def test_error_bound_proposition():
    # Proposition (err): with W of Tucker rank <= r and ||E|| <= eps ||X||, rel. error <= 3 eps
    # (theta = 1 so that every hit is an exact stored node).
    T, dims, ranks, sigma = 64, (10, 8), (3, 3, 3), 0.05
    X, t = _single_regime_tree(T, dims, ranks, B=2, sigma=sigma, theta=(1, 1))
    W = synth.piecewise_tucker(T, dims, ranks, regime=T, sigma=0.0, seed=7)
    for ts, te in [(0, 64), (3, 50), (10, 61), (20, 33)]:
        eps = tensor.frob(X[ts:te] - W[ts:te]) / tensor.frob(X[ts:te])
        r = t.query(ts, te, max_iter=20, tol=0)
        assert metrics.relative_error(X[ts:te], r["G"], r["U"]) <= 3 * eps


def test_tree_build_equals_successive_appends_of_payloads():
    X = synth.piecewise_tucker(24, (5, 4), (2, 2, 2), regime=8, sigma=0.1, seed=8)
    t = StreamSegmentTree((5, 4), (2, 2, 2), B=3, max_iter=3, tol=0)
    t.build(X)
    # the payload of each complete node depends only on its children: recompute the root's
    # left child [0, 4) blocks directly by stitching its children's payloads
    v = t.root.left
    hits = [(v.left.H, v.left.V), (v.right.H, v.right.V)]
    G, U, _, _ = stitch.stitch(hits, stitch.stitched_ranks(hits, (5, 4), (2, 2, 2)), 3, 0)
    assert metrics.model_distance(G, U, v.H, v.V) < 1e-12


# ---- planted mistakes: each pin above must catch a plausible slip in the oracle -------------

def test_pins_catch_a_transposed_projection(monkeypatch):
    # Plant a slip in Eq. (stitch-temp-2): V_i^(m)T U^(m) instead of U^(m)T V_i^(m)
    # (shape-compatible because every rank is 3); the dense-HOOI identity must fail.
    hits = _rand_hits(3, [6, 4, 5, 3], (9, 8), (3, 3, 3))
    Y = stitch.materialize_stitched(hits)
    r = stitch.stitched_ranks(hits, (9, 8), (3, 3, 3))

    def wrong(hits_, U):
        blocks = []
        for H, V in hits_:
            Z = tensor.mode_product(H, V[0], 0)
            for m in range(1, len(U)):
                Z = tensor.mode_product(Z, V[m].T @ U[m], m)
            blocks.append(tensor.unfold(Z, 0))
        return np.vstack(blocks)
    monkeypatch.setattr(stitch, "temporal_matricization", wrong)
    G, U, _, _ = stitch.stitch(hits, r, max_iter=2, tol=0)
    Gd, Ud, _, _ = hooi.tucker_als(Y, r, max_iter=2, tol=0)
    assert metrics.model_distance(G, U, Gd, Ud) > 1e-6 * tensor.frob(Y)


def test_pins_catch_a_dropped_R_factor(monkeypatch):
    rng = np.random.default_rng(5)
    H = rng.standard_normal((4, 3, 3))
    V = [_rand_orth(rng, 16, 4), _rand_orth(rng, 7, 3), _rand_orth(rng, 6, 3)]
    S = V[0][3:14]
    Q, _ = np.linalg.qr(S)
    bad = tensor.reconstruct(H, [Q] + V[1:])               # core not multiplied by R
    assert not np.allclose(bad, tensor.reconstruct(H, V)[3:14], atol=1e-6)
