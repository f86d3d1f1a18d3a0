"""GPU engine vs the FP64 oracle, through the C ABI.

Hit sets must match bit for bit.  In FP64, reconstruction errors must agree
to 1e-9 relative and factor subspaces to 1e-3 rad (expected ~1e-10).  In FP32
(the arithmetic of the whole engine path, eig and QR included), the model
itself must agree: ||Y_gpu - Y_oracle||_F <= 1e-3 ||X||_F, which by the
triangle inequality bounds the difference of the error values by the same
amount; the error values must also agree to 1e-3 relative to max(e, 0.1).
(Measured FP32 drift is ~2e-5 ||X|| per query: about 300 unit roundoffs,
accumulated over the tree levels.)  Parity runs use tol = 0 so that both
sides run the same number of ALS iterations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import series, oracle_tree, engine_tree, compare  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SMALL = dict(T=256, dims=(30, 20), ranks=(5, 5, 5), regime=64, sigma=0.01, B=4, seed=1001)
ITERS = 6


@pytest.fixture(scope="module")
def small_pair():
    c = SMALL
    X = series(c["T"], c["dims"], c["ranks"], c["regime"], c["sigma"], c["seed"])
    o = oracle_tree(X, c["dims"], c["ranks"], c["B"], ITERS, 0.0)
    e = engine_tree(X, c["dims"], c["ranks"], c["B"], ITERS, 0.0, "f64")
    return X, o, e


def test_hit_sets_bit_exact(small_pair):
    X, o, e = small_pair
    T = X.shape[0]
    Q = synth.query_ranges(T, 100, 2001)
    extra = [(a, b) for a in range(0, T, 7) for b in range(a + 1, T + 1, 5)]
    for ts, te in list(map(tuple, Q)) + extra:
        ho = o.hit_records(int(ts), int(te))
        he = [(h[0], h[1], h[2], h[3], h[4], h[5]) for h in e.hit_set(int(ts), int(te))]
        assert he == ho, (ts, te)


def test_query_parity_fp64(small_pair):
    X, o, e = small_pair
    Q = synth.query_ranges(X.shape[0], 100, 2001)
    worst = [0.0, 0.0, 0.0]
    for ts, te in Q:
        ro = o.query(int(ts), int(te))
        Ge, Ue, info = e.query(int(ts), int(te))
        assert info["ranks"] == ro["ranks"]
        assert info["iters"] == ro["iters"] == ITERS
        assert info["n_hits"] == len(ro["hits"])
        rel, dist, ang, ee, eo = compare(X, int(ts), int(te), Ge, Ue, ro["G"], ro["U"])
        worst = [max(worst[0], rel), max(worst[1], dist), max(worst[2], ang)]
        assert rel < 1e-9, (ts, te, ee, eo)
        assert ang < 1e-3, (ts, te, ang)
        for u in Ue:
            assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < 1e-12
    print("fp64 worst rel-err diff %.2e model dist %.2e angle %.2e" % tuple(worst))


def test_node_payload_parity_fp64(small_pair):
    X, o, e = small_pair
    from oracle import metrics
    for v in o.nodes():
        if v.kind not in ("L", "M"):
            continue
        w = v.tau - v.sigma
        level = w.bit_length() - 1
        H, V, r = e.node_payload(level, v.sigma >> level)
        assert list(H.shape) == list(v.H.shape)
        d = metrics.model_distance(H, V, v.H, v.V) / max(np.linalg.norm(v.H), 1e-300)
        assert d < 1e-8, (level, v.sigma, d)


def test_build_equals_appends_bitwise():
    c = dict(SMALL, T=83)
    X = series(c["T"], c["dims"], c["ranks"], c["regime"], c["sigma"], c["seed"])
    a = engine_tree(X, c["dims"], c["ranks"], c["B"], 4, 0.0, "f64")
    b = engine_tree(X, c["dims"], c["ranks"], c["B"], 4, 0.0, "f64", via_appends=True)
    nb = c["T"] // c["B"]
    for level in range(0, 8):
        for k in range(0, (nb >> level) + (1 if level == 0 else 0)):
            if level == 0 and k == nb and c["T"] % c["B"] == 0:
                continue
            Ha, Va, ra = a.node_payload(level, k)
            Hb, Vb, rb = b.node_payload(level, k)
            assert ra == rb
            assert np.array_equal(Ha, Hb) and all(np.array_equal(x, y) for x, y in zip(Va, Vb))
    for ts, te in [(0, 83), (5, 77), (80, 83), (13, 14)]:
        Ga, Ua, _ = a.query(ts, te)
        Gb, Ub, _ = b.query(ts, te)
        assert np.array_equal(Ga, Gb) and all(np.array_equal(x, y) for x, y in zip(Ua, Ub))


@pytest.mark.parametrize("T,B", [(37, 1), (61, 4), (50, 8)])
def test_tail_leaf_and_leaf_sizes(T, B):
    dims, ranks = (9, 7), (3, 3, 3)
    X = series(T, dims, ranks, 16, 0.05, 77)
    o = oracle_tree(X, dims, ranks, B, 3, 0.0)
    e = engine_tree(X, dims, ranks, B, 3, 0.0, "f64", via_appends=True)
    for ts, te in [(0, T), (T - 1, T), (3, T - 2), (T // 2, T), (1, 2)]:
        assert [tuple(h[:6]) for h in e.hit_set(ts, te)] == o.hit_records(ts, te)
        ro = o.query(ts, te)
        Ge, Ue, info = e.query(ts, te)
        assert info["ranks"] == ro["ranks"]
        rel, dist, ang, ee, eo = compare(X, ts, te, Ge, Ue, ro["G"], ro["U"])
        assert rel < 1e-9 and ang < 1e-3, (ts, te, rel, ang)


def test_four_way_and_reduced_query_ranks():
    dims, ranks = (6, 5, 4), (3, 3, 2, 2)
    T, B = 40, 4
    X = series(T, dims, ranks, 20, 0.05, 5)
    o = oracle_tree(X, dims, ranks, B, 3, 0.0)
    e = engine_tree(X, dims, ranks, B, 3, 0.0, "f64")
    for ts, te, rq in [(0, 40, None), (3, 33, None), (7, 19, (2, 2, 1, 2)), (0, 40, (1, 1, 1, 1))]:
        ro = o.query(ts, te, ranks=rq)
        Ge, Ue, info = e.query(ts, te, ranks=rq)
        assert info["ranks"] == ro["ranks"]
        rel, dist, ang, ee, eo = compare(X, ts, te, Ge, Ue, ro["G"], ro["U"])
        assert rel < 1e-9 and ang < 1e-3, (ts, te, rq, rel, ang)


def test_errors_are_reported():
    import paper_2501_06647_gb300 as tk
    t = tk.Tree((5, 4), (2, 2, 2), leaf_slices=2, dtype="f64")
    with pytest.raises(tk.TuckerError) as ei:
        t.query(0, 1)
    assert ei.value.code == -2
    X = series(10, (5, 4), (2, 2, 2), 10, 0.1, 3)
    t.build(torch.from_numpy(X).cuda())
    with pytest.raises(tk.TuckerError) as ei:
        t.build(torch.from_numpy(X).cuda())
    assert ei.value.code == -6
    for ts, te in [(-1, 3), (3, 3), (5, 11)]:
        with pytest.raises(tk.TuckerError) as ei:
            t.query(ts, te)
        assert ei.value.code == -2
    with pytest.raises(tk.TuckerError) as ei:
        t.query(0, 5, ranks=(3, 2, 2))
    assert ei.value.code == -3
    G, U, info = t.query(0, 10)
    assert info["iters"] >= 1


def test_fp32_matches_fp64_oracle():
    dims, ranks = (60, 50), (10, 10, 10)
    T, B = 512, 16
    X = series(T, dims, ranks, 128, 0.05, 1002)
    o = oracle_tree(X, dims, ranks, B, 4, 0.0)
    e = engine_tree(X, dims, ranks, B, 4, 0.0, "f32")
    Q = synth.query_ranges(T, 40, 2002, "loguniform", 16, T)
    worst = 0.0
    for ts, te in Q:
        assert [tuple(h[:6]) for h in e.hit_set(int(ts), int(te))] == o.hit_records(int(ts), int(te))
        ro = o.query(int(ts), int(te))
        Ge, Ue, info = e.query(int(ts), int(te))
        assert info["ranks"] == ro["ranks"]
        rel, dist, ang, ee, eo = compare(X, int(ts), int(te), Ge, Ue, ro["G"], ro["U"])
        worst = max(worst, dist)
        assert dist < 1e-3, (ts, te, dist)
        assert abs(ee - eo) < 1e-3 * max(eo, 0.1), (ts, te, ee, eo)
    print("fp32 worst model distance vs fp64 oracle %.2e (relative to ||X||)" % worst)


def test_batch_equals_single_queries():
    c = SMALL
    X = series(c["T"], c["dims"], c["ranks"], c["regime"], c["sigma"], c["seed"])
    e = engine_tree(X, c["dims"], c["ranks"], c["B"], 4, 0.0, "f64")
    Q = synth.query_ranges(c["T"], 50, 2001)
    out, offs, info = e.query_batch_host(Q)
    for i, (ts, te) in enumerate(Q):
        G, U, inf = e.query(int(ts), int(te))
        Gb, Ub = e.unpack(out[offs[i]:offs[i + 1]], int(te - ts))
        r = inf["ranks"]
        assert np.array_equal(G, Gb[tuple(slice(0, x) for x in r)])
        assert all(np.array_equal(u, ub[:, :x]) for u, ub, x in zip(U, Ub, r))
        assert info[i].iters == inf["iters"]


@pytest.mark.parametrize("dtype,bound", [("f64", 1e-9), ("f32", 2e-5)])
def test_noise_free_low_rank_is_exact(dtype, bound):
    """Noise-free data of Tucker rank (3, 3, 3) in a single regime, stored and
    queried at ranks (6, 6, 6): every stage (leaf ALS, child merges, partial
    hits, query stitch) is exact, so every query reconstructs its range to
    rounding, as the oracle's own exactness pin states.  The Grams then have
    exactly zero eigenvalues beyond rank 3, which the eigensolver has to treat
    as one cluster (orders 20-30 here, so the tridiagonal method runs)."""
    from oracle import metrics
    dims, B, T = (30, 24), 4, 160
    X = series(T, dims, (3, 3, 3), T, 0.0, 1234)
    e = engine_tree(X, dims, (6, 6, 6), B, 5, 0.0, dtype)
    Q = [(0, T), (5, 93), (17, 40), (3, 150), (60, 61), (128, 160)]
    for ts, te in Q:
        G, U, info = e.query(ts, te)
        # materialized residual: the cancellation form of relative_error only
        # resolves errors down to ~sqrt(eps)
        Xs = np.asarray(X[ts:te], dtype=np.float64)
        err = metrics.residual_norm_dense(Xs, np.float64(G), [np.float64(u) for u in U]) / np.linalg.norm(Xs)
        assert err < bound, (ts, te, err, info)
        for u in U:
            u = np.float64(u)
            assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < (1e-10 if dtype == "f64" else 2e-5)


def test_fp32_rank16_wide_slices_matches_fp64_oracle():
    """The batched workload's shapes (200 x 150 slices, ranks 16, leaf 16) on
    a shorter series: leaf Grams of order 200 (eigensolver arrays in global
    memory), query eigenproblems of order up to ~100.  Hit sets bit for bit;
    the FP32 model within 1e-3 ||X|| of the FP64 oracle's, as for the plain
    workload."""
    dims, ranks = (200, 150), (16, 16, 16)
    T, B = 256, 16
    X = series(T, dims, ranks, 128, 0.05, 1003)
    o = oracle_tree(X, dims, ranks, B, 3, 0.0)
    e = engine_tree(X, dims, ranks, B, 3, 0.0, "f32")
    Q = synth.query_ranges(T, 8, 2003, "loguniform", 16, T)
    for ts, te in Q:
        assert [tuple(h[:6]) for h in e.hit_set(int(ts), int(te))] == o.hit_records(int(ts), int(te))
        ro = o.query(int(ts), int(te))
        Ge, Ue, info = e.query(int(ts), int(te))
        assert info["ranks"] == ro["ranks"]
        rel, dist, ang, ee, eo = compare(X, int(ts), int(te), Ge, Ue, ro["G"], ro["U"])
        assert dist < 1e-3, (ts, te, dist)
        assert abs(ee - eo) < 1e-3 * max(eo, 0.1), (ts, te, ee, eo)


def test_five_way_matches_fp64_oracle():
    """A 5-way series (4 non-temporal modes): hit sets bit for bit, FP64
    errors within 1e-9 relative and factor subspaces within 1e-3 rad, as for
    the 3-way parity workload."""
    dims, ranks = (6, 5, 4, 3), (3, 2, 2, 2, 2)
    T, B = 48, 4
    X = series(T, dims, ranks, 24, 0.01, 1005)
    o = oracle_tree(X, dims, ranks, B, 3, 0.0)
    e = engine_tree(X, dims, ranks, B, 3, 0.0, "f64")
    for ts, te in synth.query_ranges(T, 12, 2005):
        assert [tuple(h[:6]) for h in e.hit_set(int(ts), int(te))] == o.hit_records(int(ts), int(te))
        ro = o.query(int(ts), int(te))
        Ge, Ue, info = e.query(int(ts), int(te))
        assert info["ranks"] == ro["ranks"]
        rel, dist, ang, ee, eo = compare(X, int(ts), int(te), Ge, Ue, ro["G"], ro["U"])
        assert rel < 1e-9, (ts, te, rel)
        assert ang < 1e-3, (ts, te, ang)
