"""The seeded input generators shared by the oracle checks and the engine's
tests and benchmark: determinism, shapes, the unit signal scale, the
regime-local low rank, and the query-range recipes."""
import numpy as np

import synth


def test_series_is_deterministic_and_shaped():
    a = synth.piecewise_tucker(64, (12, 10), (3, 3, 3), 32, 0.05, 7)
    b = synth.piecewise_tucker(64, (12, 10), (3, 3, 3), 32, 0.05, 7)
    c = synth.piecewise_tucker(64, (12, 10), (3, 3, 3), 32, 0.05, 8)
    assert a.shape == (64, 12, 10) and a.dtype == np.float64
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_noise_free_regimes_have_the_stated_rank_and_unit_rms():
    T, dims, ranks, regime = 96, (14, 11), (4, 3, 2), 32
    X = synth.piecewise_tucker(T, dims, ranks, regime, 0.0, 11)
    # the core is scaled so that the signal's mean square per entry is 1 in
    # expectation: over 40 regimes (24 core entries each, std of one regime's
    # mean square ~0.29) the average is within 0.15 of 1
    Z = synth.piecewise_tucker(40 * 8, dims, ranks, 8, 0.0, 12)
    ms = [np.mean(Z[s:s + 8] ** 2) for s in range(0, 40 * 8, 8)]
    assert abs(np.mean(ms) - 1.0) < 0.15
    for s0 in range(0, T, regime):
        R = X[s0:s0 + regime]
        for n, r in enumerate(ranks):
            M = np.moveaxis(R, n, 0).reshape(R.shape[n], -1)
            sv = np.linalg.svd(M, compute_uv=False)
            assert sv[r] < 1e-10 * sv[0] and sv[r - 1] > 1e-6 * sv[0]   # multilinear rank exactly r_n


def test_regime_generator_matches_shapes_and_rank():
    T, dims, ranks, regime = 80, (9, 8, 7), (3, 2, 2, 2), 40
    X = synth.piecewise_tucker_regimes(T, dims, ranks, regime, 0.0, 5, threads=2)
    Y = synth.piecewise_tucker_regimes(T, dims, ranks, regime, 0.0, 5, threads=1)
    assert X.shape == (T,) + dims and X.dtype == np.float32
    assert np.array_equal(X, Y)                                       # independent of the thread count
    M = X[:regime].reshape(regime, -1).astype(np.float64)
    sv = np.linalg.svd(M, compute_uv=False)
    assert sv[ranks[0]] < 1e-5 * sv[0]


def test_query_ranges():
    T = 500
    U = synth.query_ranges(T, 200, 3, "uniform")
    assert np.all((0 <= U[:, 0]) & (U[:, 0] < U[:, 1]) & (U[:, 1] <= T))
    L = synth.query_ranges(T, 2000, 4, "loguniform", 16, T)
    lens = L[:, 1] - L[:, 0]
    assert np.all((0 <= L[:, 0]) & (L[:, 1] <= T)) and lens.min() >= 16 and lens.max() <= T
    # log-uniform: about half of the lengths below the geometric mean of the bounds
    assert abs(np.mean(lens < np.sqrt(16 * T)) - 0.5) < 0.05
    assert np.array_equal(L, synth.query_ranges(T, 2000, 4, "loguniform", 16, T))


def test_workloads_declare_what_the_benchmark_reads():
    for name in ("fp64_small", "fp32_plain", "batched_r16", "serving_4way"):
        w = synth.WORKLOADS[name]
        assert len(w["dims"]) == len(w["ranks"]) - 1 and w["B"] >= 1
