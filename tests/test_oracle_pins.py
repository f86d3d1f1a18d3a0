"""Pins for the output-rank clamp of a stitch (oracle.stitch.stitched_ranks)
and the paper's accuracy metric (oracle.metrics.paper_relative_error, Section
8.1), each checked against something other than the oracle itself:

  * the clamp against the numerical multilinear rank of the materialized
    stitched tensor Y~ = [Y~_1; ...; Y~_s] (singular values of mat_n(Y~) above
    1e-10 sigma_1), on generic hits where each cap binds in turn: the time
    extent L, a dimension D_n, and the per-hit mode-rank sum
    sum_i min(q_in, prod_{m != n} q_im); plus hand-worked tuples;
  * the metric against closed forms: 0 when Y_A = Y_ALS, and for p = 2 the
    Eckart-Young value sqrt(sum_{k>=r} s_k^2) / sqrt(sum_{k>r} s_k^2) - 1 when
    Y_A and Y_ALS are the rank-(r-1) and rank-r truncated SVDs.

Each pin group ends with a planted mistake (a one-expression mutation of the
oracle's own source) that the pins must catch."""
import numpy as np
import pytest

from _mutate import mutant
from oracle import metrics, stitch, tensor


def _orth(rng, m, r):
    return np.linalg.qr(rng.standard_normal((m, r)))[0]


def _hits(seed, shapes, lens, dims):
    """Generic hits: random cores of the given shapes, random orthonormal factors."""
    rng = np.random.default_rng(seed)
    out = []
    for q, l in zip(shapes, lens):
        H = rng.standard_normal(q)
        V = [_orth(rng, l, q[0])] + [_orth(rng, d, r) for d, r in zip(dims, q[1:])]
        out.append((H, V))
    return out


def _multilinear_rank(hits):
    Y = stitch.materialize_stitched(hits)
    r = []
    for n in range(Y.ndim):
        s = np.linalg.svd(tensor.unfold(Y, n), compute_uv=False)
        r.append(int(np.sum(s > 1e-10 * s[0])))
    return r


# (shapes, temporal lengths, D_2..D_p, expected clamp for a large request, cap that binds)
CASES = [
    # two short hits: L = 3 binds mode 1 (time); D_3 = 5 binds mode 3
    ([(2, 3, 3), (1, 3, 3)], [2, 1], (6, 5), [3, 6, 5]),
    # partial-hit-like cores (q_1 = 1): sum_i min(q_i3, q_i1 q_i2) = 3 + 3 = 6 < D_3 = 8
    ([(1, 3, 4), (1, 3, 4)], [1, 1], (8, 8), [2, 6, 6]),
    # three hits, 4-way: D_2 = 4 binds mode 2, the mode-rank sum binds mode 4
    ([(2, 3, 2, 1), (2, 2, 2, 1), (1, 3, 2, 1)], [5, 4, 1], (4, 7, 9), [5, 4, 6, 3]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stitched_ranks_equal_numerical_multilinear_rank(case):
    shapes, lens, dims, expect = CASES[case]
    hits = _hits(10 + case, shapes, lens, dims)
    big = [50] * len(shapes[0])
    r = stitch.stitched_ranks(hits, dims, big)
    assert r == expect
    # every request at or above the tensor's multilinear rank is clamped to exactly that rank
    assert r == _multilinear_rank(hits)


def test_stitched_ranks_hand_worked():
    hits = _hits(10, *CASES[0][:3])
    assert stitch.stitched_ranks(hits, (6, 5), (2, 6, 5)) == [2, 6, 5]    # nothing binds beyond the request
    assert stitch.stitched_ranks(hits, (6, 5), (1, 10, 10)) == [1, 5, 5]  # r_2 <= r_1 r_3 (fixpoint)
    assert stitch.stitched_ranks(hits, (6, 5), (3, 1, 10)) == [3, 1, 3]   # r_3 <= r_1 r_2
    hits = _hits(11, *CASES[1][:3])
    assert stitch.stitched_ranks(hits, (8, 8), (10, 10, 10)) == [2, 6, 6]
    assert stitch.stitched_ranks(hits, (8, 8), (10, 2, 10)) == [2, 2, 4]  # r_3 <= r_1 r_2 = 4


def test_pins_catch_a_dropped_rank_sum_cap(monkeypatch):
    bad = mutant(stitch.stitched_ranks, "min(ranks[n], ext[n], cap[n])", "min(ranks[n], ext[n])")
    monkeypatch.setattr(stitch, "stitched_ranks", bad)
    shapes, lens, dims, _ = CASES[1]
    hits = _hits(11, shapes, lens, dims)
    assert stitch.stitched_ranks(hits, dims, [50, 50, 50]) != _multilinear_rank(hits)


def _svd_truncation(X, k):
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    return np.diag(s[:k]), [U[:, :k], Vt[:k].T]


def test_paper_metric_is_zero_for_the_reference_itself():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, 8, 7))
    G = rng.standard_normal((3, 3, 2))
    U = [_orth(rng, 9, 3), _orth(rng, 8, 3), _orth(rng, 7, 2)]
    assert metrics.paper_relative_error(X, G, U, G, U) == 0.0


@pytest.mark.parametrize("r", [2, 3, 6])
def test_paper_metric_eckart_young(r):
    # p = 2: the best rank-k model is the truncated SVD, with residual sqrt(sum_{j>k} s_j^2)
    rng = np.random.default_rng(4 + r)
    X = rng.standard_normal((30, 20))
    s = np.linalg.svd(X, compute_uv=False)
    Ga, Ua = _svd_truncation(X, r - 1)
    Gr, Ur = _svd_truncation(X, r)
    expect = np.sqrt(np.sum(s[r - 1:] ** 2)) / np.sqrt(np.sum(s[r:] ** 2)) - 1.0
    got = metrics.paper_relative_error(X, Ga, Ua, Gr, Ur)
    assert got > 0
    assert abs(got - expect) < 1e-10 * expect


def test_pins_catch_a_swapped_metric(monkeypatch):
    bad = mutant(metrics.paper_relative_error, "num / den - 1.0", "den / num - 1.0")
    monkeypatch.setattr(metrics, "paper_relative_error", bad)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((30, 20))
    s = np.linalg.svd(X, compute_uv=False)
    Ga, Ua = _svd_truncation(X, 2)
    Gr, Ur = _svd_truncation(X, 3)
    expect = np.sqrt(np.sum(s[2:] ** 2)) / np.sqrt(np.sum(s[3:] ** 2)) - 1.0
    assert abs(metrics.paper_relative_error(X, Ga, Ua, Gr, Ur) - expect) > 1e-3
