"""Pins for oracle.tree: Algorithms 1, 3, 4 against the paper's worked examples,
theorems, and brute force on tiny timespans."""
import json
import math
import os

import numpy as np
import pytest

from oracle.tree import StreamSegmentTree

GOLD = os.path.join(os.path.dirname(__file__), "golden")


class _Structural(StreamSegmentTree):
    """The oracle's own tree (its Algorithm 3/4 descent and Recall), with only
    the payload arithmetic stubbed: leaves get no decomposition, and the
    module's Stitch and rank clamp are replaced by dummies (autouse fixture
    below), so these pins check the real ``_insert`` / ``append`` code."""

    def _leaf_payload(self, block):
        return None, None


@pytest.fixture(autouse=True)
def _no_payload_arithmetic(monkeypatch):
    import oracle.tree as ot
    monkeypatch.setattr(ot, "stitch", lambda hits, r, max_iter, tol, *start: (None, None, 0, []))
    monkeypatch.setattr(ot, "stitched_ranks", lambda hits, dims, ranks: None)


def _tree(T, B=1, theta=(7, 10)):
    t = _Structural((1,), (1, 1), B=B, theta=theta)
    z = np.zeros((1,))
    for _ in range(T):
        t.append(z)
    return t


def test_worked_example_fig_illust():
    g = json.load(open(os.path.join(GOLD, "fig_illust.json")))
    t = _tree(g["T"], g["B"], tuple(g["theta"]))
    assert t.height() == g["height"]
    assert (t.root.sigma, t.root.tau) == tuple(g["root"])
    recs = t.hit_records(*g["query"])
    assert [list(r[2:]) for r in recs] == g["hits"]


def test_worked_example_append():
    g = json.load(open(os.path.join(GOLD, "append_example.json")))
    t = _tree(g["before"]["T"])
    assert (t.root.sigma, t.root.tau) == tuple(g["before"]["root"]) and t.root.kind == g["before"]["root_kind"]
    old_root = t.root
    t.append(np.zeros((1,)))
    assert (t.root.sigma, t.root.tau) == tuple(g["after"]["root"])
    assert t.root.left is old_root
    v, path = t.root, []
    while v is not None:
        path.append([v.sigma, v.tau])
        v = v.left if (v.left is not None and 8 < v.left.tau) else v.right
    assert path == g["after"]["path_to_leaf"]


@pytest.mark.parametrize("B", [1, 4])
def test_structure_invariants(B):
    for T in range(1, 130):
        t = _tree(T, B)
        nb, nbt = T // B, -(-T // B)
        nodes = t.nodes()
        leaves = [v for v in nodes if v.kind == 'L']
        inter = [v for v in nodes if v.kind == 'M']
        assert len(leaves) == nbt
        assert len(inter) == nb - bin(nb).count("1")          # complete internal nodes
        assert t.stitch_count == nb - bin(nb).count("1")      # one Stitch per completed node
        assert t.height() == math.ceil(math.log2(nbt)) + 1 if nbt > 1 else t.height() == 1
        for v in nodes:                                        # aligned dyadic ranges
            w = v.tau - v.sigma
            assert w & (w - 1) == 0 and v.sigma % w == 0
            if v.kind == 'M':
                assert v.tau <= nb
            if v.kind == 'P':
                assert v.sigma < nbt and v.tau > nb


def test_stitches_per_completed_block_is_trailing_zeros():
    t = _tree(0)
    z = np.zeros((1,))
    for T in range(1, 300):
        before = t.stitch_count
        t.append(z)
        assert t.stitch_count - before == ((T & -T).bit_length() - 1)


def _admissible(t, v, ts, te):
    lo, hi = t.slice_range(v)
    ov = max(0, min(te, hi) - max(ts, lo))
    if ov == 0:
        return False
    if v.kind == 'L':
        return True
    if v.kind == 'M':
        return t.theta[1] * ov >= t.theta[0] * (hi - lo)
    return False


def _brute_min_hits(t, ts, te):
    """Smallest set of admissible nodes whose clipped ranges tile [ts, te) (Eqs. (prune-obj)-(prune-c2))."""
    nodes = [v for v in t.nodes() if _admissible(t, v, ts, te)]
    best = {te: 0}
    for x in range(te - 1, ts - 1, -1):
        cands = []
        for v in nodes:
            lo, hi = t.slice_range(v)
            start = max(ts, lo)
            if start == x and hi > x:
                nxt = min(te, hi)
                if nxt in best:
                    cands.append(1 + best[nxt])
        if cands:
            best[x] = min(cands)
    return best.get(ts)


@pytest.mark.parametrize("B", [1, 2])
def test_recall_is_optimal_and_valid(B):
    # Theorem (prune-opt): Recall attains the minimum of Eq. (prune-obj) under (prune-c1)/(prune-c2).
    for T in (5, 9, 12, 16, 23):
        t = _tree(T, B)
        for ts in range(T):
            for te in range(ts + 1, T + 1):
                hits = t.recall(ts, te)
                covered = []
                for v in hits:
                    assert _admissible(t, v, ts, te)
                    lo, hi = t.slice_range(v)
                    covered.append((max(ts, lo), min(te, hi)))
                assert covered[0][0] == ts and covered[-1][1] == te
                assert all(a[1] == b[0] for a, b in zip(covered, covered[1:]))
                assert len(hits) == _brute_min_hits(t, ts, te)


def test_hit_set_bounds():
    for B in (1, 4):
        for T in (37, 64, 100):
            t = _tree(T, B)
            h = t.height()
            t1 = _tree(T, B, theta=(1, 1))
            for ts in range(0, T, 3):
                for te in range(ts + 1, T + 1, 2):
                    s = len(t.recall(ts, te))
                    s1 = len(t1.recall(ts, te))
                    assert s <= max(2 * (h - 1), 1)          # Lemma (hit-height)
                    assert s <= s1                            # pruning never enlarges the hit set
                    nblk = (te - 1) // B - ts // B + 1        # leaf blocks touched
                    assert s1 <= max(1, 2 * math.ceil(math.log2(nblk)))   # blocks touched, leaves terminal


def test_theta_one_is_canonical_cover():
    # With theta = 1 and B = 1 every hit is an entire hit: the canonical segment-tree decomposition
    # into maximal aligned dyadic intervals of complete nodes, found here greedily left to right.
    T = 77
    t = _tree(T, 1, theta=(1, 1))
    for ts in range(T):
        for te in range(ts + 1, T + 1):
            recs = [(r[2], r[3]) for r in t.hit_records(ts, te)]
            greedy, x = [], ts
            while x < te:
                w = 1
                while x % (2 * w) == 0 and x + 2 * w <= te:
                    w *= 2
                greedy.append((x, x + w))
                x += w
            assert recs == greedy
            assert len(recs) <= max(1, 2 * math.ceil(math.log2(te - ts)))


# ---- planted mistake: the pins above must catch a slip in the oracle's descent ----------------

def test_pins_catch_a_wrong_completion_test(monkeypatch):
    # Plant a slip in Algorithm 3's completion test of an intermediate node (tau_v = b + 1,
    # in block units): compare with b instead.  The stitch-count invariant must fail.
    from _mutate import mutant
    import oracle.tree as ot
    bad = mutant(ot.StreamSegmentTree._insert, "complete and v.tau == b + 1", "complete and v.tau == b")
    monkeypatch.setattr(ot.StreamSegmentTree, "_insert", bad)
    t = _tree(0)
    z = np.zeros((1,))
    counts_ok = True
    for T in range(1, 64):
        before = t.stitch_count
        t.append(z)
        counts_ok &= t.stitch_count - before == ((T & -T).bit_length() - 1)
    assert not counts_ok
