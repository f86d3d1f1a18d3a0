"""Parity of the batch kernel (k_batch, the launch the benchmark times) against
the FP64 oracle where the smaller tests do not reach:

- heavy queries in FP64: with a temporal build rank of 20 the batch runs every
  query of at least 3 hits on a whole 512-thread CTA (the threshold is
  max(3, ceil(55 / max rank))); every query is compared at the FP64 bar
  (error values within 1e-9 relative, factor subspaces within 1e-3 rad);
- the full FP32 plain workload (4096 slices of 100 x 100, ranks 10, leaf 16)
  with the stop rule off (tol = 0) and 4 ALS iterations on both sides, so that
  every one of its 1,000 queries is compared with the oracle, none skipped;
- a rank-16 tree of 200 x 150 slices (the batched workload's shapes, first
  1024 slices), 120 queries through one batched call.

The FP32 bar is the one of the other parity tests: ||Y_gpu - Y_oracle||_F <=
1e-3 ||X||_F and error values within 1e-3 max(e, 0.1).  Oracle queries run in
a process pool (spawned, so that no worker inherits the CUDA context).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from gpu_util import compare  # noqa: E402
from _oracle_pool import oracle_answers  # noqa: E402
from oracle import metrics  # noqa: E402
from oracle.tree import StreamSegmentTree  # noqa: E402

def _engine_batch(X, dims, ranks, B, max_iter, tol, dtype, Q, heavy=None):
    import paper_2501_06647_gb300 as tk
    dev = torch.device("cuda", 0)
    t = tk.Tree(dims, ranks, leaf_slices=B, max_iter=max_iter, tol=tol, dtype=dtype)
    t.build(torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64 if dtype == "f64" else np.float32)).to(dev))
    t.sync()
    if heavy is not None:
        t.heavy_hits = heavy
    offs = t.layout(Q)
    out = torch.full((int(offs[-1]),), float("nan"), dtype=torch.float64 if dtype == "f64" else torch.float32,
                     device=dev)
    info = (tk.TkQueryInfo * len(Q))()
    t.query_batch(torch.from_numpy(np.ascontiguousarray(Q)).to(dev), torch.from_numpy(offs).to(dev), out, info=info)
    return t, offs, out.cpu().numpy(), info


def _answer(t, out, offs, info, i, L):
    G, U = t.unpack(out[offs[i]:offs[i + 1]], L)
    r = list(info[i].ranks[: t.p])
    return np.float64(G[tuple(slice(0, x) for x in r)]), [np.float64(u[:, :x]) for u, x in zip(U, r)], r


def test_heavy_queries_fp64():
    dims, ranks, B, T = (24, 22), (20, 8, 8), 4, 256
    X = synth.piecewise_tucker(T, dims, ranks, T, 0.01, 31)  # one regime: a clear gap after the kept ranks
    Q = np.concatenate([synth.query_ranges(T, 150, 32), np.array([[0, T], [1, T - 1]], dtype=np.int64)])
    t, offs, out, info = _engine_batch(X, dims, ranks, B, 3, 0.0, "f64", Q)
    o = StreamSegmentTree(dims, ranks, B=B, max_iter=3, tol=0.0)
    o.build(X)
    ans = oracle_answers(o, Q)
    heavy, worst = 0, [0.0, 0.0]
    for i, (ts, te) in enumerate(Q):
        Go, Uo, ro, it, hits = ans[i]
        Ge, Ue, r = _answer(t, out, offs, info, i, int(te - ts))
        assert r == list(ro) and info[i].iters == it == 3 and info[i].n_hits == len(hits), (ts, te)
        heavy += len(hits) >= 3
        rel, dist, ang, ee, eo = compare(X, int(ts), int(te), Ge, Ue, Go, Uo)
        worst = [max(worst[0], rel), max(worst[1], ang)]
        assert rel < 1e-9, (ts, te, ee, eo)
        assert ang < 1e-3, (ts, te, ang)
    assert heavy >= 40, heavy
    print(f"heavy: {heavy}/{len(Q)} queries of >= 3 hits; worst rel diff {worst[0]:.1e}, angle {worst[1]:.1e}")
    t.close()


def test_heavy_threshold_changes_only_the_launch_shape():
    """The same FP64 batch with every query of >= 3 hits on a whole CTA (the
    default for a build rank of 20), with every query on a half CTA, and with
    every query on a whole CTA: the answers agree to FP64 rounding."""
    import paper_2501_06647_gb300 as tk
    dims, ranks, B, T = (24, 22), (20, 8, 8), 4, 256
    X = synth.piecewise_tucker(T, dims, ranks, T, 0.01, 31)
    Q = synth.query_ranges(T, 60, 33)
    answers = []
    for heavy in (None, 65, 1):
        t, offs, out, info = _engine_batch(X, dims, ranks, B, 3, 0.0, "f64", Q, heavy)
        assert t.heavy_hits == (3 if heavy is None else heavy)
        answers.append([_answer(t, out, offs, info, i, int(te - ts)) for i, (ts, te) in enumerate(Q)])
        if heavy == 1:
            t.heavy_hits = 0  # back to the default
            assert t.heavy_hits == 3
            with pytest.raises(tk.TuckerError):
                t.heavy_hits = -1
        t.close()
    # the autotuner leaves one of its candidates set and the same answers
    dev = torch.device("cuda", 0)
    t, offs, out, info = _engine_batch(X, dims, ranks, B, 3, 0.0, "f64", Q)
    rd, od = torch.from_numpy(np.ascontiguousarray(Q)).to(dev), torch.from_numpy(offs).to(dev)
    o2 = torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev)
    best, ms = t.tune_batch(rd, od, o2, reps=1)
    assert best in (3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32, 65) and t.heavy_hits == best and ms > 0
    t.query_batch(rd, od, o2, info=info)
    answers.append([_answer(t, o2.cpu().numpy(), offs, info, i, int(te - ts)) for i, (ts, te) in enumerate(Q)])
    t.close()
    for other in answers[1:]:
        for i, (ts, te) in enumerate(Q):
            (Ga, Ua, ra), (Gb, Ub, rb) = answers[0][i], other[i]
            assert ra == rb
            rel, dist, ang, ea, eb = compare(X, int(ts), int(te), Gb, Ub, Ga, Ua)
            assert rel < 1e-9 and ang < 1e-3, (ts, te, rel, ang)


def _fp32_bar(X, Q, t, offs, out, info, ans, iters):
    worst = 0.0
    for i, (ts, te) in enumerate(Q):
        ts, te = int(ts), int(te)
        Go, Uo, ro, it, hits = ans[i]
        Ge, Ue, r = _answer(t, out, offs, info, i, te - ts)
        assert r == list(ro) and info[i].iters == it == iters, (ts, te, r, ro, info[i].iters, it)
        assert info[i].n_hits == len(hits)
        assert [tuple(h[:6]) for h in t.hit_set(ts, te)] == hits, (ts, te)
        Xs = np.asarray(X[ts:te], dtype=np.float64)
        dist = metrics.model_distance(Ge, Ue, Go, Uo) / np.linalg.norm(Xs)
        worst = max(worst, dist)
        assert dist < 1e-3, (ts, te, dist)
        ee, eo = metrics.relative_error(Xs, Ge, Ue), metrics.relative_error(Xs, Go, Uo)
        assert abs(ee - eo) < 1e-3 * max(eo, 0.1), (ts, te, ee, eo)
    return worst


def test_plain_workload_every_query_fixed_iterations():
    w = synth.WORKLOADS["fp32_plain"]
    T, dims, ranks = w["T"], w["dims"], w["ranks"]
    X = synth.piecewise_tucker(T, dims, ranks, w["regime"], w["sigma"], w["seed"])
    Q = synth.query_ranges(T, w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    Q = np.concatenate([Q, np.array([(0, T), (0, 1), (T - 1, T), (17, 18), (T // 2 - 1, T // 2 + 1)],
                                    dtype=np.int64)])
    t, offs, out, info = _engine_batch(X, dims, ranks, w["B"], 4, 0.0, "f32", Q)
    assert np.isfinite(out).all()
    o = StreamSegmentTree(dims, ranks, B=w["B"], max_iter=4, tol=0.0)
    o.build(X)
    worst = _fp32_bar(X, Q, t, offs, out, info, oracle_answers(o, Q), 4)
    print(f"full size, every query: {len(Q)} queries, worst model distance {worst:.2e} ||X||")
    t.close()


def test_rank16_wide_slices_through_the_batch_kernel():
    w = synth.WORKLOADS["batched_r16"]
    T, dims, ranks = 1024, w["dims"], w["ranks"]
    X = synth.piecewise_tucker_regimes(T, dims, ranks, w["regime"], w["sigma"], w["seed"])
    Q = synth.query_ranges(T, 120, w["qseed"], "loguniform", 16, T)
    t, offs, out, info = _engine_batch(X, dims, ranks, w["B"], 3, 0.0, "f32", Q)
    assert np.isfinite(out).all()
    o = StreamSegmentTree(dims, ranks, B=w["B"], max_iter=3, tol=0.0)
    o.build(np.asarray(X, dtype=np.float64))
    worst = _fp32_bar(X, Q, t, offs, out, info, oracle_answers(o, Q), 3)
    print(f"rank 16, 200 x 150: {len(Q)} queries, worst model distance {worst:.2e} ||X||")
    t.close()
