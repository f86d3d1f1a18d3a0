"""Parity at the full size of the FP32 plain workload, in the launch that the
benchmark times.

The tree is the benchmark's: 4096 slices of 100 x 100, ranks (10, 10, 10),
leaves of 16 slices, max_iter 20, tol 0.01, FP32.  All 1,000 log-uniform
queries (16..4096) plus the extreme ranges (the whole series, single slices,
the last slice) go through one tk_range_query_batch call on device buffers,
the call the benchmark times.  Checked:

- every query: the hit set (Algorithm 1) bit for bit against the oracle's, the
  hit count the batch reports, ranks within the clamps, finite outputs,
  orthonormal factors;
- a sample of 30 queries (every 40th, and the extreme ranges) against the FP64
  oracle's own answers: effective ranks equal, and where both sides ran the
  same number of ALS iterations, the model within 1e-3 ||X|| and the error
  values within 1e-3 max(e, 0.1), the FP32 bar of the smaller parity tests;
- the same call with host buffers (the end-to-end path) gives the same
  outputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from oracle import metrics  # noqa: E402
from oracle.tree import StreamSegmentTree  # noqa: E402


def test_plain_workload_full_size_batch():
    import paper_2501_06647_gb300 as tk
    w = synth.WORKLOADS["fp32_plain"]
    T, dims, ranks = w["T"], w["dims"], w["ranks"]
    X = synth.piecewise_tucker(T, dims, ranks, w["regime"], w["sigma"], w["seed"])
    Q = synth.query_ranges(T, w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    extremes = np.array([(0, T), (0, 1), (T - 1, T), (17, 18), (T // 2 - 1, T // 2 + 1)], dtype=np.int64)
    Q = np.concatenate([Q, extremes])
    n = len(Q)

    dev = torch.device("cuda", 0)
    tree = tk.Tree(dims, ranks, leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32")
    tree.build(torch.from_numpy(X.astype(np.float32)).to(dev))
    tree.sync()
    offs = tree.layout(Q)
    out_d = torch.full((int(offs[-1]),), float("nan"), dtype=torch.float32, device=dev)
    info = (tk.TkQueryInfo * n)()
    tree.query_batch(torch.from_numpy(Q.copy()).to(dev), torch.from_numpy(offs).to(dev), out_d, info=info)
    out = out_d.cpu().numpy()
    assert np.isfinite(out).all()

    oracle = StreamSegmentTree(dims, ranks, B=w["B"], max_iter=20, tol=0.01)
    oracle.build(X)

    worst_orth = 0.0
    for i, (ts, te) in enumerate(Q):
        ts, te = int(ts), int(te)
        ho = oracle.hit_records(ts, te)
        assert [tuple(h[:6]) for h in tree.hit_set(ts, te)] == ho, (ts, te)
        assert info[i].n_hits == len(ho), (ts, te)
        r = list(info[i].ranks[: tree.p])
        assert 1 <= r[0] <= min(ranks[0], te - ts)
        assert all(1 <= a <= b for a, b in zip(r[1:], ranks[1:]))
        _, U = tree.unpack(out[offs[i]:offs[i + 1]], te - ts)
        for u, x in zip(U, r):
            u = np.float64(u[:, :x])
            worst_orth = max(worst_orth, float(np.abs(u.T @ u - np.eye(x)).max()))
    assert worst_orth < 1e-3, worst_orth

    sample = list(range(0, w["n_queries"], 40)) + list(range(w["n_queries"], n))
    agree, worst_dist = 0, 0.0
    for i in sample:
        ts, te = int(Q[i][0]), int(Q[i][1])
        ro = oracle.query(ts, te)
        r = list(info[i].ranks[: tree.p])
        assert tuple(r) == tuple(ro["ranks"]), (ts, te)
        if info[i].iters != ro["iters"]:
            continue
        agree += 1
        G, U = tree.unpack(out[offs[i]:offs[i + 1]], te - ts)
        G = np.float64(G[tuple(slice(0, x) for x in r)])
        U = [np.float64(u[:, :x]) for u, x in zip(U, r)]
        Xs = X[ts:te]
        dist = metrics.model_distance(G, U, ro["G"], ro["U"]) / np.linalg.norm(Xs)
        worst_dist = max(worst_dist, dist)
        assert dist < 1e-3, (ts, te, dist)
        ee, eo = metrics.relative_error(Xs, G, U), metrics.relative_error(Xs, ro["G"], ro["U"])
        assert abs(ee - eo) < 1e-3 * max(eo, 0.1), (ts, te, ee, eo)
    # the stop rule can flip near its threshold on either side; most must agree
    assert agree >= 0.8 * len(sample), (agree, len(sample))
    print("full size: %d queries, worst factor orthonormality %.1e, %d/%d sampled queries with equal "
          "iteration counts, worst model distance %.2e ||X||" % (n, worst_orth, agree, len(sample), worst_dist))

    host_out, _, _ = tree.query_batch_host(Q, offs, None, with_info=False)
    assert np.allclose(host_out, out, rtol=1e-5, atol=1e-5)
    tree.close()
