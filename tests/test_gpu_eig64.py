"""FP32 stitch with its eigenproblems in FP64 (tk_config.eig_fp64).

An FP32 tree may solve the eigenproblems of its stitches (Algorithm 2: the
leading eigenvectors of K K^T and N_n N_n^T, orders >= 20 by the tridiagonal
method) in FP64 on the GPU, everything else staying FP32.  On a rank-16 tree
of the batched workload's shapes (200 x 150 slices, first 1024 slices, leaf
16), 120 log-uniform queries through one batched launch, with the stop rule
off (tol = 0, 3 iterations on both sides), are compared with the FP64
oracle, for the plain FP32 stitch and the FP64-eigenproblem variant: both
must meet the FP32 bar of the other parity tests (model distance below
1e-3 ||X||, error values within 1e-3 max(e, 0.1)); the test prints each
variant's error against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from _oracle_pool import oracle_answers  # noqa: E402
from oracle import metrics  # noqa: E402
from oracle.tree import StreamSegmentTree  # noqa: E402


def _batch(X, dims, ranks, B, Q, eig_fp64):
    import paper_2501_06647_gb300 as tk
    dev = torch.device("cuda", 0)
    t = tk.Tree(dims, ranks, leaf_slices=B, max_iter=3, tol=0.0, dtype="f32", eig_fp64=eig_fp64)
    t.build(torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev))
    offs = t.layout(Q)
    out = torch.full((int(offs[-1]),), float("nan"), dtype=torch.float32, device=dev)
    info = (tk.TkQueryInfo * len(Q))()
    t.query_batch(torch.from_numpy(np.ascontiguousarray(Q)).to(dev), torch.from_numpy(offs).to(dev), out, info=info)
    return t, offs, out.cpu().numpy(), info


def test_fp64_eigenproblems_under_an_fp32_stitch():
    w = synth.WORKLOADS["batched_r16"]
    T, dims, ranks, B = 1024, w["dims"], w["ranks"], w["B"]
    X = synth.piecewise_tucker_regimes(T, dims, ranks, w["regime"], w["sigma"], w["seed"])
    Q = synth.query_ranges(T, 120, w["qseed"] + 7, "loguniform", 16, T)
    o = StreamSegmentTree(dims, ranks, B=B, max_iter=3, tol=0.0)
    o.build(np.asarray(X, dtype=np.float64))
    ans = oracle_answers(o, Q)
    stats = {}
    for eig64 in (False, True):
        t, offs, out, info = _batch(X, dims, ranks, B, Q, eig64)
        bad = [(i, tuple(int(x) for x in Q[i]), info[i].n_hits, info[i].iters, info[i].eig_max_order,
                int((~np.isfinite(out[offs[i]:offs[i + 1]])).sum()), int(offs[i + 1] - offs[i]))
               for i in range(len(Q)) if not np.isfinite(out[offs[i]:offs[i + 1]]).all()]
        assert not bad, (eig64, t.heavy_hits, bad[:10])
        assert max(f.eig_max_order for f in info) >= 20  # the tridiagonal method ran
        rel, dist = [], []
        for i, (ts, te) in enumerate(Q):
            ts, te = int(ts), int(te)
            Go, Uo, ro, it, hits = ans[i]
            G, U = t.unpack(out[offs[i]:offs[i + 1]], te - ts)
            r = list(info[i].ranks[: t.p])
            assert r == list(ro) and info[i].iters == it == 3
            G = np.float64(G[tuple(slice(0, x) for x in r)])
            U = [np.float64(u[:, :x]) for u, x in zip(U, r)]
            Xs = np.asarray(X[ts:te], dtype=np.float64)
            ee, eo = metrics.relative_error(Xs, G, U), metrics.relative_error(Xs, Go, Uo)
            d = metrics.model_distance(G, U, Go, Uo) / np.linalg.norm(Xs)
            assert abs(ee - eo) < 1e-3 * max(eo, 0.1), (eig64, ts, te, ee, eo)
            assert d < 1e-3, (eig64, ts, te, d)
            rel.append(abs(ee - eo) / eo)
            dist.append(d)
        stats["fp64 eig" if eig64 else "fp32"] = (float(np.mean(rel)), float(np.max(rel)), float(np.max(dist)))
        t.close()
    print("error values vs the FP64 oracle (mean, max relative difference; max model distance / ||X||): " +
          "; ".join(f"{k}: {a:.2e}, {b:.2e}, {c:.2e}" for k, (a, b, c) in stats.items()))
