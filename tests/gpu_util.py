"""Helpers shared by the GPU parity tests: build the oracle's tree and the
engine's tree over the same seeded series and compare their answers."""
import numpy as np

import synth
from oracle import metrics
from oracle.tree import StreamSegmentTree


def series(T, dims, ranks, regime, sigma, seed):
    return synth.piecewise_tucker(T, dims, ranks, regime, sigma, seed)


def oracle_tree(X, dims, ranks, B, max_iter, tol, theta=(7, 10)):
    t = StreamSegmentTree(dims, ranks, B=B, theta=theta, max_iter=max_iter, tol=tol)
    t.build(X)
    return t


def engine_tree(X, dims, ranks, B, max_iter, tol, dtype, theta=(7, 10), via_appends=False):
    import torch
    import paper_2501_06647_gb300 as tk
    t = tk.Tree(dims, ranks, leaf_slices=B, theta=theta, max_iter=max_iter, tol=tol, dtype=dtype)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64 if dtype == "f64" else np.float32)).cuda()
    if via_appends:
        for i in range(Xd.shape[0]):
            t.append(Xd[i])
    else:
        t.build(Xd)
    t.sync()
    return t


def compare(X, ts, te, Ge, Ue, Go, Uo):
    """Relative difference of the reconstruction errors, model distance over
    ||X||, and the largest principal angle between matching factors."""
    Xs = np.asarray(X[ts:te], dtype=np.float64)
    Ge = np.asarray(Ge, dtype=np.float64)
    Ue = [np.asarray(u, dtype=np.float64) for u in Ue]
    ee = metrics.relative_error(Xs, Ge, Ue)
    eo = metrics.relative_error(Xs, Go, Uo)
    dist = metrics.model_distance(Ge, Ue, Go, Uo) / np.linalg.norm(Xs)
    ang = max(metrics.principal_angle_max(a, b) for a, b in zip(Uo, Ue))
    return abs(ee - eo) / max(eo, 1e-300), dist, ang, ee, eo
