"""The leaf blocks' Gram matrices on the tensor cores (tk_config.math).

An FP32 tree decomposes its leaf blocks with Tucker-ALS (Section 2), whose
dense contractions are the Gram matrices mat_n(X) mat_n(X)^T of the raw block
(the HOSVD start) and of mat_n(Y_n) in every ALS step.  With TK_MATH_AUTO
they run on the tensor cores as split-TF32 products (FP32 accuracy), with
TK_MATH_TF32 as single TF32 products, with TK_MATH_CUDA_CORES on the FP32
CUDA cores.  Each tree is checked against the FP64 oracle's tree, node by
node (the stored decomposition's model distance relative to the node's
norm): the split-TF32 tree must be as close to the oracle as the CUDA-core
tree (within twice its distance, or 1e-4), the single-TF32 tree within 5e-2,
and the split-TF32 tree's queries must meet the FP32 parity bar of the other
tests.  Shapes
cover both staging paths of the tensor-core Gram (columns contiguous in
memory, and rows of the last mode) and Gram orders of one and two 128-row
tiles.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from gpu_util import series, oracle_tree  # noqa: E402
from oracle import metrics  # noqa: E402

CASES = [
    # (dims, ranks, B, T): Gram orders 64/48 (one tile), a 4-way tree (inner > 1 and inner = 1),
    # and orders 160/40 (two tiles for mode 2)
    ((64, 48), (8, 8, 8), 16, 128),
    ((40, 36, 32), (6, 6, 6, 6), 8, 64),
    ((160, 40), (10, 10, 10), 16, 96),
]


def _engine(X, dims, ranks, B, math):
    import paper_2501_06647_gb300 as tk
    t = tk.Tree(dims, ranks, leaf_slices=B, max_iter=4, tol=0.0, dtype="f32", math=math)
    t.build(torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda())
    t.sync()
    return t


def _worst_node_distance(o, e):
    worst = 0.0
    for v in o.nodes():
        if v.kind not in ("L", "M"):
            continue
        w = v.tau - v.sigma
        level = w.bit_length() - 1
        H, V, r = e.node_payload(level, v.sigma >> level)
        assert list(H.shape) == list(v.H.shape)
        d = metrics.model_distance(np.float64(H), [np.float64(x) for x in V], v.H, v.V) / np.linalg.norm(v.H)
        worst = max(worst, d)
    return worst


@pytest.mark.parametrize("case", range(len(CASES)))
def test_leaf_grams_match_the_oracle(case):
    dims, ranks, B, T = CASES[case]
    X = series(T, dims, ranks, 32, 0.05, 40 + case)
    o = oracle_tree(X, dims, ranks, B, 4, 0.0)
    worst = {}
    for math in ("cuda_cores", "auto", "tf32"):
        e = _engine(X, dims, ranks, B, math)
        worst[math] = _worst_node_distance(o, e)
        if math == "auto":
            for ts, te in synth.query_ranges(T, 12, 50 + case):
                ro = o.query(int(ts), int(te))
                Ge, Ue, info = e.query(int(ts), int(te))
                Xs = X[int(ts):int(te)]
                dist = metrics.model_distance(np.float64(Ge), [np.float64(u) for u in Ue], ro["G"], ro["U"])
                assert dist < 1e-3 * np.linalg.norm(Xs), (ts, te, dist)
        e.close()
    print(f"{dims}: worst node model distance to the FP64 oracle: " +
          ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))
    # split TF32 is as accurate as the FP32 CUDA cores; single TF32 (products
    # rounded to 11 significant bits) within 5e-2
    assert worst["auto"] <= max(2.0 * worst["cuda_cores"], 1e-4), worst
    assert worst["tf32"] < 5e-2, worst


def test_tf32_rejected_for_fp64_trees():
    import paper_2501_06647_gb300 as tk
    with pytest.raises(tk.TuckerError) as ei:
        tk.Tree((8, 8), (3, 3, 3), dtype="f64", math="tf32")
    assert ei.value.code == -1
