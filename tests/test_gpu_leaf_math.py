"""The leaf blocks' Gram matrices on the tensor cores (tk_config.math).

An FP32 tree decomposes its leaf blocks with Tucker-ALS (Section 2), whose
dense contractions are the Gram matrices mat_n(X) mat_n(X)^T of the raw block
(the HOSVD start) and of mat_n(Y_n) in every ALS step.  With TK_MATH_AUTO
they run on the tensor cores as split-TF32 products (FP32 accuracy), with
TK_MATH_TF32 as single TF32 products, with TK_MATH_CUDA_CORES on the FP32
CUDA cores.  Each tree is checked against the FP64 oracle's tree, node by
node: the stored decomposition's model distance relative to the node's
norm must stay within the arithmetic's bar (2e-4 for FP32 accuracy, 2e-2 for
TF32), and queries must meet the FP32 parity bar of the other tests.  Shapes
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

BAR = {"auto": 2e-4, "cuda_cores": 2e-4, "tf32": 2e-2}
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


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("math", ["auto", "tf32", "cuda_cores"])
def test_leaf_grams_match_the_oracle(case, math):
    dims, ranks, B, T = CASES[case]
    X = series(T, dims, ranks, 32, 0.05, 40 + case)
    o = oracle_tree(X, dims, ranks, B, 4, 0.0)
    e = _engine(X, dims, ranks, B, math)
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
    assert worst < BAR[math], (math, worst)
    if math != "tf32":
        for ts, te in synth.query_ranges(T, 12, 50 + case):
            ro = o.query(int(ts), int(te))
            Ge, Ue, info = e.query(int(ts), int(te))
            Xs = X[int(ts):int(te)]
            dist = metrics.model_distance(np.float64(Ge), [np.float64(u) for u in Ue], ro["G"], ro["U"])
            assert dist < 1e-3 * np.linalg.norm(Xs), (ts, te, dist)
    print(f"{math} {dims}: worst node model distance {worst:.2e}")
    e.close()


def test_tf32_rejected_for_fp64_trees():
    import paper_2501_06647_gb300 as tk
    with pytest.raises(tk.TuckerError) as ei:
        tk.Tree((8, 8), (3, 3, 3), dtype="f64", math="tf32")
    assert ei.value.code == -1
