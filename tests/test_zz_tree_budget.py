"""The tree's device-memory budget (tk_config.hbm_budget): a call whose
allocation would take the bytes the tree holds above the budget fails with
TK_ERR_NOMEM and changes nothing; under a budget that fits, the tree is the
same as without one, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import series, engine_tree  # noqa: E402

NOMEM = -4


def test_budget_is_enforced_and_changes_nothing_else():
    import paper_2501_06647_gb300 as tk
    dims, ranks, B, T = (30, 20), (5, 5, 5), 4, 256
    X = series(T, dims, ranks, 64, 0.01, 1001)
    ref = engine_tree(X, dims, ranks, B, 3, 0.0, "f64")
    kw = dict(leaf_slices=B, max_iter=3, tol=0.0, dtype="f64")

    # the empty tree alone (open-block slices: 4 x 30 x 20 doubles) exceeds 1 KiB
    with pytest.raises(tk.TuckerError) as ei:
        tk.Tree(dims, ranks, hbm_budget=1024, **kw)
    assert ei.value.code == NOMEM

    # 200 KiB holds the empty tree but not the arena of 64 leaf blocks (~0.45 MiB)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    t = tk.Tree(dims, ranks, hbm_budget=200 << 10, **kw)
    with pytest.raises(tk.TuckerError) as ei:
        t.build(Xd)
    assert ei.value.code == NOMEM
    assert t.T == 0 and t.arena_bytes() < (200 << 10)
    t.close()

    # 1 GiB: the same tree and answers as without a budget
    t = tk.Tree(dims, ranks, hbm_budget=1 << 30, **kw)
    t.build(Xd)
    t.sync()
    assert t.T == T and t.arena_bytes() == ref.arena_bytes()
    for level, k in [(0, 0), (0, 63), (3, 2), (6, 0)]:
        Ha, Va, ra = ref.node_payload(level, k)
        Hb, Vb, rb = t.node_payload(level, k)
        assert ra == rb and np.array_equal(Ha, Hb) and all(np.array_equal(x, y) for x, y in zip(Va, Vb))
    for ts, te in [(0, T), (5, 201), (100, 101)]:
        Ga, Ua, _ = ref.query(ts, te)
        Gb, Ub, _ = t.query(ts, te)
        assert np.array_equal(Ga, Gb) and all(np.array_equal(x, y) for x, y in zip(Ua, Ub))
    t.close()
    ref.close()
