"""Tree files (tk_tree_save / tk_tree_load): a loaded tree holds the saved
arena byte for byte, so it answers queries and takes further appends exactly
as the saved tree does.  Compared bit for bit: every node payload, queries
over the whole series, single slices and the open leaf block, before and
after more appends to both trees; saved once while the open block awaits its
decomposition and once after a query has decomposed it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import series, engine_tree  # noqa: E402


def _same_payloads(a, b):
    nbt = (a.T + a.B - 1) // a.B
    for level in range(0, 12):
        for k in range(0, max(1, nbt >> level)):
            if level > 0 and ((k + 1) << level) > a.T // a.B:
                continue  # no intermediate node completed here yet
            Ha, Va, ra = a.node_payload(level, k)
            Hb, Vb, rb = b.node_payload(level, k)
            assert ra == rb, (level, k)
            assert np.array_equal(Ha, Hb) and all(np.array_equal(x, y) for x, y in zip(Va, Vb)), (level, k)


def _same_answers(a, b, ranges):
    for ts, te in ranges:
        Ga, Ua, ia = a.query(ts, te)
        Gb, Ub, ib = b.query(ts, te)
        assert ia["ranks"] == ib["ranks"] and ia["iters"] == ib["iters"], (ts, te)
        assert np.array_equal(Ga, Gb) and all(np.array_equal(x, y) for x, y in zip(Ua, Ub)), (ts, te)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_loaded_tree_answers_and_grows_like_the_saved_one(dtype, tmp_path):
    import paper_2501_06647_gb300 as tk
    dims, ranks, B = (30, 20), (5, 5, 5), 4
    X = series(203, dims, ranks, 64, 0.01, 1001)
    a = engine_tree(X[:150], dims, ranks, B, 4, 0.0, dtype)  # 37 blocks and 2 open slices
    path = tmp_path / "a.tkt"
    a.save(path)
    b = tk.Tree.load(path, device=0)
    assert (b.T, b.dims, b.ranks, b.B, b.dtype) == (150, dims, ranks, B, dtype)
    assert b.arena_bytes() == a.arena_bytes()
    _same_payloads(a, b)
    _same_answers(a, b, [(0, 150), (3, 149), (148, 150), (149, 150), (17, 18), (40, 97)])

    # saved again after queries decomposed the open block
    path2 = tmp_path / "a2.tkt"
    a.save(path2)
    c = tk.Tree.load(path2)
    _same_payloads(a, c)
    _same_answers(a, c, [(0, 150), (147, 150)])

    # more appends to all three, across block completions and a new root
    for t in range(150, 203):
        for tr in (a, b, c):
            tr.append(X[t])
    for tr in (a, b, c):
        tr.sync()
    assert a.T == b.T == c.T == 203
    _same_payloads(a, b)
    _same_payloads(a, c)
    _same_answers(a, b, [(0, 203), (150, 203), (201, 203), (60, 190)])
    _same_answers(a, c, [(0, 203), (199, 203)])
    for tr in (a, b, c):
        tr.close()


def test_load_rejects_a_file_of_another_tree_size(tmp_path):
    import paper_2501_06647_gb300 as tk
    a = engine_tree(series(40, (9, 7), (3, 3, 3), 16, 0.05, 7), (9, 7), (3, 3, 3), 4, 3, 0.0, "f64")
    path = tmp_path / "t.tkt"
    a.save(path)
    raw = path.read_bytes()
    for bad in (raw[:-1], raw + b"\0"):
        path.write_bytes(bad)
        with pytest.raises(tk.TuckerError) as ei:
            tk.Tree.load(path)
        assert ei.value.code == -10
    path.write_bytes(raw)
    b = tk.Tree.load(path)
    _same_answers(a, b, [(0, 40), (5, 33)])
    a.close()
    b.close()
