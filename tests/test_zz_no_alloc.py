"""The allocation-free batched query entry point (tk_range_query_batch_noalloc).

Some callers cannot let a library allocate device memory at query time: a
runtime that owns all device memory through its own arena, or a latency-bound
loop that must not pay for cudaMalloc/cudaFree and the device-wide
synchronization they may cause.  This entry point runs the same batched stitch
kernel on a fixed 16 MiB device array instead of allocated workspaces.  These
tests call it through the C ABI twice in a row and check each result against
the regular batched entry point (tk_range_query_batch), within the FP64 parity
tolerance of the other GPU tests (reconstruction error values within 1e-9
relative, factors within 1e-3 rad) and elementwise for the FP32 tree.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from gpu_util import series, engine_tree  # noqa: E402
from oracle import metrics  # noqa: E402


def _batch(tree, Q):
    import paper_2501_06647_gb300 as tk
    offs = tree.layout(Q)
    dev = torch.device("cuda", 0)
    r = torch.from_numpy(Q.copy()).to(dev)
    o = torch.from_numpy(offs).to(dev)
    dt = torch.float64 if tree.dtype == "f64" else torch.float32
    ref = torch.zeros(int(offs[-1]), dtype=dt, device=dev)
    info_ref = (tk.TkQueryInfo * len(Q))()
    tree.query_batch(r, o, ref, info=info_ref)
    return offs, r, o, ref, info_ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_regular_batch_twice(dtype):
    import paper_2501_06647_gb300 as tk
    if dtype == "f64":
        dims, ranks, T, B = (30, 20), (5, 5, 5), 256, 4
        X = series(T, dims, ranks, 64, 0.01, 1001)
        Q = synth.query_ranges(T, 60, 2001)
    else:
        dims, ranks, T, B = (60, 50), (10, 10, 10), 512, 16
        X = series(T, dims, ranks, 128, 0.05, 1002)
        Q = synth.query_ranges(T, 60, 2002, "loguniform", 16, T)
    tree = engine_tree(X, dims, ranks, B, 4, 0.0, dtype)
    offs, r, o, ref, info_ref = _batch(tree, Q)
    ref_h = ref.cpu().numpy()
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        info = (tk.TkQueryInfo * len(Q))()
        tree.query_batch_noalloc(r, o, out, info=info)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        for i, (ts, te) in enumerate(Q):
            assert list(info[i].ranks) == list(info_ref[i].ranks)
            assert info[i].iters == info_ref[i].iters and info[i].n_hits == info_ref[i].n_hits
            rk = list(info[i].ranks[: tree.p])
            Ga, Ua = tree.unpack(ref_h[offs[i]:offs[i + 1]], int(te - ts))
            Gb, Ub = tree.unpack(got[offs[i]:offs[i + 1]], int(te - ts))
            Ga = np.float64(Ga[tuple(slice(0, x) for x in rk)])
            Gb = np.float64(Gb[tuple(slice(0, x) for x in rk)])
            Ua = [np.float64(u[:, :x]) for u, x in zip(Ua, rk)]
            Ub = [np.float64(u[:, :x]) for u, x in zip(Ub, rk)]
            Xs = X[int(ts):int(te)]
            ea, eb = metrics.relative_error(Xs, Ga, Ua), metrics.relative_error(Xs, Gb, Ub)
            if dtype == "f64":
                assert abs(ea - eb) <= 1e-9 * ea
                assert max(metrics.principal_angle_max(a, b) for a, b in zip(Ua, Ub)) < 1e-3
            else:
                assert np.allclose(got[offs[i]:offs[i + 1]], ref_h[offs[i]:offs[i + 1]], rtol=0, atol=1e-6)
    # an asynchronous call (no report) followed by the tree's sync gives the same output
    out = torch.zeros_like(ref)
    tree.query_batch_noalloc(r, o, out)
    tree.sync()
    assert np.allclose(out.cpu().numpy(), ref_h, rtol=0, atol=1e-12 if dtype == "f64" else 1e-6)
    tree.close()


def test_noalloc_rejects_what_does_not_fit():
    import paper_2501_06647_gb300 as tk
    # 6-way tree with rank-10 cores: one query's workspace exceeds the 16 MiB array
    t = tk.Tree((10, 10, 10, 10, 10), (10,) * 6, leaf_slices=1, dtype="f32")
    dev = torch.device("cuda", 0)
    r = torch.tensor([[0, 1]], dtype=torch.int64, device=dev)
    o = torch.tensor([0, 1], dtype=torch.int64, device=dev)
    out = torch.zeros(1, device=dev)
    with pytest.raises(tk.TuckerError) as ei:
        t.query_batch_noalloc(r, o, out)
    assert ei.value.code == -8
    t.close()


def test_noalloc_refuses_an_undecomposed_open_block():
    import paper_2501_06647_gb300 as tk
    dims, ranks = (9, 7), (3, 3, 3)
    X = series(10, dims, ranks, 10, 0.05, 4)
    t = tk.Tree(dims, ranks, leaf_slices=4, max_iter=3, tol=0.0, dtype="f64")
    t.build(torch.from_numpy(X).cuda())       # 2 complete blocks + a tail of 2 slices
    dev = torch.device("cuda", 0)
    Q = np.array([[0, 10]], dtype=np.int64)
    offs = t.layout(Q)
    r, o = torch.from_numpy(Q).to(dev), torch.from_numpy(offs).to(dev)
    out = torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev)
    with pytest.raises(tk.TuckerError) as ei:
        t.query_batch_noalloc(r, o, out)
    assert ei.value.code == -6
    t.query(0, 10)                             # a regular query decomposes the open block
    t.query_batch_noalloc(r, o, out)
    t.sync()
    t.close()


def test_noalloc_device_errors_reach_tk_sync():
    # An invalid range inside a device-resident batch is found by the kernel; the
    # call (no report) leaves it in the tree's sticky status word, which the
    # next tk_sync returns: the binding's own, right after the launch, on a
    # tree with a stream of its own, else the caller's.
    import paper_2501_06647_gb300 as tk
    dims, ranks = (9, 7), (3, 3, 3)
    X = series(32, dims, ranks, 16, 0.05, 5)
    t = engine_tree(X, dims, ranks, 4, 3, 0.0, "f64")
    dev = torch.device("cuda", 0)
    Q = np.array([[0, 8], [4, 40]], dtype=np.int64)          # the second ends beyond T = 32
    offs = t.layout(Q)
    r, o = torch.from_numpy(Q).to(dev), torch.from_numpy(offs).to(dev)
    out = torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev)
    with pytest.raises(tk.TuckerError) as ei:
        t.query_batch_noalloc(r, o, out)
        t.sync()
    assert ei.value.code == -2 and "tk_sync" in str(ei.value)
    t.close()


def test_noalloc_reports_share_the_scratch_array():
    # With reports, n tk_query_info records are staged in the 16 MiB array too:
    # a batch whose reports alone exceed it is refused (TK_ERR_TOO_BIG); the
    # same batch without reports runs.
    import paper_2501_06647_gb300 as tk
    dims, ranks = (9, 7), (3, 3, 3)
    X = series(32, dims, ranks, 16, 0.05, 6)
    t = engine_tree(X, dims, ranks, 4, 2, 0.0, "f64")
    n = (16 << 20) // ctypes.sizeof(tk.TkQueryInfo) + 1
    dev = torch.device("cuda", 0)
    Q = np.tile(np.array([[3, 5]], dtype=np.int64), (n, 1))
    offs = t.layout(Q)
    r, o = torch.from_numpy(Q).to(dev), torch.from_numpy(offs).to(dev)
    out = torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev)
    info = (tk.TkQueryInfo * n)()
    with pytest.raises(tk.TuckerError) as ei:
        t.query_batch_noalloc(r, o, out, info=info)
    assert ei.value.code == -8
    t.query_batch_noalloc(r, o, out)
    t.sync()
    ref_out = torch.zeros(int(offs[1]), dtype=torch.float64, device=dev)
    t.query_batch(r[:1].contiguous(), o[:2].contiguous(), ref_out)
    got = out.cpu().numpy()
    first = ref_out.cpu().numpy()
    assert np.allclose(got[: int(offs[1])], first, rtol=0, atol=1e-12)
    assert np.allclose(got[int(offs[-2]):], first, rtol=0, atol=1e-12)
    t.close()
