"""The C ABI refuses, with TK_ERR_ARG and before any launch, buffers passed as
device memory that are not device memory of the tree's GPU (here: host
memory), so that no kernel is ever given a host pointer."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import series, engine_tree  # noqa: E402

ARG = -1


def test_host_pointers_as_device_buffers_are_refused():
    import paper_2501_06647_gb300 as tk
    lib = tk.lib()
    dims, ranks = (9, 7), (3, 3, 3)
    X = series(32, dims, ranks, 16, 0.05, 7)
    t = engine_tree(X, dims, ranks, 4, 2, 0.0, "f64")
    Q = np.array([[0, 8]], dtype=np.int64)
    offs = t.layout(Q)
    out = np.zeros(int(offs[-1]))
    dev = torch.device("cuda", 0)
    rd, od = torch.from_numpy(Q).to(dev), torch.from_numpy(offs).to(dev)
    outd = torch.zeros(int(offs[-1]), dtype=torch.float64, device=dev)
    h = lambda a: ctypes.c_void_p(a.ctypes.data)
    d = lambda a: ctypes.c_void_p(a.data_ptr())
    n0 = t.launch_count()
    # each of the three buffers in turn on the host
    assert lib.tk_range_query_batch(t.h, 1, h(Q), d(od), None, d(outd), None, 0) == ARG
    assert lib.tk_range_query_batch(t.h, 1, d(rd), h(offs), None, d(outd), None, 0) == ARG
    assert lib.tk_range_query_batch(t.h, 1, d(rd), d(od), None, h(out), None, 0) == ARG
    assert lib.tk_range_query_batch_noalloc(t.h, 1, d(rd), d(od), None, h(out), None) == ARG
    assert lib.tk_stream_append(t.h, h(np.zeros(dims)), 0) == ARG
    assert lib.tk_range_query(t.h, 0, 8, None, h(out), None, 0) == ARG
    assert t.launch_count() == n0 and t.T == 32
    # the same call with device buffers runs
    assert lib.tk_range_query_batch(t.h, 1, d(rd), d(od), None, d(outd), None, 0) == 0
    t.sync()
    fresh = tk.Tree(dims, ranks, leaf_slices=4, dtype="f64")
    assert lib.tk_tree_build(fresh.h, h(np.ascontiguousarray(X)), 32, 0) == ARG
    assert fresh.T == 0
    fresh.close()
    t.close()
