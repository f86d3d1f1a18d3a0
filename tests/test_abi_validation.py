"""Host-side argument validation of the C ABI (include/tucket.h), called
through ctypes on a CPU host: every check here runs before the library
touches a device, so no GPU is needed.  A call that fails validation must
return its error code and change nothing."""
import ctypes

import pytest

import paper_2501_06647_gb300 as tk
from paper_2501_06647_gb300 import build as b

ARG, RANGE, RANK, CUDA = -1, -2, -3, -5


@pytest.fixture(scope="module")
def lib():
    b.build()
    return tk.lib()


def _cfg(lib, **kw):
    c = tk.TkConfig()
    assert lib.tk_config_default(ctypes.byref(c)) == 0
    c.dims[1], c.dims[2] = 30, 20
    for k, v in kw.items():
        if k == "ranks0":
            c.ranks[0] = v
        elif k == "dims1":
            c.dims[1] = v
        else:
            setattr(c, k, v)
    return c


def test_defaults_follow_the_paper(lib):
    c = tk.TkConfig()
    assert lib.tk_config_default(ctypes.byref(c)) == 0
    # Section 8.1: at most 20 ALS iterations, tolerance 0.01, theta = 0.7
    assert (c.p, c.max_iter, c.theta_num, c.theta_den, c.leaf_slices) == (3, 20, 7, 10, 1)
    assert abs(c.tol - 0.01) < 1e-15 and c.dtype == tk.TK_F32 and list(c.ranks[:3]) == [10, 10, 10]
    assert lib.tk_config_default(None) == ARG


@pytest.mark.parametrize("bad", [dict(p=1), dict(p=7), dict(leaf_slices=0), dict(theta_num=8, theta_den=7),
                                 dict(theta_den=0), dict(theta_num=0), dict(max_iter=0), dict(dtype=5),
                                 dict(ranks0=0), dict(ranks0=5000), dict(dims1=0)])
def test_invalid_configurations_are_rejected(lib, bad):
    c = _cfg(lib, **bad)
    h = ctypes.c_void_p(1234)
    assert lib.tk_tree_create(ctypes.byref(c), None, ctypes.byref(h)) == ARG
    assert h.value is None  # *out cleared, nothing created


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.tk_tree_create(None, None, ctypes.byref(h)) == ARG
    c = _cfg(lib)
    assert lib.tk_tree_create(ctypes.byref(c), None, None) == ARG
    assert lib.tk_sync(None) == ARG
    assert lib.tk_tree_build(None, None, 10, 0) == ARG
    assert lib.tk_stream_append(None, None, 0) == ARG
    assert lib.tk_range_query(None, 0, 1, None, None, None, 0) == ARG
    assert lib.tk_range_query_batch(None, 1, None, None, None, None, None, 0) == ARG
    assert lib.tk_range_query_batch_noalloc(None, 1, None, None, None, None, None) == ARG
    assert lib.tk_batch_layout(None, 1, None, None, None) == ARG
    assert lib.tk_hit_set(None, 0, 1, None, 1, None) == ARG
    assert lib.tk_timespan(None) < 0 and lib.tk_arena_bytes(None) < 0
    sh = ctypes.c_void_p()
    assert lib.tk_server_create(None, None, ctypes.byref(sh)) == ARG
    assert lib.tk_server_submit_query(None, 0, 1, None, None, None, None) == ARG
    assert lib.tk_server_submit_append(None, None, None) == ARG
    assert lib.tk_server_wait(None, 1, 0.0) == ARG
    assert lib.tk_server_drain(None, 0.0) == ARG
    lib.tk_tree_destroy(None)   # no-ops
    lib.tk_server_destroy(None)


def test_every_status_has_a_message(lib):
    msgs = [lib.tk_strerror(code) for code in range(0, -10, -1)]
    assert all(m for m in msgs) and len(set(msgs)) == len(msgs)


def test_valid_configuration_without_a_device_reports_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: creation would succeed")
    b.build()
    lib = tk.lib()
    c = _cfg(lib)
    h = ctypes.c_void_p()
    assert lib.tk_tree_create(ctypes.byref(c), None, ctypes.byref(h)) == CUDA
    assert h.value is None
