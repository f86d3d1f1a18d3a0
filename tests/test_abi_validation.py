"""Host-side argument validation of the C ABI (include/tucket.h), called
through ctypes on a CPU host: every check here runs before the library
touches a device, so no GPU is needed.  A call that fails validation must
return its error code and change nothing."""
import ctypes
import os

import pytest

import paper_2501_06647_gb300 as tk
from paper_2501_06647_gb300 import build as b

ARG, RANGE, RANK, CUDA, IO = -1, -2, -3, -5, -10


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
    assert c.hbm_budget == 0  # no memory budget
    assert lib.tk_config_default(None) == ARG


@pytest.mark.parametrize("bad", [dict(p=1), dict(p=9), dict(leaf_slices=0), dict(theta_num=8, theta_den=7),
                                 dict(theta_den=0), dict(theta_num=0), dict(max_iter=0), dict(dtype=5),
                                 dict(ranks0=0), dict(ranks0=5000), dict(dims1=0), dict(hbm_budget=-1),
                                 dict(math=-1), dict(math=3), dict(math=2, dtype=0),
                                 dict(eig_fp64=2), dict(eig_fp64=-1), dict(init=2), dict(init=-1)])
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
    v = ctypes.c_int(-7)
    assert lib.tk_batch_set_heavy_hits(None, 4) == ARG
    assert lib.tk_batch_get_heavy_hits(None, ctypes.byref(v)) == ARG and v.value == -7
    assert lib.tk_batch_tune(None, 2, None, None, None, None, 1, ctypes.byref(v), None) == ARG
    assert lib.tk_timespan(None) < 0 and lib.tk_arena_bytes(None) < 0
    sh = ctypes.c_void_p()
    assert lib.tk_server_create(None, None, ctypes.byref(sh)) == ARG
    assert lib.tk_server_submit_query(None, 0, 1, None, None, None, None) == ARG
    assert lib.tk_server_submit_append(None, None, None) == ARG
    assert lib.tk_server_wait(None, 1, 0.0) == ARG
    assert lib.tk_server_drain(None, 0.0) == ARG
    assert lib.tk_tree_save(None, b"x") == ARG
    assert lib.tk_tree_load(None, -1, None, ctypes.byref(sh)) == ARG
    assert lib.tk_tree_load(b"x", -1, None, None) == ARG
    lib.tk_tree_destroy(None)   # no-ops
    lib.tk_server_destroy(None)


def test_every_status_has_a_message(lib):
    msgs = [lib.tk_strerror(code) for code in range(0, -11, -1)]
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


class _FileHeader(ctypes.Structure):
    """The fixed header of a tree file, as tk_tree_save writes it."""
    _fields_ = [("magic", ctypes.c_char * 8), ("header_bytes", ctypes.c_uint32), ("elem_bytes", ctypes.c_uint32),
                ("cfg", tk.TkConfig), ("T", ctypes.c_int64), ("nb", ctypes.c_int64), ("nbcap", ctypes.c_int64),
                ("tail_dirty", ctypes.c_int32), ("nsec", ctypes.c_int32),
                ("sec_bytes", ctypes.c_int64 * (4 + tk.MAX_MODES))]


def _header(lib, magic=b"TKTREE\x00\x03", **kw):
    h = _FileHeader()
    h.header_bytes = ctypes.sizeof(_FileHeader)
    h.cfg = _cfg(lib, leaf_slices=4)
    h.elem_bytes = 4
    h.T, h.nb, h.nbcap, h.tail_dirty, h.nsec = 50, 12, 16, 1, 4 + tk.MAX_MODES
    for k, v in kw.items():
        setattr(h, k, v)
    # (a c_char array field stops copying at the first NUL: set the magic bytes directly)
    return magic + bytes(h)[8:]


def _load(lib, path):
    h = ctypes.c_void_p(1234)
    rc = lib.tk_tree_load(os.fsencode(path), -1, None, ctypes.byref(h))
    assert h.value is None  # nothing returned on failure
    return rc


def test_files_that_are_not_tree_files_are_rejected(lib, tmp_path):
    """Checked from the header alone, before any device work."""
    assert _load(lib, tmp_path / "missing.tkt") == IO
    f = tmp_path / "bad.tkt"
    good = _header(lib)
    bad = [b"", b"not a tree file", good[:40],                      # empty, garbage, truncated header
           _header(lib, magic=b"TKTREE\x00\x02"),                  # another format version
           _header(lib, header_bytes=8), _header(lib, nsec=3),       # another header layout
           _header(lib, elem_bytes=8),                               # element size not the dtype's
           _header(lib, nb=11),                                      # nb != T / B
           _header(lib, nbcap=12), _header(lib, nbcap=8),            # capacity not a power of two / too small
           _header(lib, T=-1, nb=0), _header(lib, tail_dirty=2)]
    for content in bad:
        f.write_bytes(content)
        assert _load(lib, f) == IO, content[:16]


def test_a_plausible_header_reaches_tree_creation():
    """A header that passes every check goes on to create the tree: without a
    device that is where it stops, with TK_ERR_CUDA."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the load would go on to read the sections")
    import tempfile
    b.build()
    lib = tk.lib()
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "h.tkt")
        with open(f, "wb") as fh:
            fh.write(_header(lib))
        assert _load(lib, f) == CUDA
