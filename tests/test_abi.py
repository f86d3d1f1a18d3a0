"""The C-ABI library builds, loads without a GPU, and exports every function
that include/tucket.h declares (no compute calls: this runs on CPU hosts)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tucket.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tk_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tk_tree_create", "tk_tree_build", "tk_stream_append", "tk_range_query", "tk_range_query_batch",
                 "tk_hit_set", "tk_tree_destroy", "tk_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2501_06647_gb300 import build as b
    path = b.build()
    h = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(h, n)]
    assert not missing, missing
    import paper_2501_06647_gb300 as pkg
    assert set(_declared()) == set(pkg._SIGS)
    h.tk_strerror.restype = ctypes.c_char_p
    assert h.tk_strerror(-3) == b"query rank below 1 or above the build rank"
