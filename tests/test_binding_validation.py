"""The Python binding rejects buffers that the kernels cannot read before any
call into the library: host arrays or CPU tensors where device memory is
expected, another GPU's tensors, and wrong dtypes or shapes (int64 ranges and
offsets, the tree's float type for outputs and slices).  CPU only: the
tensors below are stand-ins that report CUDA placement, so no GPU is touched."""
import types

import numpy as np
import pytest

import paper_2501_06647_gb300 as tk


class FakeCuda:
    """Looks like a contiguous CUDA tensor to the binding's checks."""

    def __init__(self, shape, dtype, device=0, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = "torch." + dtype
        self.is_cuda = True
        self.device = types.SimpleNamespace(index=device)
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("validation must fail before the pointer is taken")


def _tree(dtype="f32", device=0):
    t = tk.Tree.__new__(tk.Tree)
    t.h = None
    t.dims, t.ranks, t.p = (7, 5), (3, 3, 3), 3
    t.dtype, t.np_dtype, t.device, t.B = dtype, np.float32 if dtype == "f32" else np.float64, device, 4
    return t


GOOD = dict(ranges=((4, 2), "int64"), offsets=((5,), "int64"), out=((100,), "float32"))


def _args(**over):
    spec = dict(GOOD)
    spec.update(over)
    return [FakeCuda(*spec[k]) if isinstance(spec[k], tuple) else spec[k] for k in ("ranges", "offsets", "out")]


@pytest.mark.parametrize("method", ["query_batch", "query_batch_noalloc"])
@pytest.mark.parametrize("bad", [
    dict(ranges=np.zeros((4, 2), dtype=np.int64)),          # host array
    dict(ranges=((4, 2), "int32")),                          # wrong index type
    dict(ranges=((8,), "int64")),                            # not (n, 2)
    dict(offsets=((4,), "int64")),                           # not n + 1 entries
    dict(offsets=((5,), "float64")),
    dict(out=((100,), "float64")),                           # not the tree's dtype
    dict(out=((10, 10), "float32")),                         # not flat
])
def test_batch_rejects_unreadable_buffers(method, bad):
    t = _tree()
    with pytest.raises(ValueError):
        getattr(t, method)(*_args(**bad))


def test_batch_rejects_another_gpu_and_strided_tensors():
    t = _tree(device=1)
    with pytest.raises(ValueError, match="cuda:1"):
        t.query_batch(*_args())
    t = _tree()
    r, o, out = _args()
    out._c = False
    with pytest.raises(ValueError, match="contiguous"):
        t.query_batch(r, o, out)


def test_build_and_append_check_device_tensors():
    t = _tree("f64")
    with pytest.raises(ValueError):
        t.build(FakeCuda((16, 7, 5), "float32"))              # f32 data for an f64 tree
    with pytest.raises(ValueError):
        t.build(FakeCuda((16, 5, 7), "float64"))              # slices of the wrong shape
    with pytest.raises(ValueError):
        t.append(FakeCuda((7, 5), "float64", device=2))


def test_start_of_stitch_is_checked_before_creation():
    # an unknown start raises before the library creates anything (no GPU needed)
    with pytest.raises(ValueError):
        tk.Tree((7, 5), (3, 3, 3), leaf_slices=4, init="hosvd-ish")
    assert tk.INIT == {"hosvd": 0, "random": 1}
