"""Python binding of the GB300 range-query Tucker engine (TUCKET, arXiv 2501.06647).

Argument marshalling only: every step of tree build, stream update and range
query runs in the CUDA kernels of ``libtucket.so`` (built in-tree by
``build.py``) behind the C ABI of ``include/tucket.h``.  PyTorch is used for
device buffers and streams.  There is no CPU fallback: if the library is
missing, importing ``lib()`` raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtucket.so")
MAX_MODES = 8

TK_F64, TK_F32 = 0, 1
MATH = {"auto": 0, "cuda_cores": 1, "tf32": 2}
INIT = {"hosvd": 0, "random": 1}
TK_IO_DEVICE, TK_IO_HOST = 0, 1

_ERR = {
    -1: "invalid argument", -2: "time range outside [0, T) or empty", -3: "query rank out of bounds",
    -4: "device allocation failed", -5: "CUDA runtime error", -6: "invalid tree state",
    -7: "device job exceeded its workspace", -8: "request exceeds an engine limit",
    -9: "a wait ran out of time",
    -10: "tree file could not be read or written, or is not a tree file",
}


class TkConfig(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("dims", ctypes.c_int64 * MAX_MODES),
                ("ranks", ctypes.c_int32 * MAX_MODES), ("leaf_slices", ctypes.c_int32),
                ("theta_num", ctypes.c_int32), ("theta_den", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("dtype", ctypes.c_int32),
                ("device", ctypes.c_int32), ("hbm_budget", ctypes.c_int64), ("math", ctypes.c_int32),
                ("eig_fp64", ctypes.c_int32), ("seed", ctypes.c_uint64), ("init", ctypes.c_int32)]


class TkHit(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("partial", ctypes.c_int32), ("index", ctypes.c_int64),
                ("node_lo", ctypes.c_int64), ("node_hi", ctypes.c_int64), ("lo", ctypes.c_int64),
                ("hi", ctypes.c_int64)]


class TkQueryInfo(ctypes.Structure):
    _fields_ = [("ranks", ctypes.c_int32 * MAX_MODES), ("iters", ctypes.c_int32),
                ("n_hits", ctypes.c_int32), ("fit_err", ctypes.c_double), ("eig_sweeps", ctypes.c_int32),
                ("eig_max_order", ctypes.c_int32), ("device_cycles", ctypes.c_int64),
                ("eig_cycles", ctypes.c_int64), ("qr_cycles", ctypes.c_int64),
                ("hit_cycles", ctypes.c_int64), ("init_cycles", ctypes.c_int64),
                ("als_cycles", ctypes.c_int64), ("out_cycles", ctypes.c_int64),
                ("start_ns", ctypes.c_int64), ("end_ns", ctypes.c_int64)]


class TkServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_batch_out_elems", ctypes.c_int64)]


class TkServerStats(ctypes.Structure):
    _fields_ = [("queries_done", ctypes.c_int64), ("appends_done", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
                ("elapsed_s", ctypes.c_double)]


# Every symbol the header declares, with its ctypes signature.
_SIGS = {
    "tk_config_default": (ctypes.c_int, [ctypes.POINTER(TkConfig)]),
    "tk_tree_create": (ctypes.c_int, [ctypes.POINTER(TkConfig), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "tk_tree_destroy": (None, [ctypes.c_void_p]),
    "tk_tree_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]),
    "tk_stream_append": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tk_timespan": (ctypes.c_int64, [ctypes.c_void_p]),
    "tk_hit_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(TkHit),
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "tk_query_output_elems": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]),
    "tk_range_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.POINTER(TkQueryInfo), ctypes.c_int]),
    "tk_batch_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "tk_range_query_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tk_node_payload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p]),
    "tk_arena_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "tk_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "tk_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "tk_batch_set_heavy_hits": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tk_batch_get_heavy_hits": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "tk_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_float)]),
    "tk_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tk_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "tk_range_query_batch_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p]),
    "tk_tree_get_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TkConfig)]),
    "tk_tree_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "tk_tree_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "tk_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TkServerConfig),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tk_server_submit_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "tk_server_submit_append": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "tk_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double]),
    "tk_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "tk_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TkServerStats)]),
    "tk_server_destroy": (None, [ctypes.c_void_p]),
}

_lib_handle = None


def lib():
    """Load libtucket.so from the source tree (raises if it was not built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2501_06647_gb300/build.py (no CPU fallback)")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib_handle = h
    return _lib_handle


class TuckerError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_ERR.get(code, 'error')} ({code})")
        self.code = code


def _check(rc, what):
    if rc != 0:
        raise TuckerError(rc, what)


def _np_dtype(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _device_tensor(x, name, device, dtype=None, shape=None):
    """Check that x is a contiguous CUDA tensor on `device` (torch dtype name
    `dtype`, e.g. "int64", and shape `shape` where given): the kernels read
    it directly, so a host buffer or another GPU's would fault."""
    if not (hasattr(x, "is_cuda") and x.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor on cuda:{device}")
    if x.device.index != device:
        raise ValueError(f"{name} is on {x.device}, the tree is on cuda:{device}")
    if dtype is not None and str(x.dtype) != "torch." + dtype:
        raise ValueError(f"{name} must have dtype {dtype}, not {x.dtype}")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(x.shape)}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _ptr(x):
    """Address of a torch tensor or numpy array (contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def fma_rate(dtype="f32", device=0):
    """Measured FMA throughput of the device in FLOP/s (tk_probe_fma_rate)."""
    v = ctypes.c_double()
    _check(lib().tk_probe_fma_rate(TK_F64 if dtype == "f64" else TK_F32, int(device), ctypes.byref(v)),
           "tk_probe_fma_rate")
    return v.value


class Tree:
    """A stream segment tree on one GPU (Section 4.2 of the paper).

    dims are the non-temporal sizes D_2..D_p, ranks the build ranks r_1..r_p,
    leaf_slices the slices per leaf block, theta the pruning threshold as a
    fraction (num, den), dtype "f64" or "f32", hbm_budget the device bytes the
    tree may hold (0: no limit), math the arithmetic of the leaf Grams ("auto":
    split-TF32 tensor cores for FP32 trees, "cuda_cores", or "tf32"), eig_fp64
    whether an FP32 tree solves its stitch eigenproblems in FP64, init the
    start of Stitch ("hosvd", or "random" drawn from seed).
    """

    def __init__(self, dims, ranks, leaf_slices=1, theta=(7, 10), max_iter=20, tol=0.01, dtype="f32",
                 device=0, stream=None, hbm_budget=0, math="auto", eig_fp64=False, init="hosvd", seed=0):
        self.dims = tuple(int(d) for d in dims)
        self.ranks = tuple(int(r) for r in ranks)
        self.p = len(self.ranks)
        if len(self.dims) != self.p - 1:
            raise ValueError("need len(dims) == len(ranks) - 1")
        self.dtype = dtype
        self.np_dtype = _np_dtype(dtype)
        cfg = TkConfig()
        lib().tk_config_default(ctypes.byref(cfg))
        cfg.p = self.p
        for n, d in enumerate(self.dims):
            cfg.dims[n + 1] = d
        for n, r in enumerate(self.ranks):
            cfg.ranks[n] = r
        cfg.leaf_slices = int(leaf_slices)
        cfg.theta_num, cfg.theta_den = int(theta[0]), int(theta[1])
        cfg.max_iter = int(max_iter)
        cfg.tol = float(tol)
        cfg.dtype = TK_F64 if dtype == "f64" else TK_F32
        cfg.device = int(device)
        cfg.hbm_budget = int(hbm_budget)
        cfg.math = MATH[math]
        cfg.eig_fp64 = 1 if eig_fp64 else 0
        if init not in INIT:
            raise ValueError(f"init must be one of {sorted(INIT)}")
        cfg.init = INIT[init]
        cfg.seed = int(seed) & ((1 << 64) - 1)
        self.cfg = cfg
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
        _check(lib().tk_tree_create(ctypes.byref(cfg), s, ctypes.byref(h)), "tk_tree_create")
        self.h = h
        self.B = int(leaf_slices)
        self.device = int(device)
        self._stream = stream

    def save(self, path):
        """Write the tree to a file (tk_tree_save; synchronous)."""
        _check(lib().tk_tree_save(self.h, os.fsencode(path)), "tk_tree_save")

    @classmethod
    def load(cls, path, device=None, stream=None):
        """A tree read from a file written by save() (tk_tree_load), on `device`
        (default: the device recorded in the file)."""
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
        _check(lib().tk_tree_load(os.fsencode(path), -1 if device is None else int(device), s, ctypes.byref(h)),
               "tk_tree_load")
        self = cls.__new__(cls)
        self.h = h
        cfg = TkConfig()
        _check(lib().tk_tree_get_config(h, ctypes.byref(cfg)), "tk_tree_get_config")
        self.cfg = cfg
        self.p = int(cfg.p)
        self.dims = tuple(int(cfg.dims[n]) for n in range(1, self.p))
        self.ranks = tuple(int(cfg.ranks[n]) for n in range(self.p))
        self.dtype = "f64" if cfg.dtype == TK_F64 else "f32"
        self.np_dtype = _np_dtype(self.dtype)
        self.B = int(cfg.leaf_slices)
        self.device = int(cfg.device)
        self._stream = stream
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().tk_tree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- updates ---------------------------------------------------------
    def build(self, X):
        """tree_build over X (T x D_2 x ... ; torch CUDA tensor or host numpy array)."""
        io = TK_IO_DEVICE if hasattr(X, "is_cuda") and X.is_cuda else TK_IO_HOST
        if io == TK_IO_HOST:
            X = np.ascontiguousarray(X, dtype=self.np_dtype)
        else:
            _device_tensor(X, "X", self.device, self._torch_dtype(), (X.shape[0],) + self.dims)
        f = self._before(io == TK_IO_DEVICE)
        _check(lib().tk_tree_build(self.h, _ptr(X), int(X.shape[0]), io), "tk_tree_build")
        self._after(f)

    def append(self, X_T):
        """stream update with one slice (torch CUDA tensor or host numpy array)."""
        io = TK_IO_DEVICE if hasattr(X_T, "is_cuda") and X_T.is_cuda else TK_IO_HOST
        if io == TK_IO_HOST:
            X_T = np.ascontiguousarray(X_T, dtype=self.np_dtype)
        else:
            _device_tensor(X_T, "X_T", self.device, self._torch_dtype(), self.dims)
        f = self._before(io == TK_IO_DEVICE)
        _check(lib().tk_stream_append(self.h, _ptr(X_T), io), "tk_stream_append")
        self._after(f)

    # Stream ordering of device tensors.  The engine launches on the tree's
    # stream.  When that is torch's current stream, calls are asynchronous and
    # ordered like torch's own kernels (the caching allocator does not reuse a
    # freed tensor's memory before the stream reaches that point).  Otherwise
    # (a tree with a stream of its own, or another current stream) a call
    # first waits for torch's current stream, so that its inputs are written,
    # and then for the tree's stream, so that the caller may free or reuse its
    # tensors as soon as the call returns.
    def _foreign_stream(self):
        import torch
        if self._stream is None:
            return True
        return torch.cuda.current_stream(self.device).cuda_stream != self._stream.cuda_stream

    def _before(self, device_io):
        foreign = device_io and self._foreign_stream()
        if foreign:
            import torch
            torch.cuda.current_stream(self.device).synchronize()
        return foreign

    def _after(self, foreign):
        if foreign:
            self.sync()

    def _torch_dtype(self):
        return "float64" if self.dtype == "f64" else "float32"

    def _check_batch_args(self, ranges, offsets, out):
        n = int(ranges.shape[0]) if hasattr(ranges, "shape") and len(ranges.shape) == 2 else -1
        _device_tensor(ranges, "ranges", self.device, "int64", (max(n, 0), 2))
        _device_tensor(offsets, "offsets", self.device, "int64", (n + 1,))
        _device_tensor(out, "out", self.device, self._torch_dtype())
        if len(out.shape) != 1:
            raise ValueError("out must be one-dimensional")
        return n

    @property
    def T(self):
        return int(lib().tk_timespan(self.h))

    def sync(self):
        _check(lib().tk_sync(self.h), "tk_sync")

    def launch_count(self):
        return int(lib().tk_launch_count(self.h))

    def arena_bytes(self):
        return int(lib().tk_arena_bytes(self.h))

    @property
    def heavy_hits(self):
        """Hit count from which a batched query runs on a whole CTA."""
        v = ctypes.c_int(0)
        _check(lib().tk_batch_get_heavy_hits(self.h, ctypes.byref(v)), "tk_batch_get_heavy_hits")
        return int(v.value)

    @heavy_hits.setter
    def heavy_hits(self, hits):
        _check(lib().tk_batch_set_heavy_hits(self.h, int(hits)), "tk_batch_set_heavy_hits")

    # ---- queries ---------------------------------------------------------
    def hit_set(self, ts, te):
        """Algorithm 1's hit set as (level, index, node_lo, node_hi, lo, hi, partial) tuples."""
        cap = 64
        arr = (TkHit * cap)()
        n = ctypes.c_int()
        _check(lib().tk_hit_set(self.h, int(ts), int(te), arr, cap, ctypes.byref(n)), "tk_hit_set")
        return [(h.level, h.index, h.node_lo, h.node_hi, h.lo, h.hi, h.partial) for h in arr[: n.value]]

    def _ranks_arg(self, ranks):
        if ranks is None:
            return None, self.ranks
        arr = (ctypes.c_int32 * MAX_MODES)(*([int(r) for r in ranks] + [1] * (MAX_MODES - len(ranks))))
        return arr, tuple(int(r) for r in ranks)

    def unpack(self, flat, L, ranks=None):
        """Split one packed query output into (G, [U1, U2, ...]) views."""
        rq = self.ranks if ranks is None else tuple(ranks)
        c = int(np.prod(rq))
        G = flat[:c].reshape(rq)
        off = c
        U = [flat[off:off + L * rq[0]].reshape(L, rq[0])]
        off += L * rq[0]
        for n in range(1, self.p):
            U.append(flat[off:off + self.dims[n - 1] * rq[n]].reshape(self.dims[n - 1], rq[n]))
            off += self.dims[n - 1] * rq[n]
        return G, U

    def query(self, ts, te, ranks=None):
        """Range query through the C ABI with host buffers: returns (G, U, info)."""
        rarr, rq = self._ranks_arg(ranks)
        n = int(lib().tk_query_output_elems(self.h, int(ts), int(te), rarr))
        if n < 0:
            _check(n, "tk_query_output_elems")
        out = np.zeros(n, dtype=self.np_dtype)
        info = TkQueryInfo()
        _check(lib().tk_range_query(self.h, int(ts), int(te), rarr, _ptr(out), ctypes.byref(info), TK_IO_HOST),
               "tk_range_query")
        G, U = self.unpack(out, int(te) - int(ts), rq)
        r = list(info.ranks[: self.p])
        G = G[tuple(slice(0, x) for x in r)]
        U = [u[:, :x] for u, x in zip(U, r)]
        return G, U, dict(ranks=r, iters=info.iters, n_hits=info.n_hits, fit_err=info.fit_err,
                          eig_sweeps=info.eig_sweeps, eig_max_order=info.eig_max_order,
                          device_cycles=info.device_cycles, eig_cycles=info.eig_cycles,
                          qr_cycles=info.qr_cycles)

    def layout(self, ranges, ranks=None):
        ranges = np.ascontiguousarray(ranges, dtype=np.int64).reshape(-1, 2)
        rarr, _ = self._ranks_arg(ranks)
        offs = np.zeros(len(ranges) + 1, dtype=np.int64)
        _check(lib().tk_batch_layout(self.h, len(ranges), _ptr(ranges), rarr, _ptr(offs)), "tk_batch_layout")
        return offs

    def query_batch(self, ranges, offsets, out, ranks=None, info=None):
        """Batched range queries, all buffers on the device (asynchronous).

        ranges: int64 tensor (n, 2); offsets: int64 tensor (n+1); out: tensor
        of offsets[-1] elements of the tree's dtype.  info: optional host
        array of TkQueryInfo (makes the call synchronous).  Asynchronous
        only when torch's current stream is the tree's (see _foreign_stream).
        """
        n = self._check_batch_args(ranges, offsets, out)
        rarr, _ = self._ranks_arg(ranks)
        ip = ctypes.cast(info, ctypes.c_void_p) if info is not None else None
        f = self._before(True)
        _check(lib().tk_range_query_batch(self.h, n, _ptr(ranges), _ptr(offsets), rarr, _ptr(out), ip,
                                          TK_IO_DEVICE), "tk_range_query_batch")
        self._after(f)

    def tune_batch(self, ranges, offsets, out, ranks=None, reps=2):
        """Autotune the batch launch shape on this batch (tk_batch_tune):
        returns (heavy_hits, best_ms) and keeps that threshold.  Synchronous;
        overwrites out."""
        n = self._check_batch_args(ranges, offsets, out)
        rarr, _ = self._ranks_arg(ranks)
        best, ms = ctypes.c_int(0), ctypes.c_float(0.0)
        self._before(True)
        _check(lib().tk_batch_tune(self.h, n, _ptr(ranges), _ptr(offsets), rarr, _ptr(out), int(reps),
                                   ctypes.byref(best), ctypes.byref(ms)), "tk_batch_tune")
        return int(best.value), float(ms.value)

    def query_batch_noalloc(self, ranges, offsets, out, ranks=None, info=None):
        """Batched range queries that make no device allocation (device buffers).

        Same results as query_batch; the engine's scratch is a fixed 16 MiB
        device array shared by all such calls (serialize overlapping calls).
        """
        n = self._check_batch_args(ranges, offsets, out)
        rarr, _ = self._ranks_arg(ranks)
        ip = ctypes.cast(info, ctypes.c_void_p) if info is not None else None
        f = self._before(True)
        _check(lib().tk_range_query_batch_noalloc(self.h, n, _ptr(ranges), _ptr(offsets),
                                                  rarr, _ptr(out), ip), "tk_range_query_batch_noalloc")
        self._after(f)

    def query_batch_host(self, ranges, offsets=None, out=None, ranks=None, with_info=True):
        """Batched range queries through the C ABI with HOST buffers (copies inside the call)."""
        ranges = np.ascontiguousarray(ranges, dtype=np.int64).reshape(-1, 2)
        if offsets is None:
            offsets = self.layout(ranges, ranks)
        if out is None:
            out = np.zeros(int(offsets[-1]), dtype=self.np_dtype)
        rarr, _ = self._ranks_arg(ranks)
        info = (TkQueryInfo * len(ranges))() if with_info else None
        ip = ctypes.cast(info, ctypes.c_void_p) if info is not None else None
        _check(lib().tk_range_query_batch(self.h, len(ranges), _ptr(ranges), _ptr(offsets), rarr, _ptr(out), ip,
                                          TK_IO_HOST), "tk_range_query_batch")
        return out, offsets, info

    def node_payload(self, level, index):
        """A stored node's (H, [V1, V2, ...], ranks), trimmed to its logical ranks."""
        B = self.B
        lo = (int(index) << int(level)) * B
        hi = min(lo + (1 << int(level)) * B, self.T)
        n = int(lib().tk_query_output_elems(self.h, 0, hi - lo, None))
        out = np.zeros(n, dtype=self.np_dtype)
        rk = (ctypes.c_int32 * MAX_MODES)()
        _check(lib().tk_node_payload(self.h, int(level), int(index), _ptr(out), n, rk), "tk_node_payload")
        G, U = self.unpack(out, hi - lo)
        r = list(rk[: self.p])
        return G[tuple(slice(0, x) for x in r)], [u[:, :x] for u, x in zip(U, r)], r


class Server:
    """Continuous-batching server over one Tree (native worker thread).

    Queries and stream updates submitted from any thread run in submission
    order; queries waiting together are batched into one launch.  The tree
    must not be used directly while the server exists.
    """

    def __init__(self, tree, max_batch=1024, max_batch_out_elems=16 << 20):
        self.tree = tree
        cfg = TkServerConfig(int(max_batch), int(max_batch_out_elems))
        h = ctypes.c_void_p()
        _check(lib().tk_server_create(tree.h, ctypes.byref(cfg), ctypes.byref(h)), "tk_server_create")
        self.h = h
        self._live = {}  # ticket -> host buffers the worker writes into

    def submit_query(self, ts, te, ranks=None):
        """Queue a range query; returns its ticket."""
        rarr, rq = self.tree._ranks_arg(ranks)
        L = int(te) - int(ts)
        n = int(np.prod(rq)) + L * rq[0] + sum(d * r for d, r in zip(self.tree.dims, rq[1:]))
        out = np.empty(max(n, 1), dtype=self.tree.np_dtype)
        info = TkQueryInfo()
        tk = ctypes.c_uint64()
        _check(lib().tk_server_submit_query(self.h, int(ts), int(te), rarr, _ptr(out), ctypes.byref(info),
                                            ctypes.byref(tk)), "tk_server_submit_query")
        self._live[tk.value] = (out, info, L, rq)
        return tk.value

    def submit_append(self, X_T):
        """Queue a stream update with one host slice; returns its ticket."""
        X_T = np.ascontiguousarray(X_T, dtype=self.tree.np_dtype)
        tk = ctypes.c_uint64()
        _check(lib().tk_server_submit_append(self.h, _ptr(X_T), ctypes.byref(tk)), "tk_server_submit_append")
        return tk.value

    def wait(self, ticket, timeout=-1.0):
        """Wait for a request: a query gives (G, U, info), an append None."""
        _check(lib().tk_server_wait(self.h, int(ticket), float(timeout)), "tk_server_wait")
        rec = self._live.pop(int(ticket), None)
        if rec is None:
            return None
        out, info, L, rq = rec
        G, U = self.tree.unpack(out, L, rq)
        r = list(info.ranks[: self.tree.p])
        return (G[tuple(slice(0, x) for x in r)], [u[:, :x] for u, x in zip(U, r)],
                dict(ranks=r, iters=info.iters, n_hits=info.n_hits, fit_err=info.fit_err))

    def drain(self, timeout=-1.0):
        _check(lib().tk_server_drain(self.h, float(timeout)), "tk_server_drain")

    def stats(self):
        st = TkServerStats()
        _check(lib().tk_server_get_stats(self.h, ctypes.byref(st)), "tk_server_get_stats")
        return {k: getattr(st, k) for k, _ in TkServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().tk_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
