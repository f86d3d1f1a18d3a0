"""Seeded synthetic inputs shared by the oracle checks and the CUDA engine's tests.

This module only draws random numbers and assembles inputs; it contains none
of the method's arithmetic (no decomposition, stitching or tree logic).

Series: a piecewise Tucker tensor time series of shape T x D_2 x ... x D_p,
standing in for the paper's 3-way datasets (Section 8.1; the datasets are not
used).  Each regime of ``regime`` slices draws, in this order from one
``numpy.random.Generator(PCG64(seed))``: a core with N(0,1) entries of shape
r_1 x ... x r_p, a temporal factor (Q of a Gaussian l x r_1 matrix), and
non-temporal factors (Q of Gaussian D_n x r_n matrices); the regime's slab is
core x_1 A x_2 B ... (the generator's own einsum), scaled so that the signal
has unit RMS per entry (``unit_signal``) unless ``literal_scale`` is set.
Finally i.i.d. N(0, sigma^2) noise is added, slab by slab, from the same
generator.

Streaming series (``piecewise_tucker_regimes``): the same recipe, but each
regime draws from its own generator, spawned from ``SeedSequence(seed)``, and
adds its own noise; regimes are generated in parallel threads straight into a
float32 array.  It stands in for the long 4-way streams of the serving runs,
where one generator over the whole series would be too slow.

Device series (``piecewise_tucker_device``): the same recipe drawn on a CUDA
device by one seeded ``torch.Generator``, for the 8 GB large workload; the
engine's benchmark alone uses it (no oracle comparison runs at that size).

Query ranges: "uniform" draws two distinct integers of {0..T}, sorted, read
as the half-open range [a, b); "loguniform" draws L = round(exp(U[ln lo,
ln hi])) and t_s uniformly from {0..T-L}.
"""
import string

import numpy as np


def _orthonormal(rng, m, r):
    Q, _ = np.linalg.qr(rng.standard_normal((m, r)))
    return Q[:, :r]


def piecewise_tucker(T, dims, ranks, regime, sigma, seed, literal_scale=False, dtype=np.float64):
    """Seeded piecewise-Tucker series (see module docstring)."""
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    p = len(ranks)
    assert len(dims) == p - 1
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    X = np.empty((int(T),) + dims, dtype=np.float64)
    letters = string.ascii_lowercase
    core_idx = letters[:p]
    out_idx = letters[13:13 + p]
    for start in range(0, int(T), int(regime)):
        l = min(int(regime), int(T) - start)
        rr = [min(ranks[0], l)] + [min(r, d) for r, d in zip(ranks[1:], dims)]
        core = rng.standard_normal(tuple(rr))
        if not literal_scale:
            core *= np.sqrt(l * np.prod(dims) / np.prod(rr))
        facs = [_orthonormal(rng, l, rr[0])] + [_orthonormal(rng, d, r) for d, r in zip(dims, rr[1:])]
        spec = core_idx + "," + ",".join(out_idx[n] + core_idx[n] for n in range(p)) + "->" + out_idx
        X[start:start + l] = np.einsum(spec, core, *facs, optimize=True)
    for start in range(0, int(T), int(regime)):
        l = min(int(regime), int(T) - start)
        X[start:start + l] += sigma * rng.standard_normal((l,) + dims)
    return X.astype(dtype, copy=False)


def _regime(X, start, l, dims, ranks, sigma, ss, literal_scale):
    rng = np.random.Generator(np.random.PCG64(ss))
    p = len(ranks)
    letters = string.ascii_lowercase
    core_idx, out_idx = letters[:p], letters[13:13 + p]
    rr = [min(ranks[0], l)] + [min(r, d) for r, d in zip(ranks[1:], dims)]
    core = rng.standard_normal(tuple(rr))
    if not literal_scale:
        core *= np.sqrt(l * np.prod(dims) / np.prod(rr))
    facs = [_orthonormal(rng, l, rr[0])] + [_orthonormal(rng, d, r) for d, r in zip(dims, rr[1:])]
    spec = core_idx + "," + ",".join(out_idx[n] + core_idx[n] for n in range(p)) + "->" + out_idx
    for i in range(0, l, 64):  # slab by slab, to bound the float64 temporaries
        j = min(l, i + 64)
        sig = np.einsum(spec, core, facs[0][i:j], *facs[1:], optimize=True)
        X[start + i:start + j] = sig + sigma * rng.standard_normal(sig.shape)


def piecewise_tucker_regimes(T, dims, ranks, regime, sigma, seed, literal_scale=False, threads=8):
    """Seeded piecewise-Tucker series in float32, one generator per regime."""
    from concurrent.futures import ThreadPoolExecutor
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    assert len(dims) == len(ranks) - 1
    T, regime = int(T), int(regime)
    X = np.empty((T,) + dims, dtype=np.float32)
    starts = list(range(0, T, regime))
    seeds = np.random.SeedSequence(int(seed)).spawn(len(starts))
    with ThreadPoolExecutor(max_workers=max(1, int(threads))) as ex:
        futs = [ex.submit(_regime, X, s0, min(regime, T - s0), dims, ranks, sigma, ss, literal_scale)
                for s0, ss in zip(starts, seeds)]
        for f in futs:
            f.result()
    return X


def piecewise_tucker_device(T, dims, ranks, regime, sigma, seed, device):
    """Seeded piecewise-Tucker series drawn on a CUDA device, in float32 (the
    8 GB series of the large workload would take minutes on the host).  Same
    recipe as ``piecewise_tucker`` (per regime: N(0,1) core scaled to unit
    signal RMS, temporal and non-temporal factors as Q of Gaussian matrices,
    then N(0, sigma^2) noise), drawn in that order per regime from one
    ``torch.Generator`` on the device seeded with ``seed``; the values differ
    from the NumPy generators'."""
    import torch
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    p = len(ranks)
    assert len(dims) == p - 1
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    X = torch.empty((int(T),) + dims, dtype=torch.float32, device=device)
    letters = string.ascii_lowercase
    core_idx, out_idx = letters[:p], letters[13:13 + p]
    spec = core_idx + "," + ",".join(out_idx[n] + core_idx[n] for n in range(p)) + "->" + out_idx
    for start in range(0, int(T), int(regime)):
        l = min(int(regime), int(T) - start)
        rr = [min(ranks[0], l)] + [min(r, d) for r, d in zip(ranks[1:], dims)]
        core = torch.randn(tuple(rr), generator=g, device=device, dtype=torch.float64)
        core *= float(np.sqrt(l * np.prod(dims) / np.prod(rr)))
        facs = [torch.linalg.qr(torch.randn(m, r, generator=g, device=device, dtype=torch.float64))[0]
                for m, r in zip((l,) + dims, rr)]
        X[start:start + l] = torch.einsum(spec, core, *facs).to(torch.float32)
        X[start:start + l] += sigma * torch.randn((l,) + dims, generator=g, device=device, dtype=torch.float32)
    return X


def query_ranges(T, n, seed, kind="uniform", lo=16, hi=None):
    """n seeded query ranges [t_s, t_e) over a series of length T."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    T = int(T)
    out = np.empty((int(n), 2), dtype=np.int64)
    for i in range(int(n)):
        if kind == "uniform":
            a, b = rng.choice(T + 1, size=2, replace=False)
            out[i] = (min(a, b), max(a, b))
        elif kind == "loguniform":
            top = T if hi is None else min(int(hi), T)
            L = int(round(np.exp(rng.uniform(np.log(lo), np.log(top)))))
            L = max(1, min(L, T))
            ts = int(rng.integers(0, T - L + 1))
            out[i] = (ts, ts + L)
        else:
            raise ValueError(kind)
    return out


# Workloads with the shapes of the paper's 3-way series (Section 8.1) and the
# configurations the benchmark and the parity tests run.
WORKLOADS = {
    "fp64_small": dict(T=256, dims=(30, 20), ranks=(5, 5, 5), regime=64, sigma=0.01, B=4,
                       n_queries=100, kind="uniform", seed=1001, qseed=2001, dtype="f64"),
    "fp32_plain": dict(T=4096, dims=(100, 100), ranks=(10, 10, 10), regime=512, sigma=0.05, B=16,
                       n_queries=1000, kind="loguniform", lo=16, hi=4096, seed=1002, qseed=2002,
                       dtype="f32"),
    # Batched form at larger shapes: 200x150 slices, T = 8192, ranks 16, 10,000
    # concurrent queries of log-uniform length (generated regime by regime in
    # float32, like the serving stream).
    "batched_r16": dict(T=8192, dims=(200, 150), ranks=(16, 16, 16), regime=512, sigma=0.05, B=16,
                        n_queries=10000, kind="loguniform", lo=16, hi=8192, seed=1003, qseed=2003,
                        dtype="f32"),
    # 4-way stream grown by single-slice appends at append_hz while Poisson
    # range queries of log-uniform length (16..T) arrive at query_hz.
    # Large series: 500x500 slices, T = 8192 (8 GB in FP32), ranks 20, leaf 32,
    # noise 0.1, drawn on the device; log-uniform queries.
    "large_r20": dict(T=8192, dims=(500, 500), ranks=(20, 20, 20), regime=512, sigma=0.1, B=32,
                      n_queries=2000, kind="loguniform", lo=16, hi=8192, seed=1005, qseed=2005, dtype="f32"),
    "serving_4way": dict(T0=1024, T_end=16384, dims=(64, 64, 32), ranks=(8, 8, 8, 8), regime=512, sigma=0.05,
                         B=16, append_hz=1000.0, query_hz=5000.0, lo=16, seed=1004, qseed=2004, dtype="f32"),
}
