#!/usr/bin/env python3
"""Range-query throughput of the GPU engine on the batched rank-16 workload.

One step = one batched launch sequence answering the workload's 10,000
concurrent range queries (Recall, partial-hit QR, Stitch/HOOI in coefficient
space, factor assembly: every row of the hot path) over a tree already
resident in HBM: 200x150 slices, T = 8192, ranks (16,16,16), leaf 16, FP32.
Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The line also carries the one-query-per-launch (plain) method on the same
tree, in-batch p50/p99 latency, the end-to-end number through host buffers,
rooflines, the FP64 oracle on the host cores (cpu_baseline) and the
matched-error check, and sections for the FP32 plain workload (100x100,
rank 10), stream appends, serving and the leaf kernel.  --impl reference
times the FP64 CPU oracle (the literal restatement of the paper's
algorithms) on the host cores instead, on bounded samples of the same
workload.  Multi-GPU runs are replicas (every rank holds the tree and answers
its own copy of the batch; no collective on the data path).
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "range queries/sec + p50/p99 query latency at matched recon error vs plain"
UNIT = "queries/s"
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128   # FP32 FMA units per SM (Blackwell)
# DRAM bytes (read + write) of one k_batch launch answering the 10,000-query
# batch: one ncu capture of the current kernel on the workload's first 1000
# queries (123.3 MB read + 217.6 MB written, profiles/k_batch_batched_r16_full.md)
# scaled by the queries (None: not yet captured for this kernel version).
BATCH_DRAM_BYTES = 10 * (123.31e6 + 217.61e6)
ORACLE_T = 1024           # the CPU oracle's tree covers the first 1024 slices


def workload_desc(w, name):
    return (f"{name}: {w['dims'][0]}x{w['dims'][1]}xT={w['T']} piecewise Tucker rank-{tuple(w['ranks'])}, "
            f"regime {w['regime']}, sigma {w['sigma']}, leaf {w['B']} slices, {w['n_queries']} concurrent "
            f"log-uniform queries L in [{w['lo']},{w['hi']}], theta 0.7, max_iter 20, tol 0.01, FP32")


def series_of(name, T=None):
    """The workload's seeded series (its first T slices: the generator draws
    regime by regime, so a prefix is the same for any length)."""
    w = synth.WORKLOADS[name]
    T = w["T"] if T is None else T
    if name == "fp32_plain":
        X = synth.piecewise_tucker(w["T"], w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
        return w, X[:T].astype(np.float32)
    return w, synth.piecewise_tucker_regimes(T, w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])


# ---------------------------------------------------------------------------
# algorithmic FLOPs of one query in the coefficient-space form of the engine
# ---------------------------------------------------------------------------
def query_flops(hits, ranks_out, node_ranks, dims, iters):
    """FLOPs of one range query: partial-hit QR, QR of the stacked factors,
    initial Gram/eig, `iters` ALS iterations (TTM chains, Grams, eigs), the
    core, and the assembly of U1..Up.  Symmetric Grams count their packed
    triangle; an eigenproblem counts its tridiagonalization and the
    back-transformation of the kept vectors."""
    p = len(ranks_out)
    ro = list(ranks_out)
    q = []
    f = 0.0
    for (level, index, lo_n, hi_n, lo, hi, partial) in hits:
        qi = list(node_ranks)
        ell = hi - lo
        if partial:
            qi[0] = min(ell, node_ranks[0])
            n = node_ranks[0]
            f += 2.0 * ell * n * n - 2.0 / 3.0 * min(ell, n) ** 3        # Householder QR
            f += 2.0 * qi[0] * np.prod(node_ranks)                        # core x_1 R
        q.append(qi)
    k = [sum(qi[n] for qi in q) for n in range(p)]
    c = [k[0]] + [min(dims[n - 1], k[n]) for n in range(1, p)]
    r_keep = list(ro)

    def eig(n, r=None):
        # Householder tridiagonalization (4/3 n^3) and the back-transformation of
        # the r kept vectors (2 n^2 r); bisection and inverse iteration are O(n r)
        return 4.0 / 3.0 * n ** 3 + 2.0 * n * n * (r if r is not None else min(n, max(r_keep)))
    for n in range(1, p):
        Dn = dims[n - 1]
        f += 2.0 * Dn * k[n] ** 2 - 2.0 / 3.0 * min(Dn, k[n]) ** 3      # QR of Phi_n
        for qi in q:
            rest = np.prod(qi) / qi[n]
            f += qi[n] * (qi[n] + 1) * rest                                  # Gram of mat_n(H_i)
            f += 2.0 * c[n] * qi[n] ** 2 + c[n] * (c[n] + 1) * qi[n]       # R_i M_i R_i^T
        f += eig(c[n], ro[n])

    def chain(qi, order_dims, modes):
        fl, d = 0.0, list(order_dims)
        for m, a in modes:
            fl += 2.0 * np.prod(d) * a
            d[m] = a
        return fl

    for _ in range(iters):
        R0 = np.prod(ro[1:])
        for qi in q:
            for m in range(1, p):
                f += 2.0 * ro[m] * qi[m] * c[m]                           # W_im
            f += chain(qi, qi, [(m, ro[m]) for m in range(1, p)])
        f += k[0] * (k[0] + 1) * R0 + eig(c[0], ro[0])
        for n in range(1, p):
            for qi in q:
                modes = [(0, ro[0])] + [(m, ro[m]) for m in range(1, p) if m != n] + [(n, c[n])]
                for m in range(1, p):
                    if m != n:
                        f += 2.0 * ro[m] * qi[m] * c[m]
                f += chain(qi, qi, modes)
            Rn = np.prod(ro) / ro[n]
            f += c[n] * (c[n] + 1) * Rn + eig(c[n], ro[n])
        f += 2.0 * np.prod(ro) * c[p - 1]                                  # core
    for qi, (level, index, lo_n, hi_n, lo, hi, partial) in zip(q, hits):
        ell = hi - lo
        f += (4.0 if partial else 2.0) * ell * qi[0] * ro[0]               # U1 rows
    for n in range(1, p):
        f += 4.0 * dims[n - 1] * c[n] * ro[n]                              # Q_n E_n
    return f


# ---------------------------------------------------------------------------
# FP64 CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
_ORACLE = None


def _oracle_init(tree):
    global _ORACLE
    _ORACLE = tree


def _oracle_query(args):
    ts, te = args
    t0 = time.perf_counter()
    r = _ORACLE.query(int(ts), int(te))
    return time.perf_counter() - t0, r["G"], r["U"], r["iters"]


def build_oracle_tree(w, X):
    from oracle.tree import StreamSegmentTree
    t = StreamSegmentTree(w["dims"], w["ranks"], B=w["B"], max_iter=20, tol=0.01)
    t.build(np.asarray(X, dtype=np.float64))
    return t


def oracle_pool(tree, cores):
    """Spawned workers (BLAS single-threaded), each holding the oracle tree."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_oracle_init, initargs=(tree,))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(Q, limit):
    """Indices of the workload's queries inside the oracle's tree (t_e <=
    ORACLE_T): on them the tree over the first ORACLE_T slices has the same
    nodes and hit sets as the full tree (nodes complete at T never change)."""
    idx = [i for i in range(len(Q)) if Q[i][1] <= ORACLE_T]
    return idx[:limit]


def run_reference(args, name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = synth.WORKLOADS[name]
    T_or = min(ORACLE_T, w["T"])
    _, X = series_of(name, T_or)
    Q = synth.query_ranges(w["T"], w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    tree = build_oracle_tree(w, X)
    sample = [i for i in range(len(Q)) if Q[i][1] <= T_or]
    cores = host_cores()
    per_step = 64
    with oracle_pool(tree, cores) as pool:
        pool.map(_oracle_query, [tuple(Q[sample[0]])] * cores)
        times, qtimes = [], []
        for s in range(args.warmup + args.steps):
            idx = [sample[(s * per_step + j) % len(sample)] for j in range(per_step)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_query, [tuple(Q[i]) for i in idx], chunksize=1)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
                qtimes.extend(r[0] for r in res)
    total = sum(times)
    value = per_step * len(times) / total
    desc = (f"{per_step} queries per step, cycling through the {len(sample)} workload queries with t_e <= {T_or}; "
            f"oracle tree over the first {T_or} slices (built untimed), process pool, BLAS single-threaded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w, name), "impl_note": "FP64 NumPy/LAPACK oracle of the paper's algorithms"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": 1e3 * float(np.percentile(qtimes, 50)), "p99": 1e3 * float(np.percentile(qtimes, 99)),
                       "mode": f"one query per worker, {len(qtimes)} queries"},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.path = tempfile.mktemp(suffix=".csv")
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json),
    else the recipe's earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def fp32_alu_peak(tk, dev_index, sm_max_mhz):
    """FP32 CUDA-core peak from unit counts and the maximum clock, and the
    FMA rate the device sustains (tk_probe_fma_rate, CUDA events)."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    derived = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    measured = tk.fma_rate("f32", dev_index) / 1e12
    return derived, measured, sms, mhz


def batch_flops(tree, Q, info, w):
    f = 0.0
    for i, (ts, te) in enumerate(Q):
        hits = tree.hit_set(int(ts), int(te))
        ro = list(info[i].ranks[: tree.p])
        f += query_flops(hits, ro, list(w["ranks"]), list(w["dims"]), int(info[i].iters))
    return f


def plain_latency(tk, torch, tree, Q, dev, stream, idx, out_d):
    """The plain GPU method: one query per launch sequence, each timed with
    CUDA events on the tree's stream."""
    lat = []
    with torch.cuda.stream(stream):
        for i in idx:
            r = torch.from_numpy(Q[i:i + 1].copy()).to(dev)
            o = torch.from_numpy(tree.layout(Q[i:i + 1])).to(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tree.query_batch(r, o, out_d[: int(o[-1])])
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
    return lat


def pct(v, q):
    return float(np.percentile(v, q)) if len(v) else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_r16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--queries", type=int, default=0,
                    help="answer only the workload's first N queries per step (0: all; for profiling runs)")
    ap.add_argument("--heavy-hits", type=int, default=0,
                    help="batch heavy-query threshold of the headline (0: autotuned before the warm-up)")
    ap.add_argument("--large", type=int, default=1,
                    help="1: run the large-series section (500x500xT=8192, ranks 20, leaf 32); 0: skip")
    ap.add_argument("--large-only", action="store_true", help="run only the large-series section and print it")
    ap.add_argument("--eig64-steps", type=int, default=2,
                    help="timed launches of the headline batch with FP64 stitch eigenproblems (0: skip)")
    ap.add_argument("--plain-steps", type=int, default=5,
                    help="timed launches of the FP32 plain workload's 1000-query batch (0: skip)")
    ap.add_argument("--appends", type=int, default=256,
                    help="single-slice appends timed on the 4-way stream (0: skip)")
    ap.add_argument("--theta-sweep", action="store_true",
                    help="run only the pruning-threshold sweep (theta 0.5, 0.7, 0.9) and print it")
    ap.add_argument("--latency-vs-T", action="store_true",
                    help="run only the query-latency-versus-timespan series and print it")
    ap.add_argument("--appends-only", action="store_true",
                    help="run only the append-latency section and print it")
    ap.add_argument("--p-sweep", action="store_true",
                    help="run only the sweep over the number of modes (p = 3..7) and print it")
    ap.add_argument("--serve-seconds", type=float, default=15.36,
                    help="length of the serving run (appends at 1 kHz; 15.36 s covers T 1024 -> 16384)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, args.workload)

    import torch
    import paper_2501_06647_gb300 as tk

    if args.theta_sweep:
        torch.cuda.set_device(0)
        print(json.dumps({"theta_sweep": theta_sweep(tk, torch, torch.device("cuda", 0), 0)}))
        return 0
    if args.latency_vs_T:
        torch.cuda.set_device(0)
        print(json.dumps({"latency_vs_T": latency_vs_T_section(tk, torch, torch.device("cuda", 0), 0)}))
        return 0
    if args.p_sweep:
        torch.cuda.set_device(0)
        print(json.dumps({"p_sweep": p_sweep_section(tk, torch, torch.device("cuda", 0), 0)}))
        return 0
    if args.large_only:
        torch.cuda.set_device(0)
        print(json.dumps({"large_r20": large_section(tk, torch, torch.device("cuda", 0), 0)}))
        return 0
    if args.appends_only:
        torch.cuda.set_device(0)
        print(json.dumps({"appends": append_section(tk, torch, torch.device("cuda", 0), 0, args.appends)}))
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    name = args.workload
    w, X = series_of(name)
    Q = synth.query_ranges(w["T"], w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    if args.queries > 0:
        Q = np.ascontiguousarray(Q[: args.queries])
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32",
                   device=local, stream=stream)
    Xd = torch.from_numpy(X).to(dev)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    tree.build(Xd)
    tree.sync()
    build_s = time.perf_counter() - tb0
    del Xd

    offsets = tree.layout(Q)
    ranges_d = torch.from_numpy(Q.copy()).to(dev)
    offsets_d = torch.from_numpy(offsets).to(dev)
    out_d = torch.empty(int(offsets[-1]), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    # the batch launch shape (heavy-query threshold), chosen by the engine's
    # autotuner on this batch before the warm-up (untimed)
    default_heavy = tree.heavy_hits
    tt0 = time.perf_counter()
    if args.heavy_hits > 0:  # set, not tuned (profiling runs: no tuning launches)
        tree.heavy_hits = args.heavy_hits
        heavy, tune_ms = tree.heavy_hits, None
    else:
        with torch.cuda.stream(stream):
            heavy, tune_ms = tree.tune_batch(ranges_d, offsets_d, out_d, reps=1)
    tune_s = time.perf_counter() - tt0

    def step():
        tree.query_batch(ranges_d, offsets_d, out_d)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    tree.sync()

    # ---- timed region: device time of the batch launches, L2 flushed between ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = tree.launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpu_launches = tree.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    n_q = len(Q)
    total_ms, value = replica_throughput(total_ms, n_q * args.steps, world, dist, dev)
    clocks = clk.summary()
    tree.sync()

    # ---- in-batch latency: launch to each query's completion (GPU global timer) --
    with torch.cuda.stream(stream):
        flush.zero_()
    tree.sync()
    out_chk, _, info = tree.query_batch_host(Q, offsets, None, with_info=True)
    t0 = min(f.start_ns for f in info)
    done_ms = np.array([(f.end_ns - t0) / 1e6 for f in info])
    job_ms = np.array([(f.end_ns - f.start_ns) / 1e6 for f in info])

    # ---- the plain method: one query per launch, on every 50th query ------------
    plain_idx = list(range(0, n_q, 50))
    lat = plain_latency(tk, torch, tree, Q, dev, stream, plain_idx, out_d)
    plain_qps = 1e3 / float(np.mean(lat))

    # ---- end to end through the C ABI with host buffers --------------------------
    host_out = torch.empty(int(offsets[-1]), dtype=torch.float32, pin_memory=True).numpy()
    host_ranges = torch.from_numpy(Q.copy()).pin_memory().numpy()
    host_offs = torch.from_numpy(offsets.copy()).pin_memory().numpy()
    tree.query_batch_host(host_ranges, host_offs, host_out, with_info=False)
    e2e_s = 0.0
    e2e_steps = 3
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        ta = time.perf_counter()
        tree.query_batch_host(host_ranges, host_offs, host_out, with_info=False)
        e2e_s += time.perf_counter() - ta
    e2e_value = world * n_q * e2e_steps / e2e_s

    # ---- roofline of the dominant kernel (k_batch answers the whole batch) -------
    flops = batch_flops(tree, Q, info, w)
    peak, peak_meas, sms, mhz = fp32_alu_peak(tk, local, clocks.get("sm_max_mhz"))
    avg_launch_s = total_ms / 1e3 / args.steps
    achieved = flops / avg_launch_s / 1e12
    out_bytes = int(offsets[-1]) * 4
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": BATCH_DRAM_BYTES,
                "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one k_batch launch (ncu), "
                                "captured on the first 1000 queries and scaled by 10 (traffic grows with the "
                                "queries: output and per-query workspace); null: no capture of this kernel version",
                "kernel": "k_batch<float> (one persistent launch answers the whole batch, after k_plan)",
                "flops_per_launch": flops,
                "peak_note": f"FP32 CUDA-core peak from unit counts: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 "
                             f"x {mhz:.0f} MHz; measured FMA rate of this GPU (tk_probe_fma_rate) "
                             f"{peak_meas:.1f} TFLOP/s, frac of measured {achieved / peak_meas:.4f}",
                "peak_measured": peak_meas,
                "hbm_view": {"algorithmic_bytes": out_bytes + tree.arena_bytes(),
                             "achieved_gbs": (out_bytes + tree.arena_bytes()) / avg_launch_s / 1e9,
                             "note": "output written + tree read once"}}

    raw_bytes = int(X.nbytes)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(w, name) + (f" (first {n_q} queries)" if args.queries else ""),
                   "queries_per_step": n_q,
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "tree_arena_bytes": tree.arena_bytes(),
                   "heavy_hits": heavy,
                   "autotune": {"chosen_heavy_hits": heavy, "default_heavy_hits": default_heavy,
                                "best_ms": tune_ms, "seconds": tune_s,
                                "note": ("set by --heavy-hits (no tuning)" if args.heavy_hits > 0 else
                                         "tk_batch_tune: each candidate threshold timed once on this batch "
                                         "before the warm-up")}},
        "latency_ms": {"p50": pct(done_ms, 50), "p99": pct(done_ms, 99),
                       "mode": "in-batch: batch launch to each query's completion (GPU global timer), "
                               f"{n_q} concurrent queries",
                       "job_p50": pct(job_ms, 50), "job_p99": pct(job_ms, 99)},
        "plain": {"queries_per_s": plain_qps, "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
                  "queries": len(lat), "mode": "one query per launch sequence (every 50th workload query)",
                  "batched_over_plain": value / plain_qps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(Q.nbytes + offsets.nbytes),
                "d2h_bytes_per_step": out_bytes},
        "gpu_launches": gpu_launches,
        "roofline": roofline,
        "tree_build": {"seconds": build_s, "raw_bytes": raw_bytes, "roofline": {
            "bound": "hbm", "achieved": raw_bytes / build_s / 1e9, "peak": hbm_peak_gbs(), "unit": "GB/s",
            "frac": raw_bytes / build_s / 1e9 / hbm_peak_gbs(),
            "note": "raw series read once by the leaf kernel; leaves and merges are latency-bound, "
                    "so this is far below the HBM peak"}},
        "clocks": clocks,
    }

    del out_d, flush
    torch.cuda.empty_cache()
    if args.eig64_steps > 0:
        line["eig_fp64"] = eig64_throughput(tk, torch, dev, local, w, X, Q, args.eig64_steps)

    if args.plain_steps > 0:
        line["plain_r10"] = plain_section(tk, torch, dev, local, args.plain_steps)
    if args.appends > 0:
        line["appends"] = append_section(tk, torch, dev, local, args.appends)
    if args.serve_seconds > 0:
        line["serving"] = serving_section(tk, torch, dev, local, args.serve_seconds)
    if args.large:
        line["large_r20"] = large_section(tk, torch, dev, local)

    # ---- FP64 oracle on the host cores: cpu_baseline + matched-error check -------
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu_section(line, w, X, Q, offsets, tree, out_chk, info)
        except Exception as exc:  # report, do not lose the GPU measurement
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                                    "sample": None, "error": f"{type(exc).__name__}: {exc}"}
    tree.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def plain_section(tk, torch, dev, local, steps):
    """The FP32 plain workload (100x100 slices, T = 4096, ranks 10, leaf 16,
    1000 log-uniform queries): its batched launch and the one-query-per-launch
    method, L2 flushed between timed launches."""
    w, X = series_of("fp32_plain")
    Q = synth.query_ranges(w["T"], w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", device=local,
                   stream=stream)
    Xd = torch.from_numpy(X).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree.build(Xd)
    tree.sync()
    build_s = time.perf_counter() - t0
    del Xd
    offsets = tree.layout(Q)
    rd = torch.from_numpy(Q.copy()).to(dev)
    od = torch.from_numpy(offsets).to(dev)
    out = torch.empty(int(offsets[-1]), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    heavy, _ = tree.tune_batch(rd, od, out, reps=2)
    ms = []
    for k in range(steps + 2):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tree.query_batch(rd, od, out)
            b.record(stream)
        b.synchronize()
        if k >= 2:
            ms.append(a.elapsed_time(b))
    lat = plain_latency(tk, torch, tree, Q, dev, stream, list(range(0, len(Q), 5)), out)
    tree.close()
    qps = len(Q) / (np.mean(ms) / 1e3)
    return {"workload": workload_desc(w, "fp32_plain"), "batch_ms": float(np.mean(ms)), "queries_per_s": qps,
            "heavy_hits": heavy,
            "plain_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "queries": len(lat)},
            "plain_queries_per_s": 1e3 / float(np.mean(lat)), "batched_over_plain": qps * float(np.mean(lat)) / 1e3,
            "tree_build_s": build_s}


def theta_sweep(tk, torch, dev, local, thetas=((1, 2), (7, 10), (9, 10))):
    """Pruning threshold theta (Section 5.1, Algorithm 1) on the FP32 plain
    workload: per theta, the batch throughput, the mean hit-set size and
    iteration count, and the mean relative error ||X - Y|| / ||X|| of 100
    sampled queries (the reconstruction materialized on the GPU in FP64)."""
    w = synth.WORKLOADS["fp32_plain"]
    X = synth.piecewise_tucker(w["T"], w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
    Q = synth.query_ranges(w["T"], w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    X64 = torch.from_numpy(X).to(dev)
    rows = []
    for num, den in thetas:
        stream = torch.cuda.Stream(device=dev)
        tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], theta=(num, den), max_iter=20, tol=0.01,
                       dtype="f32", device=local, stream=stream)
        tree.build(Xd)
        tree.sync()
        offsets = tree.layout(Q)
        rd = torch.from_numpy(Q.copy()).to(dev)
        od = torch.from_numpy(offsets).to(dev)
        out = torch.empty(int(offsets[-1]), dtype=torch.float32, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        ms = []
        for k in range(6):
            with torch.cuda.stream(stream):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tree.query_batch(rd, od, out)
                b.record(stream)
            b.synchronize()
            if k >= 2:
                ms.append(a.elapsed_time(b))
        _, _, info = tree.query_batch_host(Q, offsets, None, with_info=True)
        errs = []
        for i in range(0, len(Q), len(Q) // 100):
            ts, te = int(Q[i][0]), int(Q[i][1])
            G, U = tree.unpack(out[int(offsets[i]):int(offsets[i + 1])], te - ts)
            Y = torch.einsum("abc,ia,jb,kc->ijk", G.double(), U[0].double(), U[1].double(), U[2].double())
            Xs = X64[ts:te]
            errs.append(float(torch.linalg.norm(Xs - Y) / torch.linalg.norm(Xs)))
        rows.append({"theta": num / den, "queries_per_s": len(Q) / (np.mean(ms) / 1e3), "batch_ms": float(np.mean(ms)),
                     "mean_hits": float(np.mean([f.n_hits for f in info])),
                     "mean_iters": float(np.mean([f.iters for f in info])),
                     "mean_rel_err": float(np.mean(errs)), "sampled_queries": len(errs)})
        tree.close()
        del out, flush
    return rows


P_SWEEP_SHAPES = [(1000, 1000), (100, 100, 100), (100, 100, 10, 10), (100, 10, 10, 10, 10), (10,) * 6]


def p_sweep_section(tk, torch, dev, local, lengths=(98, 192, 384), n_q=40, r=5, regime=100, sigma=0.05):
    """Scalability in the number of modes (the paper's synthetic series of
    1000 slices and 10^9 entries for p = 3..7, target rank 5, query lengths
    98, 192 and 384): per p, the tree build time (single-slice leaves, as in
    the paper) and the p50/p99 latency of n_q queries per length, one query
    per launch.  The series is piecewise Tucker of rank 5 per regime of 100
    slices with unit signal RMS and N(0, sigma^2) noise, drawn on the GPU from
    a seeded generator."""
    rows = []
    T = 1000
    for dims in P_SWEEP_SHAPES:
        p = len(dims) + 1
        g = torch.Generator(device=dev)
        g.manual_seed(3000 + p)
        X = torch.empty((T,) + dims, dtype=torch.float32, device=dev)
        for t0 in range(0, T, regime):
            l = min(regime, T - t0)
            Y = torch.randn((r,) * p, generator=g, device=dev)
            for n, d in enumerate((l,) + dims):
                U, _ = torch.linalg.qr(torch.randn(d, r, generator=g, device=dev))
                Y = torch.tensordot(U, Y, dims=([1], [n])).movedim(0, n)
            Y *= (l * float(np.prod(dims))) ** 0.5 / float(Y.norm())  # unit RMS per entry
            X[t0:t0 + l] = Y + sigma * torch.randn(Y.shape, generator=g, device=dev)
            del Y
        stream = torch.cuda.Stream(device=dev)
        tree = tk.Tree(dims, (r,) * p, leaf_slices=1, max_iter=20, tol=0.01, dtype="f32", device=local,
                       stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree.build(X)
        tree.sync()
        build_s = time.perf_counter() - t0
        del X
        torch.cuda.empty_cache()
        rng = np.random.default_rng(4000 + p)
        lat = {}
        for L in lengths:
            ms = []
            for s0 in rng.integers(0, T - L + 1, size=n_q):
                q = np.array([[s0, s0 + L]], dtype=np.int64)
                o = tree.layout(q)
                rd, od = torch.from_numpy(q).to(dev), torch.from_numpy(o).to(dev)
                out = torch.empty(int(o[-1]), dtype=torch.float32, device=dev)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a.record(stream)
                    tree.query_batch(rd, od, out)
                    b.record(stream)
                tree.sync()
                ms.append(a.elapsed_time(b))
            lat[str(L)] = {"p50_ms": pct(ms, 50), "p99_ms": pct(ms, 99)}
        rows.append({"p": p, "shape": [T] + list(dims), "tree_build_s": build_s, "arena_bytes": tree.arena_bytes(),
                     "latency": lat})
        tree.close()
        torch.cuda.empty_cache()
    return {"workload": f"1000 x ... (10^9 entries), rank {r}, regime {regime}, sigma {sigma}, leaves of one slice, "
                        f"FP32, tol 0.01; {n_q} queries per length, one per launch", "points": rows}


def replica_throughput(local_ms, local_units, world, dist=None, device=None):
    """Whole-job throughput of N replicas (Section 7's queries are
    independent: every rank answers its own copy of the batch, no data-path
    collective).  The job's time is the slowest rank's (max over ranks, then
    a barrier); value = all ranks' units / that time.  Returns (ms, units/s)."""
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return total_ms, world * local_units / (total_ms / 1e3)


def append_section(tk, torch, dev, local, n_app):
    """Stream-update latency (Algorithms 3-4) on the 4-way 64x64x32 stream
    (ranks 8, leaf 16, FP32): the tree is built to T0 = 1024, then n_app
    single slices already in device memory are appended one at a time, each
    timed with CUDA events on the tree's stream.  Every 16th append completes
    a leaf block: Tucker-ALS of the block plus the Stitch of every newly
    complete ancestor.  The others only store the slice (the open block is
    decomposed when a query reaches into it); the cost of that is timed too,
    as one query over the last 40 slices right after each append."""
    w = synth.WORKLOADS["serving_4way"]
    T0 = w["T0"]
    X = synth.piecewise_tucker_regimes(T0 + n_app, w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", device=local,
                   stream=stream)
    Xd = torch.from_numpy(X).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree.build(Xd[:T0])
    tree.sync()
    build_s = time.perf_counter() - t0

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    app, done, tail = [], [], []
    for k in range(n_app):
        with torch.cuda.stream(stream):  # the tree's stream: calls stay asynchronous
            T = tree.T
            a = ev()
            tree.append(Xd[T])
            b = ev()
            r = torch.tensor([[max(0, T + 1 - 40), T + 1]], dtype=torch.int64, device=dev)
            o = torch.from_numpy(tree.layout(r.cpu().numpy())).to(dev)
            out = torch.empty(int(o[-1]), dtype=torch.float32, device=dev)
            c = ev()
            tree.query_batch(r, o, out)
            d = ev()
            tree.sync()
        (done if (T + 1) % w["B"] == 0 else app).append(a.elapsed_time(b))
        if (T + 1) % w["B"] != 0:
            tail.append(c.elapsed_time(d))
    tree.close()
    q = lambda v, f: sorted(v)[min(len(v) - 1, int(f * len(v)))] if v else None
    block_bytes = w["B"] * int(np.prod(w["dims"])) * 4
    mean_done = float(np.mean(done)) if done else None
    return {
        "workload": f"4-way {w['dims'][0]}x{w['dims'][1]}x{w['dims'][2]} slices, ranks {w['ranks']}, leaf {w['B']}, "
                    f"FP32, tol 0.01; tree built to T={T0} ({build_s * 1e3:.1f} ms), then {n_app} appends",
        "append_ms": {"mean": float(np.mean(app)) if app else None, "p99": q(app, 0.99),
                      "what": "slice stored in the open block"},
        "block_complete_ms": {"mean": float(np.mean(done)) if done else None, "max": max(done) if done else None,
                              "count": len(done),
                              "what": "leaf Tucker-ALS + Stitch of the newly complete ancestors"},
        "open_block_query_ms": {"mean": float(np.mean(tail)) if tail else None, "p99": q(tail, 0.99),
                                "what": "query over the last 40 slices, decomposing the open block first"},
        "roofline": {"bound": "hbm", "kernel": "k_leaf<float> + k_stitch merges of one block completion",
                     "achieved": block_bytes / (mean_done * 1e-3) / 1e9 if mean_done else None,
                     "peak": hbm_peak_gbs(), "unit": "GB/s",
                     "frac": block_bytes / (mean_done * 1e-3) / 1e9 / hbm_peak_gbs() if mean_done else None,
                     "algorithmic_bytes": block_bytes,
                     "note": "the raw block read once; the decomposition is latency-bound (eigensolvers and "
                             "barrier-separated steps on 8 SMs), far from this bound"},
    }


def latency_vs_T_section(tk, torch, dev, local, L=384, n_q=50, checkpoints=(512, 1024, 2048, 4096)):
    """Query latency against the timespan T (the paper's experiment on
    efficiency w.r.t. T): queries of one fixed length L, while single-slice
    appends grow the stream between the measurements.  The FP32 plain
    workload's series (100x100 slices, ranks 10, leaf 16): the tree is built
    to the first checkpoint, then slices are appended one at a time up to
    each next one; at every checkpoint n_q queries [s, s + L) with a uniform
    start are answered one per launch, each timed with CUDA events on the
    tree's stream."""
    w = synth.WORKLOADS["fp32_plain"]
    T_end = max(checkpoints)
    X = synth.piecewise_tucker(T_end, w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", device=local,
                   stream=stream)
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    tree.build(Xd[:checkpoints[0]])
    tree.sync()
    rng = np.random.default_rng(w["qseed"])
    points = []
    for Tc in checkpoints:
        while tree.T < Tc:
            tree.append(Xd[tree.T])
        tree.sync()
        starts = rng.integers(0, Tc - L + 1, size=n_q)
        ms, hits = [], []
        for s0 in starts:
            r = np.array([[s0, s0 + L]], dtype=np.int64)
            o = tree.layout(r)
            rd, od = torch.from_numpy(r).to(dev), torch.from_numpy(o).to(dev)
            out = torch.empty(int(o[-1]), dtype=torch.float32, device=dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                tree.query_batch(rd, od, out)
                b.record(stream)
            tree.sync()
            ms.append(a.elapsed_time(b))
            hits.append(len(tree.hit_set(int(s0), int(s0 + L))))
        points.append({"T": int(Tc), "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                       "mean_hits": float(np.mean(hits))})
    tree.close()
    return {"workload": f"{w['dims'][0]}x{w['dims'][1]} slices, ranks {tuple(w['ranks'])}, leaf {w['B']}, FP32, "
                        f"tol 0.01; built to T={checkpoints[0]}, then single-slice appends",
            "query_length": L, "queries_per_point": n_q, "points": points}


def serving_section(tk, torch, dev, local, seconds):
    """Continuous batching under load: a 4-way 64x64x32 stream (ranks 8, leaf
    16, FP32) grows from T0 = 1024 by single-slice appends at 1 kHz while range
    queries of log-uniform length (16..T as of arrival) arrive as a Poisson
    process at 5k/s; all go through the native server.  Latency is submit to
    result in host memory (host clock).  Then a burst of 4096 queries at the
    final T measures the server's saturated throughput."""
    w = synth.WORKLOADS["serving_4way"]
    T0 = w["T0"]
    n_app = int(round(seconds * w["append_hz"]))
    T_end = T0 + n_app
    # slice t of the stream is slice t mod 4096 of the seeded series (whole
    # regimes of 512, so the regime structure is kept; 16384 distinct slices
    # of 64x64x32 would be 8.6 GB to generate)
    POOL = 4096
    X = synth.piecewise_tucker_regimes(min(T_end, POOL), w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", device=local)
    tree.build(torch.from_numpy(X[:T0]).to(dev))
    tree.sync()
    # arrival schedule: appends every 1 ms, queries at exponential gaps
    rng = np.random.Generator(np.random.PCG64(w["qseed"]))
    n_q = int(seconds * w["query_hz"] * 1.5) + 16
    qt = np.cumsum(rng.exponential(1.0 / w["query_hz"], n_q))
    qt = qt[qt < seconds]
    at = (np.arange(n_app) + 0.5) / w["append_hz"]
    events = sorted([(t, 1, i) for i, t in enumerate(at)] + [(t, 0, i) for i, t in enumerate(qt)])
    u = rng.uniform(size=(len(qt), 2))
    dims, rk = w["dims"], w["ranks"]
    fixed = int(np.prod(rk)) + sum(d * r for d, r in zip(dims, rk[1:]))
    K = 512
    ring = np.empty((K, fixed + T_end * rk[0]), dtype=np.float32)
    ring_ticket = [0] * K
    lib_ = tk.lib()
    srv = tk.Server(tree, max_batch=1024, max_batch_out_elems=64 << 20)
    tkt = ctypes.c_uint64()
    T_sub, qi, lens = T0, 0, []
    t0 = time.perf_counter()
    for t_ev, kind, i in events:
        while time.perf_counter() - t0 < t_ev:
            pass
        if kind == 1:
            srv.submit_append(X[T_sub % POOL])
            T_sub += 1
            continue
        Lq = int(round(np.exp(np.log(w["lo"]) + u[i, 0] * (np.log(T_sub) - np.log(w["lo"])))))
        Lq = max(1, min(Lq, T_sub))
        ts = min(int(u[i, 1] * (T_sub - Lq + 1)), T_sub - Lq)
        slot = qi % K
        if ring_ticket[slot]:
            lib_.tk_server_wait(srv.h, ring_ticket[slot], -1.0)
        rc = lib_.tk_server_submit_query(srv.h, ts, ts + Lq, None, ring[slot].ctypes.data, None, ctypes.byref(tkt))
        if rc != 0:
            raise tk.TuckerError(rc, "tk_server_submit_query")
        ring_ticket[slot] = tkt.value
        lens.append(Lq)
        qi += 1
    srv.drain()
    st_load = srv.stats()
    for slot in range(K):
        if ring_ticket[slot]:
            lib_.tk_server_wait(srv.h, ring_ticket[slot], -1.0)
            ring_ticket[slot] = 0
    srv.close()
    # saturated burst at the final T (a fresh server, so that its counters start at zero)
    srv = tk.Server(tree, max_batch=1024, max_batch_out_elems=64 << 20)
    nb = 4096
    qb = synth.query_ranges(T_end, nb, w["qseed"] + 1, "loguniform", w["lo"], T_end)
    sizes = [fixed + int(te - ts) * rk[0] for ts, te in qb]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    flat = np.empty(int(offs[-1]), dtype=np.float32)
    base = flat.ctypes.data
    for j, (ts, te) in enumerate(qb):
        rc = lib_.tk_server_submit_query(srv.h, int(ts), int(te), None, base + 4 * int(offs[j]), None,
                                         ctypes.byref(tkt))
        if rc != 0:
            raise tk.TuckerError(rc, "tk_server_submit_query")
    srv.drain()
    st_burst = srv.stats()
    srv.close()
    tree.close()
    return {
        "workload": f"4-way {dims[0]}x{dims[1]}x{dims[2]}xT, T {T0}->{T_end} by appends at "
                    f"{w['append_hz']:.0f} Hz (slice t = slice t mod {POOL} of the seeded series), Poisson queries "
                    f"at {w['query_hz']:.0f}/s of log-uniform length {w['lo']}..T, ranks {rk}, leaf {w['B']}, FP32, "
                    "tol 0.01",
        "seconds": seconds, "queries": int(st_load["queries_done"]), "appends": int(st_load["appends_done"]),
        "offered_qps": len(qt) / seconds, "served_qps": st_load["queries_done"] / st_load["elapsed_s"],
        "latency_ms": {"p50": st_load["latency_p50_ms"], "p99": st_load["latency_p99_ms"],
                       "max": st_load["latency_max_ms"], "clock": "host, submit to result in host memory"},
        "mean_batch": st_load["mean_batch"], "mean_query_len": float(np.mean(lens)) if lens else 0.0,
        "burst": {"queries": nb, "qps": st_burst["queries_done"] / st_burst["elapsed_s"],
                  "mean_batch": st_burst["mean_batch"], "latency_p50_ms": st_burst["latency_p50_ms"],
                  "latency_p99_ms": st_burst["latency_p99_ms"], "T": T_end},
    }


def cpu_section(line, w, X, Q, offsets, tree, out_chk, info):
    """FP64 oracle on the host cores (cpu_baseline) and the matched-error
    check of the batched FP32 answers, on the workload's queries with t_e <=
    ORACLE_T (the oracle's tree covers the first ORACLE_T slices)."""
    tree_o = build_oracle_tree(w, X[:ORACLE_T])
    cores = host_cores()
    sample = oracle_sample(Q, 400)
    with oracle_pool(tree_o, cores) as pool:
        pool.map(_oracle_query, [tuple(Q[sample[0]])] * cores)
        t0 = time.perf_counter()
        res = pool.map(_oracle_query, [tuple(Q[i]) for i in sample], chunksize=1)
        wall = time.perf_counter() - t0
    line["cpu_baseline"] = {"value": len(sample) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{len(sample)} workload queries with t_e <= {ORACLE_T}; oracle tree over the "
                                      f"first {ORACLE_T} slices (same nodes and hit sets there), built untimed; "
                                      "process pool, BLAS single-threaded per worker"}
    from oracle import metrics
    eg, eo, dd = [], [], []
    for j, i in enumerate(sample[:150]):
        ts, te = int(Q[i][0]), int(Q[i][1])
        G, U = tree.unpack(out_chk[offsets[i]:offsets[i + 1]], te - ts)
        r = list(info[i].ranks[: tree.p])
        G = np.float64(G[tuple(slice(0, x) for x in r)])
        U = [np.float64(u[:, :x]) for u, x in zip(U, r)]
        Xs = np.asarray(X[ts:te], dtype=np.float64)
        eg.append(metrics.relative_error(Xs, G, U))
        eo.append(metrics.relative_error(Xs, res[j][1], res[j][2]))
        dd.append(metrics.model_distance(G, U, res[j][1], res[j][2]) / np.linalg.norm(Xs))
    eg, eo = np.array(eg), np.array(eo)
    variants = precision_variants(w, X, Q, sample[:150], res)
    line["accuracy"] = {"variants": variants,"queries": len(eg), "mean_rel_err_gpu": float(np.mean(eg)),
                        "mean_rel_err_oracle_fp64": float(np.mean(eo)),
                        "mean_rel_err_relative_diff": float(abs(np.mean(eg) - np.mean(eo)) / np.mean(eo)),
                        "max_abs_err_diff": float(np.max(np.abs(eg - eo))),
                        "max_model_distance_rel": float(np.max(dd)),
                        "matched_vs_plain": "the batched launch and the one-query-per-launch method run the same "
                                            "kernels on the same tree: identical errors",
                        "note": "both with tol 0.01; iteration counts may differ near the threshold"}


def precision_variants(w, X, Q, idx, res):
    """Error of other arithmetic variants against the FP64 oracle on the same
    sampled queries: trees over the oracle's prefix of the series (the same
    nodes and hit sets for these queries) with the stitch eigenproblems in
    FP64, or the leaf Grams as single TF32 or on FP32 CUDA cores."""
    import torch
    import paper_2501_06647_gb300 as tk
    from oracle import metrics
    out = {}
    Qs = np.ascontiguousarray(Q[idx])
    for name, kw in (("fp32_stitch_fp64_eig", dict(eig_fp64=True)), ("leaf_grams_tf32", dict(math="tf32")),
                     ("leaf_grams_cuda_cores", dict(math="cuda_cores"))):
        t = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", **kw)
        t.build(torch.from_numpy(np.ascontiguousarray(X[:ORACLE_T])).cuda())
        offs = t.layout(Qs)
        o, _, info = t.query_batch_host(Qs, offs, None, with_info=True)
        eg, eo, dd = [], [], []
        for j, (ts, te) in enumerate(Qs):
            ts, te = int(ts), int(te)
            G, U = t.unpack(o[offs[j]:offs[j + 1]], te - ts)
            r = list(info[j].ranks[: t.p])
            G = np.float64(G[tuple(slice(0, x) for x in r)])
            U = [np.float64(u[:, :x]) for u, x in zip(U, r)]
            Xs = np.asarray(X[ts:te], dtype=np.float64)
            eg.append(metrics.relative_error(Xs, G, U))
            eo.append(metrics.relative_error(Xs, res[j][1], res[j][2]))
            dd.append(metrics.model_distance(G, U, res[j][1], res[j][2]) / np.linalg.norm(Xs))
        eg, eo = np.array(eg), np.array(eo)
        out[name] = {"mean_rel_err_relative_diff": float(abs(np.mean(eg) - np.mean(eo)) / np.mean(eo)),
                     "max_abs_err_diff": float(np.max(np.abs(eg - eo))),
                     "max_model_distance_rel": float(np.max(dd))}
        t.close()
    return out


def large_section(tk, torch, dev, local, n_app=32, n_err=12, n_plain=10):
    """The large series (500x500 slices, T = 8192, 8 GB in FP32, ranks 20,
    leaf 32, noise 0.1), drawn on the device: tree build (HBM roofline of the
    raw series read), the autotuned batch over its 2,000 log-uniform queries,
    single-query latency, n_app single-slice appends (one of which completes
    a leaf block of 500x500 Gram orders), and the relative error of sampled
    answers against the data (||X - Y||^2 = ||X||^2 - 2 <X x_n U_n^T, G> +
    ||G||^2, in FP64 on the device)."""
    w = synth.WORKLOADS["large_r20"]
    T = w["T"]
    t0 = time.perf_counter()
    X = synth.piecewise_tucker_device(T + n_app, w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"], dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32", device=local,
                   stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        tree.build(X[:T])
    tree.sync()
    build_s = time.perf_counter() - t0
    raw = T * int(np.prod(w["dims"])) * 4
    Q = synth.query_ranges(T, w["n_queries"], w["qseed"], "loguniform", w["lo"], w["hi"])
    offsets = tree.layout(Q)
    rd = torch.from_numpy(Q.copy()).to(dev)
    od = torch.from_numpy(offsets).to(dev)
    out = torch.empty(int(offsets[-1]), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        heavy, _ = tree.tune_batch(rd, od, out, reps=1)
        ms = []
        for k in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tree.query_batch(rd, od, out)
            b.record(stream)
            b.synchronize()
            if k >= 1:
                ms.append(a.elapsed_time(b))
    batch_ms = float(np.mean(ms))
    lat = plain_latency(tk, torch, tree, Q, dev, stream, list(range(0, len(Q), len(Q) // n_plain)), out)
    # errors of sampled answers against the data
    out_h, _, info = tree.query_batch_host(Q[:n_err], None, None, with_info=True)
    offs_h = tree.layout(Q[:n_err])
    errs = []
    for i in range(n_err):
        ts, te = int(Q[i][0]), int(Q[i][1])
        G, U = tree.unpack(out_h[offs_h[i]:offs_h[i + 1]], te - ts)
        r = list(info[i].ranks[: tree.p])
        G = torch.from_numpy(np.float64(G[tuple(slice(0, x) for x in r)])).to(dev)
        U = [torch.from_numpy(np.float64(u[:, :x])).to(dev) for u, x in zip(U, r)]
        xx, xg = 0.0, 0.0
        for c0 in range(ts, te, 256):
            c1 = min(te, c0 + 256)
            Xc = X[c0:c1].to(torch.float64)
            xx += float((Xc * Xc).sum())
            P = torch.einsum("tij,ta,ib,jc->abc", Xc, U[0][c0 - ts:c1 - ts], U[1], U[2])
            xg += float((P * G).sum())
        gg = float((G * G).sum())
        errs.append(float(np.sqrt(max(0.0, xx - 2 * xg + gg) / xx)))
    # appends: the open block fills and completes (leaf Tucker-ALS of a 32x500x500 block, then the merges)
    app, done = [], []
    for k in range(n_app):
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tree.append(X[tree.T])
            b.record(stream)
        b.synchronize()
        (done if tree.T % w["B"] == 0 else app).append(a.elapsed_time(b))
    arena = tree.arena_bytes()
    tree.close()
    del X, out
    torch.cuda.empty_cache()
    return {"workload": workload_desc(w, "large_r20"), "generate_s": gen_s,
            "tree_build": {"seconds": build_s, "raw_bytes": raw, "arena_bytes": arena,
                           "roofline": {"bound": "hbm", "achieved": raw / build_s / 1e9, "peak": hbm_peak_gbs(),
                                        "unit": "GB/s", "frac": raw / build_s / 1e9 / hbm_peak_gbs()}},
            "batch": {"queries": len(Q), "ms": batch_ms, "queries_per_s": len(Q) / (batch_ms / 1e3),
                      "heavy_hits": heavy},
            "plain": {"latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)}, "queries": len(lat),
                      "queries_per_s": 1e3 / float(np.mean(lat))},
            "rel_err_vs_data": {"queries": n_err, "mean": float(np.mean(errs)), "max": float(np.max(errs)),
                                "note": "relative reconstruction error of the answers against the raw series"},
            "appends": {"append_ms_mean": float(np.mean(app)) if app else None,
                        "block_complete_ms": done, "count": n_app}}


def eig64_throughput(tk, torch, dev, local, w, X, Q, steps):
    """The headline batch on a tree whose stitch eigenproblems run in FP64
    (tk_config.eig_fp64), autotuned and timed like the headline."""
    stream = torch.cuda.Stream(device=dev)
    tree = tk.Tree(w["dims"], w["ranks"], leaf_slices=w["B"], max_iter=20, tol=0.01, dtype="f32",
                   device=local, stream=stream, eig_fp64=True)
    tree.build(torch.from_numpy(X).to(dev))
    tree.sync()
    offsets = tree.layout(Q)
    rd = torch.from_numpy(Q.copy()).to(dev)
    od = torch.from_numpy(offsets).to(dev)
    out = torch.empty(int(offsets[-1]), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    heavy, _ = tree.tune_batch(rd, od, out, reps=1)
    ms = []
    for k in range(steps + 1):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tree.query_batch(rd, od, out)
            b.record(stream)
        b.synchronize()
        if k >= 1:
            ms.append(a.elapsed_time(b))
    tree.close()
    return {"ms_per_step": float(np.mean(ms)), "queries_per_s": len(Q) / (np.mean(ms) / 1e3), "heavy_hits": heavy,
            "note": "same workload and batch as the headline, stitch eigenproblems (orders >= 20) in FP64"}


if __name__ == "__main__":
    sys.exit(main())
