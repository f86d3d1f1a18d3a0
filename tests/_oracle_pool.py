"""Answers of the FP64 oracle for many range queries at once, in a pool of
spawned processes (one query per task, BLAS single-threaded per worker).  It
imports nothing of the CUDA engine, so that the workers never touch a GPU."""
import multiprocessing as mp
import os

_TREE = None


def _init(tree):
    global _TREE
    _TREE = tree


def _ask(rng):
    r = _TREE.query(int(rng[0]), int(rng[1]))
    return r["G"], r["U"], r["ranks"], r["iters"], r["hits"]


def oracle_answers(tree, Q, workers=16):
    """[(G, U, ranks, iters, hit records)] of the oracle tree for each range of Q."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4
    with mp.get_context("spawn").Pool(max(1, min(workers, cores)), initializer=_init, initargs=(tree,)) as pool:
        return pool.map(_ask, [tuple(int(x) for x in q) for q in Q], chunksize=4)
