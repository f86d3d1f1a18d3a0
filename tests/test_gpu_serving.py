"""The continuous-batching server (tk_server_*) through the C ABI.

Queries and stream updates are submitted as one interleaved burst (and from
several threads), so that the worker batches them.  Every query's answer must
be the one a twin tree gives when the same requests are replayed one at a time
in submission order: same hit count, ranks and iteration count; in FP64 the
reconstruction errors within 1e-9 relative and the factor subspaces within
1e-3 rad (the parity tolerance of the other GPU tests), in FP32 every output
element within 1e-5 (a batch may run a query in a larger CTA than a single
launch does, which changes reduction order).
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import synth  # noqa: E402
from gpu_util import series, engine_tree  # noqa: E402
from oracle import metrics  # noqa: E402

CASES = {
    "f64": dict(dims=(30, 20), ranks=(5, 5, 5), B=4, T0=128, T1=192, regime=64, sigma=0.01, seed=1001),
    "f32": dict(dims=(60, 50), ranks=(10, 10, 10), B=16, T0=256, T1=384, regime=128, sigma=0.05, seed=1002),
}


def _script(T0, T1, n_queries, seed):
    """Interleaved requests: ('a', t) appends slice t, ('q', ts, te) queries."""
    rng = np.random.default_rng(seed)
    T, reqs, nq = T0, [], 0
    while nq < n_queries or T < T1:
        if T < T1 and (nq >= n_queries or rng.random() < 0.3):
            reqs.append(("a", T))
            T += 1
        else:
            a = int(rng.integers(0, T))
            b = int(rng.integers(a + 1, T + 1))
            reqs.append(("q", a, b))
            nq += 1
    return reqs


def _same(dtype, X, ts, te, got, want):
    Gs, Us, Is = got
    Gt, Ut, It = want
    assert Is["ranks"] == It["ranks"] and Is["n_hits"] == It["n_hits"] and Is["iters"] == It["iters"]
    if dtype == "f32":
        for a, b in zip([Gs] + Us, [Gt] + Ut):
            assert np.allclose(a, b, rtol=0, atol=1e-5), (ts, te)
        return
    Xs = X[ts:te]
    ea = metrics.relative_error(Xs, Gs, Us)
    eb = metrics.relative_error(Xs, Gt, Ut)
    assert abs(ea - eb) <= 1e-9 * eb, (ts, te)
    assert max(metrics.principal_angle_max(a, b) for a, b in zip(Us, Ut)) < 1e-3


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_served_mix_matches_sequential_replay(dtype):
    import paper_2501_06647_gb300 as tk
    c = CASES[dtype]
    X = series(c["T1"], c["dims"], c["ranks"], c["regime"], c["sigma"], c["seed"])
    if dtype == "f32":
        X = X.astype(np.float32)
    reqs = _script(c["T0"], c["T1"], 240, 7)
    tree = engine_tree(X[: c["T0"]], c["dims"], c["ranks"], c["B"], 4, 0.0, dtype)
    twin = engine_tree(X[: c["T0"]], c["dims"], c["ranks"], c["B"], 4, 0.0, dtype)
    srv = tk.Server(tree, max_batch=64)
    tickets = []
    for r in reqs:
        tickets.append(srv.submit_append(X[r[1]]) if r[0] == "a" else srv.submit_query(r[1], r[2]))
    got = [srv.wait(k, timeout=120.0) for k in tickets]
    st = srv.stats()
    srv.close()
    n_app = sum(1 for r in reqs if r[0] == "a")
    assert st["queries_done"] == len(reqs) - n_app and st["appends_done"] == n_app
    assert st["batches"] < st["queries_done"]            # the burst was batched
    assert st["mean_batch"] <= 64
    assert tree.T == twin.T + n_app == c["T1"]
    for r, g in zip(reqs, got):
        if r[0] == "a":
            assert g is None
            twin.append(X[r[1]])
        else:
            _same(dtype, X, r[1], r[2], g, twin.query(r[1], r[2]))
    tree.close()
    twin.close()


def test_concurrent_submitters_and_admission_limits():
    import paper_2501_06647_gb300 as tk
    c = CASES["f64"]
    X = series(c["T0"], c["dims"], c["ranks"], c["regime"], c["sigma"], c["seed"])
    tree = engine_tree(X, c["dims"], c["ranks"], c["B"], 4, 0.0, "f64")
    twin = engine_tree(X, c["dims"], c["ranks"], c["B"], 4, 0.0, "f64")
    srv = tk.Server(tree, max_batch=4)
    rng = np.random.default_rng(11)
    ranges = [(int(a), int(rng.integers(a + 1, c["T0"] + 1))) for a in rng.integers(0, c["T0"], 64)]
    results = [None] * len(ranges)

    def worker(w):
        mine = [(i, srv.submit_query(*ranges[i])) for i in range(w, len(ranges), 4)]
        for i, k in mine:
            results[i] = srv.wait(k, timeout=120.0)

    th = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    st = srv.stats()
    assert st["queries_done"] == len(ranges) and st["mean_batch"] <= 4
    # a range past the submitted end, before and after the append that makes it valid
    with pytest.raises(tk.TuckerError) as ei:
        srv.submit_query(0, c["T0"] + 1)
    assert ei.value.code == -2
    ka = srv.submit_append(X[-1])
    kq = srv.submit_query(0, c["T0"] + 1)
    srv.drain(timeout=120.0)
    assert srv.wait(ka, timeout=1.0) is None
    G, U, info = srv.wait(kq, timeout=1.0)
    assert U[0].shape[0] == c["T0"] + 1
    srv.close()
    for (ts, te), g in zip(ranges, results):
        _same("f64", X, ts, te, g, twin.query(ts, te))
    # an output budget smaller than one query is refused at submission
    small = tk.Server(twin, max_batch_out_elems=100)
    with pytest.raises(tk.TuckerError) as ei:
        small.submit_query(0, 50)
    assert ei.value.code == -8
    small.close()
    tree.close()
    twin.close()


def test_wait_times_out_and_the_ticket_stays_collectable():
    # A wait whose limit runs out returns TK_ERR_TIMEOUT and changes nothing:
    # the request still completes and is collected by a later wait.  The
    # server is kept busy by 600 queries in batches of 64 on a rank-16 tree,
    # so the last one cannot be answered within 0.1 ms of its submission.
    import paper_2501_06647_gb300 as tk
    w = synth.WORKLOADS["batched_r16"]
    T = 512
    X = synth.piecewise_tucker_regimes(T, w["dims"], w["ranks"], w["regime"], w["sigma"], w["seed"])
    tree = engine_tree(X, w["dims"], w["ranks"], w["B"], 20, 0.01, "f32")
    srv = tk.Server(tree, max_batch=64)
    Q = synth.query_ranges(T, 600, 77, "loguniform", 64, T)
    tickets = [srv.submit_query(int(a), int(b)) for a, b in Q]
    with pytest.raises(tk.TuckerError) as ei:
        srv.wait(tickets[-1], timeout=1e-4)
    assert ei.value.code == -9
    G, U, info = srv.wait(tickets[-1], timeout=120.0)
    assert U[0].shape[0] == int(Q[-1][1] - Q[-1][0]) and info["iters"] >= 1
    for k in tickets[:-1]:
        srv.wait(k, timeout=120.0)
    assert srv.stats()["queries_done"] == len(Q)
    srv.close()
    tree.close()
