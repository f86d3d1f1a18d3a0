"""Partial-hit approximation (Eq. (partial-tucker)) and Stitch (Algorithm 2).

TEST INFRASTRUCTURE ONLY: a literal FP64 restatement of Section 5, which forms
the matricizations Z^(n) explicitly, exactly as Eq. (stitch-temp-2) and
Eq. (stitch-nontemp-3) write them, and takes LAPACK SVDs of them.

A hit decomposition is a pair (H, V): core H (q_1 x ... x q_p) and factors
V[0] (temporal, l x q_1, orthonormal columns) and V[n] (D_n x q_n, orthonormal).

Readings of what the paper leaves open:
  * the offsets t_i of Algorithm 2 are prefix sums of the CLIPPED lengths
    |[T_s,T_e) cap [sigma_v, tau_v)|, so that t_s = L;
  * "randomly initialize U^(2..p)" is replaced by default by the implicit
    HOSVD of the stitched tensor: U^(n) = leading eigenvectors of
    sum_i V_i^(n) mat_n(H_i) mat_n(H_i)^T V_i^(n)T  (= mat_n(Y~) mat_n(Y~)^T
    because every V_i^(m) has orthonormal columns); init="random" draws them
    from the seeded counter-based generator of ``rng`` instead;
  * "reshape Z^(p) into r_1 x ... x r_{p-1} x D_p" is read as folding Z^(p) as
    the mode-p matricization, so G = fold_p(U^(p)T Z^(p)) = Y~ x_n U^(n)T;
  * the stopping quantity is e = sqrt(max(0, 1 - ||G||^2/||Y~||^2)) with
    ||Y~||^2 = sum_i ||H_i||^2, and the stop rule is the one of ``hooi``;
  * output ranks are clamped so that no requested factor exceeds the rank the
    stitched tensor can have: r_n' = min(r_n, D_n, sum_i min(q_{i,n},
    prod_{m!=n} q_{i,m})) (D_1 = L), then the fixpoint of ``hooi.clamp_ranks``.
"""
import numpy as np

from .tensor import unfold, fold, mode_product, frob, leading_left_singular_vectors
from .hooi import stop_error
from .rng import seeded_factors


def partial_hit(H, V, row_lo, row_hi):
    """Eq. (partial-tucker): restrict node (H, V) to temporal rows [row_lo, row_hi).

    The rows of V[0] are sliced and factored by a reduced QR (LAPACK), slice =
    Q R; the core becomes H x_1 R and the temporal factor becomes Q.
    """
    S = np.asarray(V[0], dtype=np.float64)[row_lo:row_hi]
    Q, R = np.linalg.qr(S, mode="reduced")
    H2 = mode_product(H, R, 0)
    return H2, [Q] + [np.asarray(v, dtype=np.float64) for v in V[1:]]


def stitched_ranks(hits, dims, ranks):
    """Output-rank clamp for a stitch of ``hits`` (see module docstring)."""
    p = len(ranks)
    L = sum(h[1][0].shape[0] for h in hits)
    ext = [L] + [int(d) for d in dims]
    cap = []
    for n in range(p):
        tot = 0
        for H, _ in hits:
            q = H.shape
            prod = 1
            for m in range(p):
                if m != n:
                    prod *= q[m]
            tot += min(q[n], prod)
        cap.append(tot)
    r = [int(min(ranks[n], ext[n], cap[n])) for n in range(p)]
    changed = True
    while changed:
        changed = False
        for n in range(p):
            prod = 1
            for m in range(p):
                if m != n:
                    prod *= r[m]
            if r[n] > prod:
                r[n] = prod
                changed = True
    return r


def init_factors(hits, r):
    """Implicit HOSVD initialization of U^(2..p) (reading of Algorithm 2's init)."""
    p = len(r)
    U = [None] * p
    for n in range(1, p):
        D = hits[0][1][n].shape[0]
        S = np.zeros((D, D))
        for H, V in hits:
            Hn = unfold(H, n)
            S += V[n] @ (Hn @ Hn.T) @ V[n].T
        w, E = np.linalg.eigh(S)
        order = np.argsort(-w, kind="stable")
        U[n] = E[:, order[: r[n]]].copy()
    return U


def temporal_matricization(hits, U):
    """Eq. (stitch-temp-2): Z^(1) = [mat_1(H_i x_1 V_i^(1) x_m (U^(m)T V_i^(m)))]_i stacked."""
    p = len(U)
    blocks = []
    for H, V in hits:
        Y = mode_product(H, V[0], 0)
        for m in range(1, p):
            Y = mode_product(Y, U[m].T @ V[m], m)
        blocks.append(unfold(Y, 0))
    return np.vstack(blocks)


def nontemporal_matricization(hits, U, n, offsets):
    """Eq. (stitch-nontemp-3): Z^(n) = sum_i mat_n(H_i x_1 (U^(1)_[t_{i-1},t_i)T V_i^(1))
    x_{m != 1,n} (U^(m)T V_i^(m)) x_n V_i^(n))."""
    p = len(U)
    Z = None
    for i, (H, V) in enumerate(hits):
        U1i = U[0][offsets[i]:offsets[i + 1]]
        Y = mode_product(H, U1i.T @ V[0], 0)
        for m in range(1, p):
            if m == n:
                Y = mode_product(Y, V[n], n)
            else:
                Y = mode_product(Y, U[m].T @ V[m], m)
        Zi = unfold(Y, n)
        Z = Zi if Z is None else Z + Zi
    return Z


def stitch(hits, ranks, max_iter=20, tol=0.01, init="hosvd", seed=0):
    """Algorithm 2 (Stitch) on the hit decompositions, in time order.

    ``ranks`` must already be the output ranks (see ``stitched_ranks``).
    init: "hosvd" (the implicit HOSVD start) or "random" (Algorithm 2's
    random U^(2..p), drawn by ``rng.seeded_factors`` from ``seed``).
    Returns (G, U, iters, errs).
    """
    p = len(ranks)
    r = [int(x) for x in ranks]
    hits = [(np.asarray(H, dtype=np.float64), [np.asarray(v, dtype=np.float64) for v in V])
            for H, V in hits]
    lengths = [V[0].shape[0] for _, V in hits]
    offsets = [0]
    for l in lengths:
        offsets.append(offsets[-1] + l)
    ynorm2 = sum(frob(H) ** 2 for H, _ in hits)
    if init == "random":
        U = seeded_factors([hits[0][1][n].shape[0] for n in range(1, p)], r, seed)
    elif init == "hosvd":
        U = init_factors(hits, r)
    else:
        raise ValueError(init)
    e_prev = np.inf
    errs = []
    G = None
    it = 0
    for it in range(1, max_iter + 1):
        Z1 = temporal_matricization(hits, U)
        U[0] = leading_left_singular_vectors(Z1, r[0])
        Zn = None
        for n in range(1, p):
            Zn = nontemporal_matricization(hits, U, n, offsets)
            U[n] = leading_left_singular_vectors(Zn, r[n])
        if p == 1:
            Zn = Z1
        gshape = list(r)
        G = fold(U[p - 1].T @ Zn, p - 1, gshape)
        e = stop_error(frob(G) ** 2, ynorm2)
        errs.append(e)
        if tol > 0 and abs(e - e_prev) < tol:
            break
        e_prev = e
    return G, U, it, errs


def materialize_stitched(hits):
    """Y~ = [Y~_1; ...; Y~_s] as a dense array (for brute-force checks on tiny inputs)."""
    blocks = []
    for H, V in hits:
        Y = H
        for m, v in enumerate(V):
            Y = mode_product(Y, v, m)
        blocks.append(Y)
    return np.concatenate(blocks, axis=0)
