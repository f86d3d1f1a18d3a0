"""Dense Tucker-ALS (HOOI) of Section 2, in FP64 NumPy.  Test infrastructure only.

Section 2: Tucker decomposition minimizes ||G x_1 U1 ... x_p Up - X||_F^2
(Eq. (tuckerals)); Tucker-ALS updates one factor at a time, U^(n) being the r_n
leading left singular vectors of mat_n(X x_{m!=n} U^(m)T) (Eq. (als-mat)), and
the optimal core is X x_n U^(n)T over all modes.

Readings of what the paper leaves open:
  * ranks are clamped per mode: r_n' = min(r_n, D_n), then repeatedly
    r_n' = min(r_n', prod_{m!=n} r_m') until nothing changes, so that every
    matricization has at least r_n' columns;
  * initialization is HOSVD: U^(n), n >= 2, are the leading left singular
    vectors of mat_n(X) (U^(1) is computed first inside the loop);
  * one iteration updates modes 1..p in order (Gauss-Seidel), then the core;
  * the stopping quantity is e = sqrt(max(0, 1 - ||G||^2/||X||^2)); the loop
    stops after ``max_iter`` iterations, or earlier once |e_k - e_{k-1}| < tol
    (e_0 = +inf, so at least two iterations run when tol > 0); tol <= 0 means
    exactly ``max_iter`` iterations.  Section 8.1 uses max_iter=20, tol=0.01.
"""
import numpy as np

from .tensor import unfold, mode_product, multi_mode_product, frob, leading_left_singular_vectors


def clamp_ranks(shape, ranks):
    """Per-mode rank clamp (reading of the paper's silence on r_n > D_n)."""
    r = [int(min(int(a), int(b))) for a, b in zip(ranks, shape)]
    changed = True
    while changed:
        changed = False
        for n in range(len(r)):
            prod = 1
            for m in range(len(r)):
                if m != n:
                    prod *= r[m]
            if r[n] > prod:
                r[n] = prod
                changed = True
    return r


def stop_error(gnorm2, xnorm2):
    """Relative residual implied by an orthogonal Tucker model: sqrt(1 - |G|^2/|X|^2)."""
    if xnorm2 <= 0.0:
        return 0.0
    return float(np.sqrt(max(0.0, 1.0 - gnorm2 / xnorm2)))


def tucker_als(X, ranks, max_iter=20, tol=0.01):
    """Tucker-ALS of Section 2 on a dense tensor X (temporal mode first).

    Returns (G, U, iters, errs) with U[n] of shape D_n x r_n' (orthonormal
    columns), G of shape r_1' x ... x r_p', ``iters`` the number of ALS
    iterations run and ``errs`` the stopping quantity after each iteration.
    """
    X = np.asarray(X, dtype=np.float64)
    p = X.ndim
    r = clamp_ranks(X.shape, ranks)
    U = [None] * p
    for n in range(1, p):
        U[n] = leading_left_singular_vectors(unfold(X, n), r[n])
    xnorm2 = frob(X) ** 2
    e_prev = np.inf
    errs = []
    G = None
    it = 0
    for it in range(1, max_iter + 1):
        for n in range(p):
            Y = X
            for m in range(p):
                if m != n:
                    Y = mode_product(Y, U[m].T, m)
            U[n] = leading_left_singular_vectors(unfold(Y, n), r[n])
        G = multi_mode_product(X, [u.T for u in U])
        e = stop_error(frob(G) ** 2, xnorm2)
        errs.append(e)
        if tol > 0 and abs(e - e_prev) < tol:
            break
        e_prev = e
    return G, U, it, errs
