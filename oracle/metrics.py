"""Accuracy metrics of Section 8.1, in FP64 NumPy.  Test infrastructure only.

Section 8.1 reports, per query, the relative error of a method A against
Tucker-ALS from scratch: ||X - Y_A||_F / ||X - Y_ALS||_F - 1.  We also report
the plain relative reconstruction error ||X - Y||_F / ||X||_F.
"""
import numpy as np

from .tensor import multi_mode_product, frob, reconstruct
from .hooi import tucker_als


def residual_norm(X, G, U):
    """||X - G x_n U^(n)||_F for orthonormal U, via ||X||^2 - 2<X x_n U^(n)T, G> + ||G||^2."""
    X = np.asarray(X, dtype=np.float64)
    P = multi_mode_product(X, [u.T for u in U])
    r2 = frob(X) ** 2 - 2.0 * float(np.sum(P * G)) + frob(G) ** 2
    return float(np.sqrt(max(0.0, r2)))


def residual_norm_dense(X, G, U):
    """Same quantity by materializing the reconstruction (tiny inputs only)."""
    return frob(np.asarray(X, dtype=np.float64) - reconstruct(G, U))


def relative_error(X, G, U):
    """||X - Y||_F / ||X||_F."""
    nx = frob(X)
    return residual_norm(X, G, U) / nx if nx > 0 else 0.0


def from_scratch(X, ranks, max_iter=20, tol=0.01):
    """Tucker-ALS on the raw subtensor (the paper's reference method, Section 8.2)."""
    return tucker_als(X, ranks, max_iter, tol)


def paper_relative_error(X, G, U, G_als, U_als):
    """Section 8.1 metric ||X - Y_A|| / ||X - Y_ALS|| - 1."""
    den = residual_norm(X, G_als, U_als)
    num = residual_norm(X, G, U)
    return num / den - 1.0 if den > 0 else float("inf") if num > 0 else 0.0


def principal_angle_max(A, B):
    """Largest principal angle between span(A) and span(B) (orthonormal columns),
    computed from sines: sigma_max((I - A A^T) B), which resolves tiny angles."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    R = B - A @ (A.T @ B)
    s = np.linalg.norm(R, 2) if R.size else 0.0
    return float(np.arcsin(min(1.0, s)))


def model_distance(Ga, Ua, Gb, Ub):
    """||Y_a - Y_b||_F for two orthogonal Tucker models of the same tensor shape.

    Per mode, a Householder QR [U_a, U_b] = Q [R_a, R_b] (exact to rounding at
    any rank) expresses both factors in one orthonormal basis Q, so
    ||Y_a - Y_b|| = ||G_a x_n R_a - G_b x_n R_b||: a small dense difference
    with no cancellation, accurate down to rounding of the tiny tensors.
    """
    Ra, Rb = [], []
    for ua, ub in zip(Ua, Ub):
        ua = np.asarray(ua, dtype=np.float64)
        ub = np.asarray(ub, dtype=np.float64)
        _, R = np.linalg.qr(np.hstack([ua, ub]), mode="reduced")
        Ra.append(R[:, :ua.shape[1]])
        Rb.append(R[:, ua.shape[1]:])
    A = multi_mode_product(np.asarray(Ga, dtype=np.float64), Ra)
    B = multi_mode_product(np.asarray(Gb, dtype=np.float64), Rb)
    return frob(A - B)
