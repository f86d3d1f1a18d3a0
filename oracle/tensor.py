"""Basic tensor operations of Appendix A, in FP64 NumPy.  Test infrastructure only.

Appendix A fixes the conventions used everywhere else:
  * indices start at 0;
  * vec(X) puts entry X[i_1..i_p] at position j = sum_n i_n * prod_{m>n} D_m,
    i.e. row-major (C) order;
  * mat_n(X) is D_n x (prod_{m!=n} D_m); its row i is vec of the slice with
    the n-th index fixed to i (the remaining modes keep their order);
  * the mode-n product G x_n U satisfies mat_n(G x_n U) = U mat_n(G);
  * ||X||_F is the square root of the sum of squared entries.
"""
import numpy as np


def vec(X):
    """Appendix A vectorization: row-major flattening."""
    return np.asarray(X, dtype=np.float64).reshape(-1)


def unfold(X, n):
    """Appendix A mode-n matricization mat_n(X)."""
    X = np.asarray(X)
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def fold(M, n, shape):
    """Inverse of ``unfold``: the tensor of ``shape`` whose mat_n is M."""
    shape = tuple(int(s) for s in shape)
    rest = shape[:n] + shape[n + 1:]
    return np.moveaxis(np.asarray(M).reshape((shape[n],) + rest), 0, n)


def mode_product(X, U, n):
    """Appendix A mode-n product X x_n U, defined by mat_n(X x_n U) = U mat_n(X)."""
    X = np.asarray(X, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    shape = list(X.shape)
    shape[n] = U.shape[0]
    return fold(U @ unfold(X, n), n, shape)


def multi_mode_product(X, mats):
    """X x_0 mats[0] x_1 mats[1] ...; a ``None`` entry skips that mode."""
    Y = np.asarray(X, dtype=np.float64)
    for n, U in enumerate(mats):
        if U is not None:
            Y = mode_product(Y, U, n)
    return Y


def frob(X):
    """Appendix A Frobenius norm."""
    return float(np.sqrt(np.sum(np.square(np.asarray(X, dtype=np.float64)))))


def leading_left_singular_vectors(M, r):
    """The r leading left singular vectors of M (Section 2, Eq. (als-mat)).

    LAPACK's SVD is the library step (divide and conquer, gesdd; if that
    driver reports non-convergence, which some LAPACK builds do on rare
    inputs, the same SVD is taken with the QR-iteration driver gesvd).  Only
    the spanned subspace is unique.
    """
    M = np.asarray(M, dtype=np.float64)
    try:
        U, _, _ = np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:
        import scipy.linalg
        U, _, _ = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
    return U[:, :r].copy()


def reconstruct(G, U):
    """G x_0 U[0] x_1 U[1] ... : the tensor a Tucker decomposition stands for."""
    return multi_mode_product(G, U)
