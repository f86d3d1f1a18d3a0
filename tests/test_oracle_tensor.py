"""Pins for oracle.tensor against Appendix A's definitions, written as loops."""
import itertools

import numpy as np

from oracle import tensor


def _rand(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def test_vec_index_formula():
    D = (3, 4, 2)
    X = _rand(D)
    v = tensor.vec(X)
    for idx in itertools.product(*[range(d) for d in D]):
        j = sum(idx[n] * int(np.prod(D[n + 1:])) for n in range(len(D)))
        assert v[j] == X[idx]


def test_unfold_is_stack_of_vectorized_slices():
    D = (3, 4, 2, 5)
    X = _rand(D, 1)
    for n in range(len(D)):
        M = tensor.unfold(X, n)
        assert M.shape == (D[n], int(np.prod(D)) // D[n])
        for i in range(D[n]):
            sl = [slice(None)] * len(D)
            sl[n] = i
            # row i = vec of the slice with the n-th index fixed (remaining modes in order)
            expect = [X[tuple(list(rest[:n]) + [i] + list(rest[n:]))]
                      for rest in itertools.product(*[range(D[m]) for m in range(len(D)) if m != n])]
            assert np.array_equal(M[i], np.array(expect))
        assert np.array_equal(tensor.fold(M, n, D), X)


def test_mode_product_elementwise():
    D = (3, 4, 2)
    X = _rand(D, 2)
    U = _rand((5, 4), 3)
    Y = tensor.mode_product(X, U, 1)
    assert Y.shape == (3, 5, 2)
    for a, b, c in itertools.product(range(3), range(5), range(2)):
        assert abs(Y[a, b, c] - sum(U[b, j] * X[a, j, c] for j in range(4))) < 1e-12


def test_kronecker_form_of_mode1_matricization():
    # Section 5.2 rewrites mat_1(H x_1 A x_2 B x_3 C) = A mat_1(H) (B kron C)^T under row-major vec.
    H = _rand((2, 3, 4), 4)
    A, B, C = _rand((5, 2), 5), _rand((6, 3), 6), _rand((7, 4), 7)
    Y = tensor.multi_mode_product(H, [A, B, C])
    lhs = tensor.unfold(Y, 0)
    rhs = A @ tensor.unfold(H, 0) @ np.kron(B, C).T
    assert np.allclose(lhs, rhs, atol=1e-12)
    # and mode 2: mat_2(Y) = B mat_2(H) (A kron C)^T
    assert np.allclose(tensor.unfold(Y, 1), B @ tensor.unfold(H, 1) @ np.kron(A, C).T, atol=1e-12)


def test_reverse_associativity():
    # footnote of Section 5.1: Z x_n A x_n B = Z x_n (B A)
    Z = _rand((3, 4, 2), 8)
    A, B = _rand((5, 4), 9), _rand((6, 5), 10)
    assert np.allclose(tensor.mode_product(tensor.mode_product(Z, A, 1), B, 1),
                       tensor.mode_product(Z, B @ A, 1), atol=1e-12)


def test_frobenius():
    X = _rand((3, 4, 5), 11)
    assert abs(tensor.frob(X) - np.sqrt(sum(x * x for x in X.ravel()))) < 1e-12


def test_leading_left_singular_vectors_span():
    rng = np.random.default_rng(12)
    Q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    s = np.array([10, 9, 8, 1, 0.5, 0.1, 0.01, 0.001])
    M = Q @ np.diag(s) @ np.linalg.qr(rng.standard_normal((8, 8)))[0]
    U = tensor.leading_left_singular_vectors(M, 3)
    P = U @ U.T
    assert np.allclose(P, Q[:, :3] @ Q[:, :3].T, atol=1e-12)
