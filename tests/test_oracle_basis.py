"""Pins of the oracle's 1D building blocks against closed forms and library routines.

Each check is independent of the code it tests: closed forms written out by
hand, scipy's Jacobi polynomials and Gauss-Legendre rule, numpy polynomial
fitting, and exactness properties of the quadrature.
"""
import numpy as np
import pytest
from numpy.polynomial import Polynomial
from scipy import special

from oracle import basis


def test_gll_small_closed_forms():
    x, w = basis.gll(2)
    np.testing.assert_allclose(x, [-1, 1], atol=0)
    np.testing.assert_allclose(w, [1, 1], rtol=1e-15)
    x, w = basis.gll(3)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    # Q = 4: interior points +-1/sqrt(5), weights 1/6, 5/6
    x, w = basis.gll(4)
    np.testing.assert_allclose(x, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], rtol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)


@pytest.mark.parametrize("Q", range(2, 13))
def test_gll_exactness_and_symmetry(Q):
    x, w = basis.gll(Q)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-14)
    np.testing.assert_allclose(w.sum(), 2.0, rtol=1e-14)
    # exact for degree <= 2Q-3 (closed form int x^k = 2/(k+1) for even k, 0 odd)
    for k in range(0, 2 * Q - 2):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, (Q, k)
    # and not for degree 2Q-2: the GLL remainder for f = x^{2N} (N = Q-1) is
    # int f - sum w f = -(N+1) N^3 2^{2N+1} ((N-1)!)^4 / ((2N+1) ((2N)!)^3) f^{(2N)},
    # f^{(2N)} = (2N)!  (Abramowitz & Stegun 25.4.32)
    N = Q - 1
    k = 2 * N
    from math import factorial
    rem = -(N + 1) * N ** 3 * 2.0 ** (2 * N + 1) * factorial(N - 1) ** 4 / (
        (2 * N + 1) * float(factorial(2 * N)) ** 2)
    err = 2.0 / (k + 1) - np.sum(w * x ** k)
    np.testing.assert_allclose(err, rem, rtol=1e-6)
    # interior points are the roots of P_{Q-1}' (scipy's Legendre polynomial)
    # (P_N' = N (x P_N - P_{N-1}) / (x^2 - 1) with scipy's Legendre values)
    if Q > 2:
        xi = x[1:-1]
        dP = N * (xi * special.eval_legendre(N, xi) - special.eval_legendre(N - 1, xi)) / (xi ** 2 - 1)
        np.testing.assert_allclose(dP, 0.0, atol=1e-12 * N * N)


def test_jacobi_closed_forms():
    x = np.linspace(-1, 1, 41)
    np.testing.assert_allclose(basis.jacobi(0, 1, 1, x), 1.0)
    np.testing.assert_allclose(basis.jacobi(1, 1, 1, x), 2 * x, atol=1e-15)
    np.testing.assert_allclose(basis.jacobi(2, 1, 1, x), (15 * x ** 2 - 3) / 4, atol=1e-14)
    for n in range(0, 12):
        for (a, b) in [(1, 1), (2, 2), (0, 0), (1, 2)]:
            np.testing.assert_allclose(basis.jacobi(n, a, b, x), special.eval_jacobi(n, a, b, x),
                                       rtol=1e-12, atol=1e-12)
    # P^{1,1}_{n-1} = 2/(n+1) P_n'
    for n in range(1, 10):
        dP = special.legendre(n).deriv()
        np.testing.assert_allclose(basis.jacobi(n - 1, 1, 1, x), 2.0 / (n + 1) * dP(x), atol=1e-11)


def test_jacobi_orthogonality():
    xg, wg = special.roots_legendre(40)
    wt = wg * (1 - xg) * (1 + xg)
    V = np.stack([basis.jacobi(n, 1, 1, xg) for n in range(10)], axis=1)
    Gm = V.T @ (wt[:, None] * V)
    off = Gm - np.diag(np.diag(Gm))
    assert np.max(np.abs(off)) < 1e-12
    assert np.all(np.diag(Gm) > 0)


def test_jacobi_derivative():
    x = np.linspace(-0.99, 0.99, 23)
    for n in range(1, 9):
        fit = Polynomial.fit(x, special.eval_jacobi(n, 1, 1, x), n).deriv()
        np.testing.assert_allclose(basis.jacobi_deriv(n, 1, 1, x), fit(x), rtol=1e-9, atol=1e-9)


def test_modified_basis_identities():
    x = np.linspace(-1, 1, 37)
    # P = 1: hat functions
    B = basis.modified_basis(1, x)
    np.testing.assert_allclose(B[:, 0], (1 - x) / 2)
    np.testing.assert_allclose(B[:, 1], (1 + x) / 2)
    for P in range(1, 10):
        B = basis.modified_basis(P, x)
        np.testing.assert_allclose(B[:, 0] + B[:, P], 1.0, atol=1e-15)
        ends = basis.modified_basis(P, np.array([-1.0, 1.0]))
        np.testing.assert_allclose(ends[:, 1:P], 0.0, atol=1e-15)
        np.testing.assert_allclose(ends[0, [0, P]], [1, 0])
        np.testing.assert_allclose(ends[1, [0, P]], [0, 1])
        Bm = basis.modified_basis(P, -x)
        for p in range(1, P):
            np.testing.assert_allclose(Bm[:, p], (-1) ** (p - 1) * B[:, p], atol=1e-14)
        np.testing.assert_allclose(Bm[:, 0], B[:, P], atol=1e-15)
        # bubble p equals (1-x)(1+x)/4 times scipy's Jacobi polynomial
        for p in range(1, P):
            np.testing.assert_allclose(B[:, p], (1 - x) * (1 + x) / 4 * special.eval_jacobi(p - 1, 1, 1, x),
                                       atol=1e-13)


def test_modified_basis_derivative():
    x = np.linspace(-1, 1, 29)
    for P in range(1, 10):
        B = basis.modified_basis(P, x)
        dB = basis.modified_basis_deriv(P, x)
        for p in range(P + 1):
            fit = Polynomial.fit(x, B[:, p], P).deriv()
            np.testing.assert_allclose(dB[:, p], fit(x), atol=1e-10)


def test_collocation_derivative_closed_form():
    """Textbook GLL differentiation matrix:
    D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) (i != j), D_00 = -N(N+1)/4,
    D_NN = N(N+1)/4, other diagonal entries 0."""
    for Q in range(2, 12):
        N = Q - 1
        x, _ = basis.gll(Q)
        LN = special.eval_legendre(N, x)
        Dref = np.zeros((Q, Q))
        for i in range(Q):
            for j in range(Q):
                if i != j:
                    Dref[i, j] = LN[i] / (LN[j] * (x[i] - x[j]))
        Dref[0, 0] = -N * (N + 1) / 4
        Dref[N, N] = N * (N + 1) / 4
        D = basis.collocation_derivative(Q)
        np.testing.assert_allclose(D, Dref, atol=1e-12 * max(1, N * N))
        # exact on polynomials of degree <= Q-1
        for k in range(Q):
            np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) if k else 0 * x,
                                       atol=1e-11 * N * N)


def test_lagrange_interpolates():
    z, _ = basis.gll(6)
    L, dL = basis.lagrange(z, z)
    np.testing.assert_allclose(L, np.eye(6), atol=1e-15)
    x = np.linspace(-1, 1, 17)
    L, dL = basis.lagrange(z, x)
    np.testing.assert_allclose(L.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dL.sum(axis=1), 0.0, atol=1e-12)
    f = 3 * z ** 5 - z ** 2 + 0.5
    np.testing.assert_allclose(L @ f, 3 * x ** 5 - x ** 2 + 0.5, atol=1e-13)
    np.testing.assert_allclose(dL @ f, 15 * x ** 4 - 2 * x, atol=1e-12)
