"""One-dimensional building blocks of the oracle (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

* Gauss-Lobatto-Legendre points and weights: the quadrature the paper's
  Python example uses (§3.5, Listing lst:python, ``PointsType.GaussLobattoLegendre``).
* Jacobi polynomials P_n^{(alpha,beta)} in the standard (Szego) normalisation
  P_n^{(a,b)}(1) = binom(n+a, n); the paper writes P^{1,1}_{p-1} without
  fixing a normalisation (§2.1 display of phi_p), this is the reading used.
* The modified C0 ("modal") basis phi_p of §2.1, in the paper's index order:
  p = 0 left vertex, 0 < p < P bubbles, p = P right vertex.
* Lagrange interpolation through arbitrary nodes, evaluated with its
  derivative at arbitrary points (used for the iso-parametric geometry and for
  the collocation derivative of PhysDeriv).
"""
import numpy as np


def legendre(N, x):
    """P_N(x) and P_N'(x) by the three-term Legendre recurrence.

    (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1};  P_N' from
    (1-x^2) P_N' = N (P_{N-1} - x P_N), with the endpoint values
    P_N'(+-1) = (+-1)^{N-1} N(N+1)/2 substituted where 1-x^2 = 0.
    """
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for n in range(1, N):
        p_prev, p = p, ((2 * n + 1) * x * p - n * p_prev) / (n + 1)
    one_m_x2 = 1.0 - x * x
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = N * (p_prev - x * p) / one_m_x2
    end = np.abs(one_m_x2) < 1e-300
    dp = np.where(end, np.sign(x) ** (N - 1) * N * (N + 1) / 2.0, dp)
    return p, dp


def gll(Q):
    """Q Gauss-Lobatto-Legendre points (ascending) and weights on [-1, 1].

    The end points are -1 and 1; the Q-2 interior points are the roots of
    P_{Q-1}'.  They are found by Newton's method on f = P_N' (N = Q-1) with
    f' = P_N'' taken from Legendre's equation
    (1-x^2) P'' = 2x P' - N(N+1) P, starting from the Chebyshev-Gauss-Lobatto
    points.  Weights: w_i = 2 / (N (N+1) P_N(xi_i)^2).
    """
    if Q < 2:
        raise ValueError("GLL needs Q >= 2")
    N = Q - 1
    x = -np.cos(np.pi * np.arange(Q) / N)
    interior = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(N, interior)
        d2p = (2.0 * interior * dp - N * (N + 1) * p) / (1.0 - interior ** 2)
        step = dp / d2p
        interior -= step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    x[1:-1] = interior
    x[0], x[-1] = -1.0, 1.0
    # make the point set exactly symmetric (the Newton iterates agree to
    # rounding; symmetrising removes the last-bit asymmetry)
    x = 0.5 * (x - x[::-1])
    p, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * p ** 2)
    return x, w


def jacobi(n, alpha, beta, x):
    """P_n^{(alpha,beta)}(x), standard normalisation, by the three-term recurrence.

    P_0 = 1, P_1 = ((alpha+beta+2) x + alpha - beta) / 2 and for m >= 2
    2m(m+a+b)(2m+a+b-2) P_m = (2m+a+b-1)((2m+a+b)(2m+a+b-2) x + a^2 - b^2) P_{m-1}
                               - 2(m+a-1)(m+b-1)(2m+a+b) P_{m-2}.
    """
    x = np.asarray(x, dtype=np.float64)
    if n < 0:
        return np.zeros_like(x)
    a, b = float(alpha), float(beta)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = 0.5 * ((a + b + 2.0) * x + a - b)
    for m in range(2, n + 1):
        c = 2.0 * m + a + b
        lhs = 2.0 * m * (m + a + b) * (c - 2.0)
        t1 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b)
        t2 = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c
        p0, p1 = p1, (t1 * p1 - t2 * p0) / lhs
    return p1


def jacobi_deriv(n, alpha, beta, x):
    """d/dx P_n^{(a,b)} = (n+a+b+1)/2 * P_{n-1}^{(a+1,b+1)}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + alpha + beta + 1.0) * jacobi(n - 1, alpha + 1, beta + 1, x)


def modified_basis(P, x):
    """Values phi_p(x) of the order-P modified C0 basis, shape (len(x), P+1).

    phi_0 = (1-x)/2, phi_p = (1-x)/2 (1+x)/2 P^{1,1}_{p-1}(x) for 0<p<P,
    phi_P = (1+x)/2 (§2.1).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty((x.size, P + 1))
    left, right = 0.5 * (1.0 - x), 0.5 * (1.0 + x)
    out[:, 0] = left
    out[:, P] = right
    for p in range(1, P):
        out[:, p] = left * right * jacobi(p - 1, 1, 1, x)
    return out


def modified_basis_deriv(P, x):
    """Derivatives phi_p'(x), shape (len(x), P+1), by the product rule.

    d/dx[(1-x)(1+x)/4 J(x)] = -x/2 J(x) + (1-x^2)/4 J'(x).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty((x.size, P + 1))
    out[:, 0] = -0.5
    out[:, P] = 0.5
    for p in range(1, P):
        J = jacobi(p - 1, 1, 1, x)
        dJ = jacobi_deriv(p - 1, 1, 1, x)
        out[:, p] = -0.5 * x * J + 0.25 * (1.0 - x * x) * dJ
    return out


def lagrange(nodes, x):
    """Lagrange basis through ``nodes`` and its derivative, evaluated at ``x``.

    Returns (L, dL), each of shape (len(x), len(nodes)), with
    L[i, m] = prod_{k != m} (x_i - z_k) / (z_m - z_k) and dL its derivative
    by the product rule (sum over the dropped factor).
    """
    z = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = z.size
    L = np.ones((x.size, n))
    dL = np.zeros((x.size, n))
    for m in range(n):
        others = [k for k in range(n) if k != m]
        denom = np.prod([z[m] - z[k] for k in others])
        for k in others:
            L[:, m] *= x - z[k]
        for drop in others:
            term = np.ones(x.size)
            for k in others:
                if k != drop:
                    term *= x - z[k]
            dL[:, m] += term
        L[:, m] /= denom
        dL[:, m] /= denom
    return L, dL


def collocation_derivative(Q):
    """D[i, j] = l_j'(xi_i) on the Q GLL points (the collocation derivative)."""
    xi, _ = gll(Q)
    _, dL = lagrange(xi, xi)
    return dL
