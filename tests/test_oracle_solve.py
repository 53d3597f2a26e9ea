"""Pins of the oracle's assembly, solvers and adjoint.

* PCG against a dense Cholesky solve of the explicitly assembled matrix.
* Assembly invariants: C0 continuity of the assembled field, global DOF count.
* Manufactured periodic solution u* = sin(2 pi x) sin(2 pi y) sin(2 pi z):
  the error decreases exponentially as the order P grows.
* Adjoint gradients against brute-force central differences (the loss is
  quadratic in each argument, so differences are exact up to rounding).
"""
import numpy as np
import pytest
from scipy import linalg

from oracle import adjoint, geometry, operators, solve


def test_assembly_map_counts_and_continuity():
    for dim, N, P in [(2, 3, 2), (3, 2, 3)]:
        mesh = geometry.StructuredMesh(dim, N, P, amp=0.05)
        l2g = solve.local_to_global(mesh)
        ng = solve.n_global(mesh)
        assert ng == (N * P) ** dim
        assert set(np.unique(l2g)) == set(range(ng))
        # interior (bubble-only) modes appear once; vertices 2^dim times
        counts = np.bincount(l2g, minlength=ng)
        assert counts.max() == 2 ** dim and counts.min() == 1
        # a global field is continuous across element faces: evaluate the
        # gathered local expansions at the shared face quadrature points
        rng = np.random.default_rng(0)
        xg = rng.uniform(-1, 1, ng)
        u = operators.bwd_trans(mesh, xg[l2g])
        Q = P + 2
        nq = Q ** dim
        for e in range(mesh.E):
            pos = mesh.element_index(e)
            nb = ((pos[0] + 1) % N) + N * pos[1] + (N * N * pos[2] if dim == 3 else 0)
            ue = u[e * nq:(e + 1) * nq].reshape((Q,) * dim)
            un = u[nb * nq:(nb + 1) * nq].reshape((Q,) * dim)
            np.testing.assert_allclose(ue[..., -1], un[..., 0], atol=1e-13)


@pytest.mark.parametrize("dim,N,P", [(2, 2, 3), (3, 2, 2), (3, 2, 3)])
def test_pcg_matches_dense_cholesky(dim, N, P):
    mesh = geometry.StructuredMesh(dim, N, P, amp=0.05)
    l2g = solve.local_to_global(mesh)
    A = solve.assembled_matrix(mesh, l2g)
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    rng = np.random.default_rng(2)
    b = rng.uniform(-1, 1, A.shape[0])
    x_ref = linalg.cho_solve(linalg.cho_factor(A), b)
    diag = solve.jacobi_diagonal(mesh, l2g)
    np.testing.assert_allclose(diag, np.diag(A), rtol=1e-13)
    x, it, rel = solve.pcg(lambda v: solve.apply_assembled(mesh, l2g, v), b, diag, tol=1e-13)
    assert rel <= 1e-13
    np.testing.assert_allclose(x, x_ref, atol=1e-12 * np.abs(x_ref).max())
    np.testing.assert_allclose(A @ x, b, atol=1e-11)


def test_manufactured_solution_converges_spectrally():
    errs = []
    # 3^3 elements: on 2^3 elements sin(2 pi x) is even about every element
    # centre and odd orders add nothing, which gives a staircase instead
    for P in range(2, 8):
        mesh = geometry.StructuredMesh(3, 3, P, amp=0.05)
        l2g = solve.local_to_global(mesh)
        rhs, u_star = solve.manufactured_rhs(mesh, l2g)
        diag = solve.jacobi_diagonal(mesh, l2g)
        x, it, rel = solve.pcg(lambda v: solve.apply_assembled(mesh, l2g, v), rhs, diag, tol=1e-12)
        u = operators.bwd_trans(mesh, x[l2g])
        errs.append(np.abs(u - u_star).max())
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0), errs
    slope = np.polyfit(np.arange(2, 8), np.log(errs), 1)[0]
    assert slope < -1.0, (slope, errs)       # exponential decay in P
    assert errs[-1] < 1e-4


def test_adjoint_against_finite_differences():
    mesh = geometry.StructuredMesh(3, 2, 3, amp=0.05)
    rng = np.random.default_rng(4)
    nl, nq = mesh.coef_off[-1], mesh.quad_off[-1]
    u = rng.uniform(-1, 1, nl)
    f = rng.uniform(-1, 1, nl)
    lam = 1.0 + 0.5 * rng.uniform(-1, 1, nq)
    kap = 1.0 + 0.3 * rng.uniform(-1, 1, nq)
    L0, gu, gl, gk = adjoint.gradients(mesh, u, f, lam, kap)
    np.testing.assert_allclose(L0, adjoint.loss(mesh, u, f, lam, kap), rtol=1e-15)
    h = 1e-6
    for idx in rng.choice(nl, 6, replace=False):
        e = np.zeros(nl); e[idx] = h
        fd = (adjoint.loss(mesh, u + e, f, lam, kap) - adjoint.loss(mesh, u - e, f, lam, kap)) / (2 * h)
        np.testing.assert_allclose(gu[idx], fd, rtol=1e-7, atol=1e-9 * abs(L0))
    for idx in rng.choice(nq, 6, replace=False):
        e = np.zeros(nq); e[idx] = h
        fd = (adjoint.loss(mesh, u, f, lam + e, kap) - adjoint.loss(mesh, u, f, lam - e, kap)) / (2 * h)
        np.testing.assert_allclose(gl[idx], fd, rtol=1e-6, atol=1e-9 * abs(L0))
        fd = (adjoint.loss(mesh, u, f, lam, kap + e) - adjoint.loss(mesh, u, f, lam, kap - e)) / (2 * h)
        np.testing.assert_allclose(gk[idx], fd, rtol=1e-6, atol=1e-9 * abs(L0))
