"""GPU parity of the assembled solve (Jacobi-PCG: FP64, FP32-inner with FP64
refinement, FP32 with reliable updates) against the oracle, plus the error
paths of the solver."""
import numpy as np
import pytest
import torch
from scipy import linalg

import paper_1906_03489_gb300 as spx
from oracle import operators, solve
from paper_1906_03489_gb300 import mesh, synth

from _cases import Case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def manufactured_rhs_gpu(c, l2g, ng, lam=1.0):
    """Assembled IProduct of f* = (lam + 4 pi^2 d) u*, u* = prod sin(2 pi x_m), on the GPU."""
    d = c.dim
    Q = int(c.plan.orders[0]) + 2
    X = c.g["xq"].reshape(c.plan.E, d, Q ** d)
    u_star = torch.prod(torch.sin(2 * np.pi * X), dim=1).reshape(-1).contiguous()
    f_star = (lam + 4 * np.pi ** 2 * d) * u_star
    return spx.assemble(c.plan, l2g, spx.iproduct(c.plan, f_star), ng), u_star


@pytest.mark.parametrize("dim,N,P", [(3, 2, 3), (2, 3, 4), (3, 3, 2)])
@pytest.mark.parametrize("precision", ["f64", "f32_refine", "f32_reliable"])
def test_solve_matches_dense_cholesky(dim, N, P, precision):
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    A = solve.assembled_matrix(c.om, solve.local_to_global(c.om))
    b = synth.uniform(synth.rng(31), ng)
    x_ref = linalg.cho_solve(linalg.cho_factor(A), b)
    x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, torch.tensor(b, device="cuda"), tol=1e-12, precision=precision,
                           check_every=5)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    assert rel_err(x, x_ref) <= 1e-10
    # the residual the solver reports is the true one (up to the rounding of
    # recomputing it on the host at the 1e-12 level)
    true_res = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert true_res <= 2e-12 and abs(true_res - info["rel_residual"]) <= 1e-13


@pytest.mark.parametrize("precision", ["f64", "f32_refine", "f32_reliable"])
def test_manufactured_solution_matches_oracle(precision):
    dim, N, P = 3, 4, 4
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    rhs, u_star = manufactured_rhs_gpu(c, l2g, ng)
    ol2g = solve.local_to_global(c.om)
    orhs, ou_star = solve.manufactured_rhs(c.om, ol2g)
    assert rel_err(rhs, orhs) <= 1e-12
    assert rel_err(u_star, ou_star) <= 1e-12
    x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, rhs, tol=1e-12, precision=precision)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    diag = solve.jacobi_diagonal(c.om, ol2g)
    xo, _, _ = solve.pcg(lambda v: solve.apply_assembled(c.om, ol2g, v), orhs, diag, tol=1e-12)
    assert rel_err(x, xo) <= 1e-8
    # discretisation error against u* equals the oracle's
    u = spx.bwd_trans(c.plan, spx.gather(c.plan, l2g, x)).cpu().numpy()
    uo = operators.bwd_trans(c.om, xo[ol2g])
    err, erro = np.abs(u - u_star.cpu().numpy()).max(), np.abs(uo - ou_star).max()
    assert abs(err - erro) <= 1e-8 and err < 1e-2


def test_graph_and_eager_are_bitwise_equal():
    dim, N, P = 3, 3, 3
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    b = torch.tensor(synth.uniform(synth.rng(32), ng), device="cuda")
    for precision in ("f64", "f32_refine", "f32_reliable"):
        xg, ig = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision=precision, use_graph=True, check_every=7)
        xe, ie = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision=precision, use_graph=False, check_every=7)
        assert torch.equal(xg, xe)
        assert ig["iters"] == ie["iters"]


def test_not_converged_and_nonfinite_are_reported():
    dim, N, P = 3, 3, 3
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    b = torch.tensor(synth.uniform(synth.rng(33), ng), device="cuda")
    x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f64", maxit=3, raise_on_fail=False)
    assert info["status"] == 4 and info["iters"] == 3 and info["rel_residual"] > 1e-10
    bn = b.clone()
    bn[3] = float("nan")                                   # poisoned input, injected on the host side
    x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, bn, tol=1e-10, precision="f64", raise_on_fail=False)
    assert info["status"] == 5
    bad = l2g.clone()
    bad[0] = -1
    with pytest.raises(spx.SpxError):
        spx.cg_solve(c.plan, 1.0, bad, ng, b)
    with pytest.raises(spx.SpxError):                      # workspace too small
        spx.cg_solve(c.plan, 1.0, l2g, ng, b, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))


def test_resume_from_saved_iterate():
    """Checkpoint / resume: a solve restarted from a saved iterate converges to the same solution."""
    dim, N, P = 3, 3, 3
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    b = torch.tensor(synth.uniform(synth.rng(34), ng), device="cuda")
    x_part, info = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f64", maxit=10,
                                raise_on_fail=False)
    assert info["status"] == 4
    x, info2 = spx.cg_solve(c.plan, 1.0, l2g, ng, b, x0=x_part, tol=1e-10, precision="f64")
    xr, _ = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f64")
    assert info2["status"] == 0
    assert rel_err(x, xr.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("inner_tol", [1e-1, 1e-3])
def test_reliable_updates_replace_the_residual(inner_tol):
    """precision 2: each FP32 stretch lowers the true FP64 residual by about inner_tol, the run is
    not restarted (fewer FP32 iterations than restarted refinement at the same inner_tol), and the
    iteration cap is a cap on all FP32 iterations."""
    dim, N, P = 3, 4, 4
    c = Case(dim, N, P=P, amp=0.05)
    l2g, ng = mesh.periodic_l2g(dim, N, P)
    b = torch.tensor(synth.uniform(synth.rng(35), ng), device="cuda")
    xr, ir = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f32_reliable", inner_tol=inner_tol)
    xf, if_ = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f32_refine", inner_tol=inner_tol)
    x64, _ = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-12, precision="f64")
    assert ir["status"] == 0 and ir["rel_residual"] <= 1e-10
    assert rel_err(xr, x64.cpu().numpy()) <= 1e-8
    # ten decades in steps of inner_tol (the last step may be shorter)
    steps = int(np.ceil(10 / -np.log10(inner_tol)))
    assert steps <= ir["outer_iters"] <= steps + 3
    assert ir["iters"] <= if_["iters"]
    x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, b, tol=1e-10, precision="f32_reliable", inner_tol=inner_tol,
                           maxit=7, raise_on_fail=False)
    assert info["status"] == 4 and info["iters"] == 7
