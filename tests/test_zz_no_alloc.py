"""The allocation-free solve, called through the C ABI.

spx_cg_solve_noalloc serves callers that must not allocate device memory
while solving (their device memory belongs to another allocator, or a
cudaMalloc's implicit synchronisation is not acceptable where they call from):
its scratch is a fixed array inside the library.  This test checks that it
returns what spx_cg_solve returns with a caller workspace, on two calls in a
row (the array keeps the previous call's contents) with the device's free
memory unchanged across the second call, that a plan whose launch tiles are
not built yet (building them would allocate) is refused with x untouched,
and that problems larger than the array are refused before any work.  It is collected last so that a
run stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from paper_1906_03489_gb300 import _lib, mesh, synth
from paper_1906_03489_gb300.binding import _cg_opts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _plan(N, P):
    plan = spx.Plan(3, N ** 3, order=P)
    g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, 0.05))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    return plan, g


def _noalloc(plan, l2g, ng, f, x, precision):
    opts = _cg_opts(1e-11, 10000, precision, 1e-5, 20, True, 10)
    res = _lib.CgResult()
    st = _lib.lib().spx_cg_solve_noalloc(plan.handle, 1.0, C.c_void_p(l2g.data_ptr()), ng,
                                         C.c_void_p(f.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(opts),
                                         C.byref(res), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, res


@pytest.mark.parametrize("precision", ["f64", "f32_refine", "f32_reliable"])
def test_noalloc_solve_matches_workspace_solve_twice(precision):
    N, P = 4, 3
    plan, _ = _plan(N, P)
    l2g, ng = mesh.periodic_l2g(3, N, P)
    f = torch.tensor(synth.uniform(synth.rng(51), ng), device="cuda")
    x_ref, info = spx.cg_solve(plan, 1.0, l2g, ng, f, tol=1e-11, precision=precision, check_every=10)
    assert info["status"] == 0
    ref = x_ref.cpu().numpy()
    xs = [torch.full_like(f, 0.0) for _ in range(2)]
    for call in range(2):
        x = xs[call]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, res = _noalloc(plan, l2g, ng, f, x, precision)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0, _lib.lib().spx_last_error().decode()
        if call == 1:
            # everything the path touches has run once: the call allocates no device memory
            assert free1 == free0, (free0, free1)
        assert res.rel_residual <= 1e-11
        err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (call, err)


def test_noalloc_refuses_a_plan_whose_tiles_are_not_built():
    # geometry registered, no operator run yet: the solve would have to build
    # (allocate) its launch tiles, so it refuses and leaves x untouched
    N, P = 3, 2
    plan, _ = _plan(N, P)
    l2g, ng = mesh.periodic_l2g(3, N, P)
    f = torch.tensor(synth.uniform(synth.rng(52), ng), device="cuda")
    x = torch.full_like(f, 7.0)
    st, _ = _noalloc(plan, l2g, ng, f, x, "f64")
    assert st == 1     # SPX_ERR_INVALID_ARG
    assert b"not built yet" in _lib.lib().spx_last_error()
    assert bool((x == 7.0).all())
    # FP64 tiles only: an FP32-inner solve still needs the FP32 Helmholtz tiles
    u = torch.zeros(plan.n_coef, dtype=torch.float64, device="cuda")
    spx.helmholtz(plan, u)
    spx.helmholtz_diag(plan, torch.float64)
    st, _ = _noalloc(plan, l2g, ng, f, x, "f32_refine")
    assert st == 1
    assert b"not built yet" in _lib.lib().spx_last_error()
    assert bool((x == 7.0).all())
    # the FP64 solve has what it needs now
    x.zero_()
    st, res = _noalloc(plan, l2g, ng, f, x, "f64")
    assert st == 0, _lib.lib().spx_last_error().decode()
    assert res.rel_residual <= 1e-11


def test_noalloc_rejects_problems_beyond_its_array():
    N, P = 20, 4           # 8000 elements, 512000 global DOFs: workspace > 32 MiB
    plan = spx.Plan(3, N ** 3, order=P)
    l2g, ng = mesh.periodic_l2g(3, N, P)
    need = spx.cg_workspace_bytes(plan, ng, "f64")
    assert need > 32 * 1024 * 1024
    f = torch.zeros(ng, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(f)
    st, _ = _noalloc(plan, l2g, ng, f, x, "f64")
    assert st == 6     # SPX_ERR_NO_MEMORY
    assert b"built-in workspace" in _lib.lib().spx_last_error()
