"""CPU checks of the C ABI: the library loads, exports every function that
include/spx.h declares, and its host-side tables agree with the oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "spx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_03489_gb300 import build
    build.build()
    from paper_1906_03489_gb300 import _lib
    return _lib.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["spx_bwd_trans", "spx_iproduct", "spx_phys_deriv", "spx_helmholtz", "spx_cg_solve",
                     "spx_helmholtz_adjoint", "spx_geom_factors", "spx_plan_create", "spx_autotune"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1906_03489_gb300 import _lib
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert sorted(_lib.SIGNATURES) == names


@pytest.mark.parametrize("P,Q", [(1, 2), (1, 3), (2, 4), (4, 6), (6, 8), (8, 10), (8, 9), (3, 4)])
def test_host_basis_tables_match_oracle(lib, P, Q):
    from oracle import basis
    from paper_1906_03489_gb300 import basis_tables
    t = basis_tables(P, Q)
    x, w = basis.gll(Q)
    np.testing.assert_allclose(t["xi"], x, atol=1e-15)
    np.testing.assert_allclose(t["w"], w, rtol=1e-14)
    np.testing.assert_allclose(t["B"], basis.modified_basis(P, x), atol=1e-14)
    np.testing.assert_allclose(t["dB"], basis.modified_basis_deriv(P, x), atol=1e-13)
    np.testing.assert_allclose(t["D"], basis.collocation_derivative(Q), atol=1e-12)


def test_basis_tables_reject_bad_sizes(lib):
    from paper_1906_03489_gb300 import SpxError, basis_tables
    with pytest.raises(SpxError):
        basis_tables(0, 4)
    with pytest.raises(SpxError):
        basis_tables(4, 17)


@pytest.mark.parametrize("dim,N,P", [(2, 3, 2), (3, 2, 3), (3, 3, 4)])
def test_periodic_map_matches_oracle(dim, N, P):
    from oracle import geometry, solve
    from paper_1906_03489_gb300 import mesh
    l2g, ng = mesh.periodic_l2g(dim, N, P, device="cpu")
    om = geometry.StructuredMesh(dim, N, P)
    np.testing.assert_array_equal(l2g.numpy(), solve.local_to_global(om))
    assert ng == solve.n_global(om)


def test_adapt_orders_host_entry_point_matches_oracle(lib):
    """spx_adapt_orders is host code: the §4.2 order update, checked on the CPU."""
    from oracle import adapt
    import paper_1906_03489_gb300 as spx
    rng = np.random.default_rng(9)
    S = 10.0 ** rng.uniform(-12, 0, 200)
    P = rng.integers(2, 9, 200).astype(np.int32)
    for lo, hi, pmin, pmax in ((1e-8, 1e-3, 2, 8), (1e-6, 1e-6, 3, 6), (0.0, 1.0, 2, 2)):
        np.testing.assert_array_equal(spx.adapt_orders(S, P, lo, hi, pmin, pmax),
                                      adapt.adapt_orders(S, P, lo, hi, pmin, pmax))
    with pytest.raises(spx.SpxError):
        spx.adapt_orders(S, P, 1e-3, 1e-8, 2, 8)        # lower > upper
    with pytest.raises(spx.SpxError):
        spx.adapt_orders(S, P, 1e-8, 1e-3, 1, 8)        # P_min < 2


@pytest.mark.parametrize("dim,n_elem,order,orders,qoff,status", [
    (4, 8, 3, None, 2, 1),              # dimension outside {2, 3}
    (3, -1, 3, None, 2, 1),             # negative element count
    (3, 8, 9, None, 2, 1),              # uniform order above 8
    (3, 8, 0, None, 2, 1),              # uniform order below 1
    (3, 3, 0, [2, 9, 4], 2, 1),         # a per-element order above 8
    (3, 8, 3, None, 3, 2),              # q_offset outside {1, 2}
])
def test_plan_create_validates_before_touching_the_device(lib, dim, n_elem, order, orders, qoff, status):
    """Invalid plan descriptions are refused with a status and a message, before any CUDA call."""
    import ctypes as C
    from paper_1906_03489_gb300 import _lib
    d = _lib.PlanDesc()
    d.dim, d.n_elem, d.uniform_order, d.q_offset = dim, n_elem, order, qoff
    keep = None
    if orders is not None:
        keep = np.asarray(orders, dtype=np.int32)
        d.elem_order = keep.ctypes.data_as(C.POINTER(C.c_int32))
    h = C.c_void_p()
    assert lib.spx_plan_create(C.byref(h), C.byref(d)) == status
    assert not h.value
    assert lib.spx_last_error().decode().startswith("plan_create")
