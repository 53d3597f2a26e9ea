"""CPU checks of caller-supplied basis tables (spx_basis_desc): the nodal
tables the library offers match the oracle's Lagrange polynomials, and plan
creation refuses inconsistent descriptions before any device call."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1906_03489_gb300 import build
    build.build()
    from paper_1906_03489_gb300 import _lib
    return _lib.lib()


@pytest.mark.parametrize("P,Q", [(1, 2), (2, 3), (4, 5), (4, 6), (6, 8), (8, 9), (8, 10)])
def test_nodal_basis_tables_match_oracle(lib, P, Q):
    from oracle import basis
    from paper_1906_03489_gb300 import nodal_basis_tables
    t = nodal_basis_tables(P, Q)
    z, _ = basis.gll(P + 1)
    xi, _ = basis.gll(Q)
    L, dL = basis.lagrange(z, xi)
    np.testing.assert_allclose(t["B"], L, atol=1e-13)
    np.testing.assert_allclose(t["dB"], dL, atol=1e-11 * np.abs(dL).max())
    if Q == P + 1:
        np.testing.assert_allclose(t["B"], np.eye(Q), atol=1e-14)


def _plan(basis, order=3, q_offset=2, orders=None):
    from paper_1906_03489_gb300 import Plan
    return Plan(3, 8 if orders is None else len(orders), order=None if orders is not None else order,
                orders=orders, q_offset=q_offset, basis=basis)


def _modified(P, Q):
    from paper_1906_03489_gb300 import basis_tables
    return basis_tables(P, Q)


@pytest.mark.parametrize("case", ["wrong_q", "bad_d", "bad_w", "bad_db", "missing_order", "nan"])
def test_plan_refuses_inconsistent_basis(lib, case):
    from paper_1906_03489_gb300 import SpxError
    P = 3
    t = _modified(P, P + 2)
    d = {"B": t["B"], "dB": t["dB"], "D": t["D"], "w": t["w"]}
    basis = {P: d}
    kw = {}
    if case == "wrong_q":   # a desc whose Q is not P + q_offset, built without the binding
        import ctypes as C
        from paper_1906_03489_gb300 import _lib
        arr = (_lib.BasisDesc * 1)()
        B = np.ascontiguousarray(t["B"])
        arr[0].P, arr[0].Q, arr[0].B = P, P + 1, B.ctypes.data
        desc = _lib.PlanDesc()
        desc.dim, desc.n_elem, desc.uniform_order, desc.q_offset = 3, 8, P, 2
        desc.n_basis, desc.basis, desc.basis_memory = 1, arr, _lib.SPX_MEM_HOST
        h = C.c_void_p()
        st = lib.spx_plan_create(C.byref(h), C.byref(desc))
        assert st == 1 and b"P + q_offset" in lib.spx_last_error()
        return
    if case == "bad_d":
        d["D"] = t["D"] * 1.001
    elif case == "bad_w":
        d["w"] = t["w"] * 1.001
    elif case == "bad_db":
        d["dB"] = t["dB"] + 1e-3
    elif case == "missing_order":
        kw["orders"] = np.array([3, 4, 3, 4], np.int32)
    elif case == "nan":
        B = t["B"].copy()
        B[1, 1] = np.nan
        d["B"] = B
    with pytest.raises(SpxError) as ei:
        _plan(basis, order=P, **kw)
    expect = {"wrong_q": "P + q_offset", "bad_d": "collocation derivative", "bad_w": "GLL weights",
              "bad_db": "derivative of B", "missing_order": "no basis description", "nan": "not finite"}[case]
    assert expect in str(ei.value)


@pytest.mark.parametrize("Q", [2, 3, 6, 9, 10])
def test_gauss_radau_matches_oracle(lib, Q):
    from oracle import collapsed
    from paper_1906_03489_gb300 import gauss_radau
    x, w = gauss_radau(Q)
    xo, wo = collapsed.gauss_radau(Q)
    np.testing.assert_allclose(x, xo, atol=1e-14)
    np.testing.assert_allclose(w, wo, rtol=1e-12)


def test_collapsed_plans_refuse_what_they_do_not_support(lib):
    from paper_1906_03489_gb300 import Plan, SpxError
    with pytest.raises(SpxError, match="triangles are 2D"):
        Plan(3, 4, order=2, shape="tri")
    with pytest.raises(SpxError, match="uniform order"):
        Plan(2, 4, orders=np.array([2, 3, 2, 3], np.int32), shape="tri")
    with pytest.raises(SpxError, match="uniform order"):
        Plan(3, 4, order=2, q_offset=1, shape="prism")
