"""GPU parity of the elemental operators against the FP64 oracle.

Every comparison is element by element on seeded inputs.  Tolerances:
relative max error (max |y - y_ref| / max |y_ref|) <= 1e-12 for FP64 kernels
and <= 1e-5 for FP32 kernels.
"""
import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import operators
from paper_1906_03489_gb300 import synth

from _cases import Case, rel_err

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
DTYPES = [torch.float64, torch.float32]

# (dim, N, P, amp): several tiles with a ragged tail, both dimensions, the
# order range 1..8 and both Q = P+2 (default) and Q = P+1
SHAPES = [(3, 3, 4, 0.05), (3, 5, 2, 0.05), (3, 2, 8, 0.05), (3, 3, 1, 0.05), (3, 4, 6, 0.05),
          (2, 16, 4, 0.0), (2, 7, 3, 0.05), (2, 5, 8, 0.05), (2, 3, 1, 0.0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _case(dim, N, P, amp, q_offset=2):
    return Case(dim, N, P=P, amp=amp, q_offset=q_offset)


@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_geometry_factors(dim, N, P, amp):
    c = _case(dim, N, P, amp)
    geom, dxi, xq = c.om.factors_flat()
    assert rel_err(c.g["geom"], geom) <= 1e-12
    assert rel_err(c.g["dxi"], dxi) <= 1e-12
    assert rel_err(c.g["xq"], xq) <= 1e-12
    assert rel_err(c.g["geom32"], geom) <= 1e-6


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_bwd_trans(dim, N, P, amp, dtype):
    c = _case(dim, N, P, amp)
    u, ut = c.coef(1, dtype)
    ref = operators.bwd_trans(c.om, u)
    assert rel_err(spx.bwd_trans(c.plan, ut), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_iproduct(dim, N, P, amp, dtype):
    c = _case(dim, N, P, amp)
    f, ft = c.quad(2, dtype)
    ref = operators.iproduct(c.om, f)
    assert rel_err(spx.iproduct(c.plan, ft), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_phys_deriv(dim, N, P, amp, dtype):
    c = _case(dim, N, P, amp)
    f, ft = c.quad(3, dtype)
    refs = operators.phys_deriv(c.om, f)
    outs = spx.phys_deriv(c.plan, ft)
    scale = max(np.abs(r).max() for r in refs)
    for o, r in zip(outs, refs):
        assert np.abs(o.cpu().double().numpy() - r).max() / scale <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_helmholtz(dim, N, P, amp, dtype):
    c = _case(dim, N, P, amp)
    u, ut = c.coef(4, dtype)
    ref = operators.helmholtz(c.om, u, lam=1.0)
    assert rel_err(spx.helmholtz(c.plan, ut, lam=1.0), ref) <= TOL[dtype]
    ref2 = operators.helmholtz(c.om, u, lam=2.5)
    assert rel_err(spx.helmholtz(c.plan, ut, lam=2.5), ref2) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P", [(3, 3, 4), (2, 4, 5), (3, 2, 7)])
def test_helmholtz_with_fields(dim, N, P, dtype):
    c = _case(dim, N, P, 0.05)
    u, ut = c.coef(5, dtype)
    lam = 1.0 + 0.5 * synth.uniform(synth.rng(6), c.plan.n_quad)
    kap = 1.0 + 0.3 * synth.uniform(synth.rng(7), c.plan.n_quad)
    ref = operators.helmholtz(c.om, u, lam_field=lam, kappa_field=kap)
    lt = torch.tensor(lam, device="cuda", dtype=dtype)
    kt = torch.tensor(kap, device="cuda", dtype=dtype)
    assert rel_err(spx.helmholtz(c.plan, ut, lam_field=lt, kappa_field=kt), ref) <= TOL[dtype]
    refk = operators.helmholtz(c.om, u, lam=0.7, kappa_field=kap)
    assert rel_err(spx.helmholtz(c.plan, ut, lam=0.7, kappa_field=kt), refk) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_q_offset_one(dtype):
    c = _case(3, 3, 3, 0.05, q_offset=1)
    u, ut = c.coef(8, dtype)
    assert rel_err(spx.helmholtz(c.plan, ut), operators.helmholtz(c.om, u)) <= TOL[dtype]
    assert rel_err(spx.bwd_trans(c.plan, ut), operators.bwd_trans(c.om, u)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N", [(3, 5), (2, 9)])
def test_variable_order(dim, N, dtype):
    gen = synth.rng(3)
    orders = synth.orders(gen, N ** dim, 1, 8)
    c = Case(dim, N, orders=orders, amp=0.05)
    u, ut = c.coef(9, dtype)
    f, ft = c.quad(10, dtype)
    assert rel_err(spx.helmholtz(c.plan, ut), operators.helmholtz(c.om, u)) <= TOL[dtype]
    assert rel_err(spx.bwd_trans(c.plan, ut), operators.bwd_trans(c.om, u)) <= TOL[dtype]
    assert rel_err(spx.iproduct(c.plan, ft), operators.iproduct(c.om, f)) <= TOL[dtype]
    refs = operators.phys_deriv(c.om, f)
    outs = spx.phys_deriv(c.plan, ft)
    scale = max(np.abs(r).max() for r in refs)
    for o, r in zip(outs, refs):
        assert np.abs(o.cpu().double().numpy() - r).max() / scale <= TOL[dtype]


@pytest.mark.parametrize("nthreads", [512, 640, 768])
@pytest.mark.parametrize("eb,stages", [(1, 0), (2, 1), (3, 2)])
def test_variable_order_pair_classes(nthreads, eb, stages):
    """FP32 variable-order Helmholtz with element pairs up to P = 5, 6 and 8
    (the launch's threads class), several tile sizes and prefetch depths; each
    CTA keeps to one order's run of tiles (here runs of a few tiles, fewer
    than the CTAs an SM's share would give them)."""
    orders = synth.orders(synth.rng(27), 5 ** 3, 1, 8)
    c = Case(3, 5, orders=orders, amp=0.05)
    u, ut = c.coef(28, torch.float32)
    c.plan.set_tile("helmholtz", torch.float32, eb, nthreads, stages)
    assert rel_err(spx.helmholtz(c.plan, ut), operators.helmholtz(c.om, u)) <= 1e-5


def test_variable_order_equals_uniform_launches():
    """One variable-order launch gives, element by element, what uniform launches give."""
    dim, N = 3, 4
    orders = synth.orders(synth.rng(11), N ** dim, 2, 5)
    c = Case(dim, N, orders=orders, amp=0.05)
    u, ut = c.coef(12, torch.float64)
    y = spx.helmholtz(c.plan, ut).cpu().numpy()
    for P in np.unique(orders):
        cu = Case(dim, N, P=int(P), amp=0.05)
        # uniform-order input holding u_e on the elements of this order
        uu = np.zeros(cu.plan.n_coef)
        n = (int(P) + 1) ** dim
        for e in np.nonzero(orders == P)[0]:
            uu[e * n:(e + 1) * n] = u[c.plan.coef_off[e]:c.plan.coef_off[e + 1]]
        yu = spx.helmholtz(cu.plan, torch.tensor(uu, device="cuda")).cpu().numpy()
        scale = np.abs(yu).max()
        for e in np.nonzero(orders == P)[0]:
            np.testing.assert_allclose(y[c.plan.coef_off[e]:c.plan.coef_off[e + 1]], yu[e * n:(e + 1) * n],
                                       rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("dtype", DTYPES)
def test_bitwise_reproducible(dtype):
    c = _case(3, 4, 4, 0.05)
    _, ut = c.coef(13, dtype)
    a = spx.helmholtz(c.plan, ut)
    b = spx.helmholtz(c.plan, ut)
    assert torch.equal(a, b)


def test_empty_and_single_element():
    p = spx.Plan(3, 0, order=4)
    assert p.n_coef == 0 and p.n_quad == 0
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    spx.helmholtz(p, z, out=torch.zeros(0, dtype=torch.float64, device="cuda"))
    c = _case(3, 1, 4, 0.0)
    u, ut = c.coef(14)
    assert rel_err(spx.helmholtz(c.plan, ut), operators.helmholtz(c.om, u)) <= 1e-12


@pytest.mark.parametrize("eb,nthreads,stages", [(1, 64, 1), (3, 128, 2), (7, 192, 3), (16, 512, 2), (64, 512, 1)])
def test_tile_shapes_do_not_change_results(eb, nthreads, stages):
    c = _case(3, 5, 3, 0.05)
    u, ut = c.coef(15)
    ref = operators.helmholtz(c.om, u)
    for op in ("helmholtz", "bwd_trans"):
        try:
            c.plan.set_tile(op, torch.float64, eb, nthreads, stages)
        except spx.SpxError as e:
            assert e.status == 2   # tile does not fit: unsupported, reported
            continue
    assert rel_err(spx.helmholtz(c.plan, ut), ref) <= 1e-12
    assert rel_err(spx.bwd_trans(c.plan, ut), operators.bwd_trans(c.om, u)) <= 1e-12


@pytest.mark.parametrize("eb,budget,pf", [(1, 512, 1), (2, 640, 2), (3, 768, 3), (8, 512, 0), (13, 640, 2),
                                           (24, 768, 1), (20, 1024, 4)])
def test_pair_kernel_tiles_do_not_change_results(eb, budget, pf):
    """FP32 3D Helmholtz (two elements per thread): odd and even tile sizes, a
    ragged last tile (5^3 elements), every register budget and prefetch depth."""
    c = _case(3, 5, 4, 0.05)
    u, ut = c.coef(18, torch.float32)
    ref = operators.helmholtz(c.om, u)
    c.plan.set_tile("helmholtz", torch.float32, eb, budget, pf)
    assert c.plan.get_tile("helmholtz", torch.float32, 4) == (eb, budget, pf)
    assert rel_err(spx.helmholtz(c.plan, ut), ref) <= 1e-5


@pytest.mark.parametrize("P,q_offset", [(4, 2), (4, 1), (8, 2), (2, 1)])
@pytest.mark.parametrize("eb,budget,pf", [(1, 768, 0), (2, 1024, 1), (7, 1280, 2), (13, 1536, 3), (24, 1024, 4),
                                           (64, 1536, 1)])
def test_streaming_pair_tiles_do_not_change_results(P, q_offset, eb, budget, pf):
    """FP32 3D BwdTrans and IProductWRTBase in the element-pair layout: odd and
    even tile sizes, a ragged last tile (3^3 elements), every register class
    (the smallest spills at high orders), inputs carried in registers (0) or
    staged through a ring of 1..4 shared-memory slots, Q = P+1 and P+2.  A
    tile over 1024 threads or the shared memory is refused, not run."""
    c = _case(3, 3, P, 0.05, q_offset)
    u, ut = c.coef(22, torch.float32)
    f, ft = c.quad(23, torch.float32)
    for op in ("bwd_trans", "iproduct"):
        try:
            c.plan.set_tile(op, torch.float32, eb, budget, pf)
        except spx.SpxError as e:
            assert e.status == 2 and not (P <= 4 and eb <= 7)   # refused as too large; small tiles fit
            return
        assert c.plan.get_tile(op, torch.float32, P) == (eb, budget, pf)
    assert rel_err(spx.bwd_trans(c.plan, ut), operators.bwd_trans(c.om, u)) <= 1e-5
    assert rel_err(spx.iproduct(c.plan, ft), operators.iproduct(c.om, f)) <= 1e-5


@pytest.mark.parametrize("P,q_offset", [(2, 2), (4, 2), (4, 1), (8, 2)])
@pytest.mark.parametrize("nthreads,stages", [(896, 0), (1024, 1), (512, 0)])
def test_role_register_classes(P, q_offset, nthreads, stages):
    """FP64 3D Helmholtz with Q^2 threads per element: the 72-register class
    (nthreads > 512; it spills at the highest orders) and the 128-register
    class give the oracle's result, on the largest tile that fits (512
    threads, the shared memory) and on a ragged tile of at most 3 elements."""
    c = _case(3, 3, P, 0.05, q_offset)
    u, ut = c.coef(26)
    ref = operators.helmholtz(c.om, u)
    Q = P + q_offset
    for top in (max(1, 512 // Q ** 2), 3):
        for eb in range(top, 0, -1):
            try:
                c.plan.set_tile("helmholtz", torch.float64, eb, nthreads, stages)
                break
            except spx.SpxError as e:
                assert e.status == 2 and eb > 1   # too large for the shared memory; one element always fits
        assert rel_err(spx.helmholtz(c.plan, ut), ref) <= 1e-12


@pytest.mark.parametrize("stages", [0, 2])
def test_streaming_pair_unaligned_views(stages):
    """FP32 3D BwdTrans and IProductWRTBase on 4-byte-offset views: every
    staged range then has ragged head and tail words."""
    c = _case(3, 3, 4, 0.05)
    u, _ = c.coef(24)
    f, _ = c.quad(25)

    def view(x, off):
        big = torch.zeros(x.size + off + 1, dtype=torch.float32, device="cuda")
        big[off:off + x.size] = torch.tensor(x, device="cuda", dtype=torch.float32)
        return big[off:off + x.size]

    for op in ("bwd_trans", "iproduct"):
        c.plan.set_tile(op, torch.float32, 5, 1024, stages)
    y = spx.bwd_trans(c.plan, view(u, 1), out=view(np.zeros(c.plan.n_quad), 3))
    assert rel_err(y, operators.bwd_trans(c.om, u)) <= 1e-5
    z = spx.iproduct(c.plan, view(f, 2), out=view(np.zeros(c.plan.n_coef), 1))
    assert rel_err(z, operators.iproduct(c.om, f)) <= 1e-5


def test_pair_kernel_tile_too_large_is_refused():
    c = _case(3, 2, 4, 0.05)
    with pytest.raises(spx.SpxError) as e:
        c.plan.set_tile("helmholtz", torch.float32, 28, 512, 0)   # 28 staged geometry blocks: > 227 KB
    assert e.value.status == 2


def test_pair_kernel_unaligned_and_fields():
    """FP32 3D Helmholtz on 4-byte-offset views, with lambda and kappa fields."""
    c = _case(3, 3, 5, 0.05)
    u, _ = c.coef(19)
    lam, _ = c.quad(20)
    kap, _ = c.quad(21)
    lam, kap = 1.5 + 0.5 * lam, 1.0 + 0.25 * kap
    ref = operators.helmholtz(c.om, u, lam_field=lam, kappa_field=kap)

    def view(x, off):
        big = torch.zeros(x.size + off + 1, dtype=torch.float32, device="cuda")
        big[off:off + x.size] = torch.tensor(x, device="cuda", dtype=torch.float32)
        return big[off:off + x.size]

    out = view(np.zeros(c.plan.n_coef), 3)
    y = spx.helmholtz(c.plan, view(u, 1), lam_field=view(lam, 2), kappa_field=view(kap, 3), out=out)
    assert rel_err(y, ref) <= 1e-5


def test_autotune_keeps_results():
    c = _case(3, 6, 4, 0.05)
    u, ut = c.coef(16, torch.float32)
    out = torch.empty(c.plan.n_coef, dtype=torch.float32, device="cuda")
    c.plan.autotune("helmholtz", torch.float32, ut, out, reps=2)
    eb, nt, st = c.plan.get_tile("helmholtz", torch.float32, 4)
    assert 1 <= eb <= 64 and nt % 32 == 0 and 0 <= st <= 4   # stages 0: no L2 prefetch (pair kernel)
    assert rel_err(spx.helmholtz(c.plan, ut), operators.helmholtz(c.om, u)) <= 1e-5


def test_autotune_streaming_ops_keeps_results():
    """The autotuner's search over the FP32 BwdTrans / IProductWRTBase pair
    kernels (tile, register class, input ring depth; timed after an L2
    eviction) leaves results at the FP32 bar, and its choice is a valid tile."""
    c = _case(3, 4, 4, 0.05)
    u, ut = c.coef(29, torch.float32)
    f, ft = c.quad(30, torch.float32)
    q = torch.empty(c.plan.n_quad, dtype=torch.float32, device="cuda")
    m = torch.empty(c.plan.n_coef, dtype=torch.float32, device="cuda")
    c.plan.autotune("bwd_trans", torch.float32, ut, q, reps=2)
    c.plan.autotune("iproduct", torch.float32, ft, m, reps=2)
    for op in ("bwd_trans", "iproduct"):
        eb, nt, st = c.plan.get_tile(op, torch.float32, 4)
        assert 1 <= eb <= 64 and 32 <= nt <= 2048 and 0 <= st <= 4
    assert rel_err(spx.bwd_trans(c.plan, ut), operators.bwd_trans(c.om, u)) <= 1e-5
    assert rel_err(spx.iproduct(c.plan, ft), operators.iproduct(c.om, f)) <= 1e-5


def test_unaligned_buffers():
    """Element blocks at arbitrary 8-byte offsets (views into larger buffers)."""
    c = _case(3, 3, 3, 0.05)
    u, _ = c.coef(17)
    big = torch.zeros(c.plan.n_coef + 3, dtype=torch.float64, device="cuda")
    big[1:1 + c.plan.n_coef] = torch.tensor(u, device="cuda")
    out = torch.zeros(c.plan.n_coef + 3, dtype=torch.float64, device="cuda")
    spx.helmholtz(c.plan, big[1:1 + c.plan.n_coef], out=out[3:3 + c.plan.n_coef])
    assert rel_err(out[3:3 + c.plan.n_coef], operators.helmholtz(c.om, u)) <= 1e-12


def test_invalid_arguments_are_reported():
    c = _case(3, 2, 3, 0.05)
    _, ut = c.coef(18)
    with pytest.raises(spx.SpxError):
        spx.helmholtz(c.plan, ut, out=ut)            # aliasing
    p2 = spx.Plan(3, 8, order=3)
    with pytest.raises(spx.SpxError):
        spx.helmholtz(p2, ut)                          # geometry not registered
    with pytest.raises(spx.SpxError):
        spx.Plan(3, 8, order=9)                        # order out of range
    with pytest.raises(spx.SpxError):
        spx.Plan(4, 8, order=3)                        # bad dimension
    assert c.plan.device_status() == 0
