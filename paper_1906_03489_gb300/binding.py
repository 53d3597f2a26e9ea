"""Thin torch-facing binding of the spx C ABI.

Argument marshalling only: every operator runs in the CUDA library; tensors
supply device memory, ``torch.cuda.current_stream()`` supplies the stream.
Outputs are allocated with torch when the caller does not pass them.
"""
import ctypes as C

import numpy as np
import torch

from ._lib import (SPX_F32, SPX_F64, SPX_MEM_DEVICE, SPX_MEM_HOST, SPX_SHAPE_PRISM, SPX_SHAPE_TENSOR, SPX_SHAPE_TET,
                   SPX_SHAPE_TRI,
                   OPS, BasisDesc, CgOpts, CgResult, PlanDesc, SpxError, check, lib)

__all__ = ["Plan", "basis_tables", "nodal_basis_tables", "gauss_radau", "geom_factors", "bwd_trans", "iproduct", "phys_deriv", "helmholtz", "fwd_trans",
           "integral", "sensor", "adapt_orders",
           "helmholtz_adjoint", "helmholtz_diag", "gather", "assemble", "dot", "cg_workspace_bytes", "cg_solve",
           "SpxError"]


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _code(dtype):
    if dtype == torch.float64:
        return SPX_F64
    if dtype == torch.float32:
        return SPX_F32
    raise TypeError(f"unsupported dtype {dtype}")


def _dev(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    return t


def basis_tables(P, Q):
    """Host FP64 tables of order P on Q GLL points: dict xi, w, B, dB, D (numpy)."""
    xi, w = np.zeros(Q), np.zeros(Q)
    B, dB, D = np.zeros((Q, P + 1)), np.zeros((Q, P + 1)), np.zeros((Q, Q))
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    check(lib().spx_basis_tables(P, Q, ptr(xi), ptr(w), ptr(B), ptr(dB), ptr(D)))
    return dict(xi=xi, w=w, B=B, dB=dB, D=D)


def nodal_basis_tables(P, Q):
    """Host FP64 tables of the GLL nodal (Lagrange) basis of order P at Q GLL points: dict B, dB (numpy)."""
    B, dB = np.zeros((Q, P + 1)), np.zeros((Q, P + 1))
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    check(lib().spx_nodal_basis_tables(P, Q, ptr(B), ptr(dB)))
    return dict(B=B, dB=dB)


def _basis_descs(basis, q_offset):
    """spx_basis_desc array from {P: {"B": ..., "dB": ..., "D": ..., "w": ...}}: numpy arrays
    (host) or CUDA tensors (device), all of one kind.  Returns (array, memory kind, keep-alive list)."""
    items = sorted(basis.items())
    arr = (BasisDesc * len(items))()
    keep, kinds = [], set()
    for t, (P, tabs) in enumerate(items):
        arr[t].P, arr[t].Q = int(P), int(P) + q_offset
        for name in ("B", "dB", "D", "w"):
            v = tabs.get(name)
            if v is None:
                setattr(arr[t], name, None)
                continue
            if isinstance(v, torch.Tensor) and v.is_cuda:
                v = v.to(torch.float64).contiguous()
                kinds.add(SPX_MEM_DEVICE)
                setattr(arr[t], name, v.data_ptr())
            else:
                v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
                kinds.add(SPX_MEM_HOST)
                setattr(arr[t], name, v.ctypes.data)
            keep.append(v)
    if len(kinds) > 1:
        raise TypeError("basis tables must be all host arrays or all CUDA tensors")
    return arr, (kinds.pop() if kinds else SPX_MEM_HOST), keep


class Plan:
    """A mesh of E elements of dimension 2 or 3 with per-element orders.

    basis: optional caller-supplied basis tables per order,
    {P: {"B": [Q][P+1], "dB": [Q][P+1] or None, "D": None, "w": None}}, as
    numpy arrays or CUDA tensors (spx_basis_desc); default the modified basis.
    """

    def __init__(self, dim, n_elem, order=None, orders=None, q_offset=2, basis=None, shape="tensor"):
        self.dim, self.E, self.q_offset = int(dim), int(n_elem), int(q_offset)
        self.shape = shape
        desc = PlanDesc()
        desc.dim, desc.n_elem, desc.q_offset = self.dim, self.E, self.q_offset
        desc.shape = {"tensor": SPX_SHAPE_TENSOR, "tri": SPX_SHAPE_TRI, "prism": SPX_SHAPE_PRISM,
                      "tet": SPX_SHAPE_TET}[shape]
        keep = None
        if basis:
            arr, mem, keep = _basis_descs(basis, self.q_offset)
            desc.n_basis, desc.basis, desc.basis_memory = len(arr), arr, mem
        self._orders = None
        if orders is not None:
            self._orders = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
            if self._orders.size != self.E:
                raise ValueError("orders must have n_elem entries")
            desc.elem_order = self._orders.ctypes.data_as(C.POINTER(C.c_int32))
            desc.uniform_order = 0
        else:
            desc.elem_order = None
            desc.uniform_order = int(order)
        h = C.c_void_p()
        check(lib().spx_plan_create(C.byref(h), C.byref(desc)))
        del keep   # the plan copied the tables
        self.handle = h
        nc, nq = C.c_int64(), C.c_int64()
        check(lib().spx_plan_sizes(h, C.byref(nc), C.byref(nq)))
        self.n_coef, self.n_quad = nc.value, nq.value
        co = np.zeros(self.E + 1, dtype=np.int64)
        qo = np.zeros(self.E + 1, dtype=np.int64)
        check(lib().spx_plan_offsets(h, co.ctypes.data_as(C.POINTER(C.c_int64)),
                                     qo.ctypes.data_as(C.POINTER(C.c_int64))))
        self.coef_off, self.quad_off = co, qo
        self.orders = self._orders if self._orders is not None else np.full(self.E, int(order), np.int32)
        self._keep = {}

    def close(self):
        if getattr(self, "handle", None):
            lib().spx_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, dtype, geom, dxi=None):
        """Registers geometry tensors of one precision (kept alive by the plan)."""
        code = _code(dtype)
        if geom is not None:
            _dev(geom, "geom")
        if dxi is not None:
            _dev(dxi, "dxi_dx")
        check(lib().spx_plan_set_geometry(self.handle, code, _p(geom), _p(dxi)))
        self._keep[code] = (geom, dxi)

    def set_tile(self, op, dtype, eb, nthreads=256, stages=2, order=-1):
        check(lib().spx_plan_set_tile(self.handle, OPS[op], _code(dtype), order, eb, nthreads, stages))

    def get_tile(self, op, dtype, order):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(lib().spx_plan_get_tile(self.handle, OPS[op], _code(dtype), order, C.byref(a), C.byref(b),
                                      C.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, op, dtype, inp, out, reps=5):
        check(lib().spx_autotune(self.handle, OPS[op], _code(dtype), _p(inp), _p(out), reps, _stream()))

    def device_status(self, reset=True):
        s = C.c_int()
        check(lib().spx_plan_device_status(self.handle, C.byref(s), 1 if reset else 0))
        return s.value


def gauss_radau(Q):
    """Host FP64 Gauss-Radau-Legendre points (with -1) and weights: (x, w) numpy arrays."""
    x, w = np.zeros(Q), np.zeros(Q)
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    check(lib().spx_gauss_radau(Q, ptr(x), ptr(w)))
    return x, w


def geom_factors(plan, nodes, want_f32=True, want_xq=True):
    """FP64 geometric factors from nodal coordinates (device FP64 tensor; for
    triangle / prism plans the (E, d+1, d) affine vertices)."""
    _dev(nodes, "nodes")
    d = plan.dim
    nf = 7 if d == 3 else 4
    kw = dict(device=nodes.device)
    geom = torch.empty(nf * plan.n_quad, dtype=torch.float64, **kw)
    dxi = torch.empty(d * d * plan.n_quad, dtype=torch.float64, **kw)
    xq = torch.empty(d * plan.n_quad, dtype=torch.float64, **kw) if want_xq else None
    g32 = torch.empty(nf * plan.n_quad, dtype=torch.float32, **kw) if want_f32 else None
    d32 = torch.empty(d * d * plan.n_quad, dtype=torch.float32, **kw) if want_f32 else None
    check(lib().spx_geom_factors(plan.handle, _p(nodes), _p(geom), _p(dxi), _p(xq), _p(g32), _p(d32), _stream()))
    return dict(geom=geom, dxi=dxi, xq=xq, geom32=g32, dxi32=d32)


def bwd_trans(plan, coef, out=None):
    _dev(coef, "coef")
    out = torch.empty(plan.n_quad, dtype=coef.dtype, device=coef.device) if out is None else out
    check(lib().spx_bwd_trans(plan.handle, _code(coef.dtype), _p(coef), _p(out), _stream()))
    return out


def iproduct(plan, f, out=None):
    _dev(f, "f")
    out = torch.empty(plan.n_coef, dtype=f.dtype, device=f.device) if out is None else out
    check(lib().spx_iproduct(plan.handle, _code(f.dtype), _p(f), _p(out), _stream()))
    return out


def fwd_trans(plan, f, out=None):
    """Galerkin projection of quadrature-point values onto the expansion (per element)."""
    _dev(f, "f")
    out = torch.empty(plan.n_coef, dtype=f.dtype, device=f.device) if out is None else out
    check(lib().spx_fwd_trans(plan.handle, _code(f.dtype), _p(f), _p(out), _stream()))
    return out


def integral(plan, f, out=None):
    """Sum of JW f over the mesh as a device FP64 scalar tensor (``float(...)`` synchronises)."""
    _dev(f, "f")
    out = torch.empty((), dtype=torch.float64, device=f.device) if out is None else out
    check(lib().spx_integral(plan.handle, _code(f.dtype), _p(f), _p(out), _stream()))
    return out


def sensor(plan, coef, out=None):
    """Adaptive-order error sensor S_e per element (FP64 device tensor [n_elem])."""
    _dev(coef, "coef")
    if coef.dtype != torch.float64:
        raise TypeError("the sensor is FP64 only")
    out = torch.empty(plan.E, dtype=torch.float64, device=coef.device) if out is None else out
    check(lib().spx_sensor(plan.handle, _p(coef), _p(out), _stream()))
    return out


def adapt_orders(S, orders, lower, upper, p_min=2, p_max=8):
    """New per-element orders from the sensor values (host int32 numpy array)."""
    S = np.ascontiguousarray(S.detach().cpu().numpy() if isinstance(S, torch.Tensor) else S, dtype=np.float64)
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    new = np.empty_like(orders)
    check(lib().spx_adapt_orders(S.size, S.ctypes.data_as(C.c_void_p), orders.ctypes.data_as(C.c_void_p),
                                 float(lower), float(upper), int(p_min), int(p_max), new.ctypes.data_as(C.c_void_p)))
    return new


def phys_deriv(plan, f, outs=None):
    _dev(f, "f")
    if outs is None:
        outs = [torch.empty(plan.n_quad, dtype=f.dtype, device=f.device) for _ in range(plan.dim)]
    d2 = outs[2] if plan.dim == 3 else None
    check(lib().spx_phys_deriv(plan.handle, _code(f.dtype), _p(f), _p(outs[0]), _p(outs[1]), _p(d2), _stream()))
    return outs


def helmholtz(plan, u, lam=1.0, lam_field=None, kappa_field=None, out=None):
    _dev(u, "u")
    out = torch.empty(plan.n_coef, dtype=u.dtype, device=u.device) if out is None else out
    check(lib().spx_helmholtz(plan.handle, _code(u.dtype), float(lam), _p(lam_field), _p(kappa_field), _p(u),
                              _p(out), _stream()))
    return out


def helmholtz_adjoint(plan, u, g, want_lambda=True, want_kappa=True):
    _dev(u, "u")
    _dev(g, "g")
    gl = torch.empty(plan.n_quad, dtype=torch.float64, device=u.device) if want_lambda else None
    gk = torch.empty(plan.n_quad, dtype=torch.float64, device=u.device) if want_kappa else None
    check(lib().spx_helmholtz_adjoint(plan.handle, _p(u), _p(g), _p(gl), _p(gk), _stream()))
    return gl, gk


def helmholtz_diag(plan, dtype=torch.float64, lam=1.0, device="cuda"):
    out = torch.empty(plan.n_coef, dtype=dtype, device=device)
    check(lib().spx_helmholtz_diag(plan.handle, _code(dtype), float(lam), _p(out), _stream()))
    return out


def gather(plan, l2g, xg, out=None):
    _dev(l2g, "l2g")
    _dev(xg, "global")
    out = torch.empty(plan.n_coef, dtype=xg.dtype, device=xg.device) if out is None else out
    check(lib().spx_gather(plan.handle, _code(xg.dtype), _p(l2g), xg.numel(), _p(xg), _p(out), _stream()))
    return out


def assemble(plan, l2g, local, n_global, out=None):
    """global[g] = sum over local entries mapped to g (FP atomics)."""
    _dev(l2g, "l2g")
    _dev(local, "local")
    out = torch.empty(int(n_global), dtype=local.dtype, device=local.device) if out is None else out
    check(lib().spx_assemble(plan.handle, _code(local.dtype), _p(l2g), int(n_global), _p(local), _p(out),
                             _stream()))
    return out


def dot(plan, a, b, out=None):
    """<a, b> at FP64 accuracy as a device FP64 scalar tensor (the solver's reduction)."""
    _dev(a, "a")
    _dev(b, "b")
    if a.dtype != b.dtype or a.numel() != b.numel():
        raise TypeError("a and b must have the same dtype and length")
    out = torch.empty((), dtype=torch.float64, device=a.device) if out is None else out
    check(lib().spx_dot(plan.handle, _code(a.dtype), a.numel(), _p(a), _p(b), _p(out), _stream()))
    return out


def _cg_opts(tol, maxit, precision, inner_tol, max_outer, use_graph, check_every):
    o = CgOpts()
    o.tol, o.maxit = float(tol), int(maxit)
    o.precision = {"f64": 0, "f32_refine": 1, "f32_reliable": 2}[precision]
    o.inner_tol, o.max_outer = float(inner_tol), int(max_outer)
    o.use_graph, o.check_every = int(bool(use_graph)), int(check_every)
    return o


def cg_workspace_bytes(plan, n_global, precision="f32_refine", **kw):
    o = _cg_opts(kw.get("tol", 1e-10), kw.get("maxit", 10000), precision, kw.get("inner_tol", 1e-5),
                 kw.get("max_outer", 20), kw.get("use_graph", True), kw.get("check_every", 25))
    n = C.c_size_t()
    check(lib().spx_cg_workspace_bytes(plan.handle, int(n_global), C.byref(o), C.byref(n)))
    return n.value


def cg_solve(plan, lam, l2g, n_global, f, x0=None, tol=1e-10, maxit=10000, precision="f32_refine",
             inner_tol=1e-5, max_outer=20, use_graph=True, check_every=25, workspace=None, raise_on_fail=True):
    """Jacobi-PCG on the assembled operator; returns (x, result dict).

    precision: "f64" (all-FP64 PCG), "f32_refine" (FP32 PCG restarted inside
    FP64 iterative refinement) or "f32_reliable" (one FP32 PCG run whose
    residual is replaced by the FP64 one each time it fell by inner_tol).
    """
    _dev(l2g, "l2g")
    _dev(f, "f")
    o = _cg_opts(tol, maxit, precision, inner_tol, max_outer, use_graph, check_every)
    nb = C.c_size_t()
    check(lib().spx_cg_workspace_bytes(plan.handle, int(n_global), C.byref(o), C.byref(nb)))
    if workspace is None:
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=f.device)
    x = torch.zeros_like(f) if x0 is None else x0.clone()
    res = CgResult()
    st = lib().spx_cg_solve(plan.handle, float(lam), _p(l2g), int(n_global), _p(f), _p(x), _p(workspace),
                            workspace.numel(), C.byref(o), C.byref(res), _stream())
    info = dict(status=st, iters=res.iters, outer_iters=res.outer_iters, rel_residual=res.rel_residual)
    if st != 0 and raise_on_fail:
        check(st)
    return x, info
