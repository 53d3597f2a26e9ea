"""ctypes loader of the spx C ABI (include/spx.h).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation of any operator.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libspx.so")

SPX_F64, SPX_F32 = 0, 1
OPS = {"bwd_trans": 0, "iproduct": 1, "phys_deriv": 2, "helmholtz": 3, "helmholtz_adjoint": 4,
       "helmholtz_diag": 5, "fwd_trans": 6, "sensor": 7}

STATUS = {
    0: "SPX_OK", 1: "SPX_ERR_INVALID_ARG", 2: "SPX_ERR_UNSUPPORTED", 3: "SPX_ERR_CUDA",
    4: "SPX_ERR_NOT_CONVERGED", 5: "SPX_ERR_NONFINITE", 6: "SPX_ERR_NO_MEMORY", 7: "SPX_ERR_TIMEOUT",
}


class SpxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class BasisDesc(C.Structure):
    _fields_ = [("P", C.c_int), ("Q", C.c_int), ("B", C.c_void_p), ("dB", C.c_void_p), ("D", C.c_void_p),
                ("w", C.c_void_p)]


SPX_MEM_HOST, SPX_MEM_DEVICE = 0, 1


class PlanDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_elem", C.c_int64), ("elem_order", C.POINTER(C.c_int32)),
                ("uniform_order", C.c_int), ("q_offset", C.c_int), ("n_basis", C.c_int),
                ("basis", C.POINTER(BasisDesc)), ("basis_memory", C.c_int), ("shape", C.c_int)]


SPX_SHAPE_TENSOR, SPX_SHAPE_TRI, SPX_SHAPE_PRISM, SPX_SHAPE_TET = 0, 1, 2, 3


class CgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double),
                ("max_outer", C.c_int), ("use_graph", C.c_int), ("check_every", C.c_int)]


class CgResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("rel_residual", C.c_double)]


P = C.c_void_p
I32, I64, D = C.c_int, C.c_int64, C.c_double
DP = C.POINTER(C.c_double)

SIGNATURES = {
    "spx_last_error": (C.c_char_p, []),
    "spx_version": (C.c_char_p, []),
    "spx_basis_tables": (I32, [I32, I32, DP, DP, DP, DP, DP]),
    "spx_nodal_basis_tables": (I32, [I32, I32, DP, DP]),
    "spx_gauss_radau": (I32, [I32, DP, DP]),
    "spx_plan_create": (I32, [C.POINTER(P), C.POINTER(PlanDesc)]),
    "spx_plan_destroy": (I32, [P]),
    "spx_plan_sizes": (I32, [P, C.POINTER(I64), C.POINTER(I64)]),
    "spx_plan_offsets": (I32, [P, C.POINTER(I64), C.POINTER(I64)]),
    "spx_plan_device_status": (I32, [P, C.POINTER(C.c_int), I32]),
    "spx_plan_set_geometry": (I32, [P, I32, P, P]),
    "spx_plan_set_tile": (I32, [P, I32, I32, I32, I32, I32, I32]),
    "spx_plan_get_tile": (I32, [P, I32, I32, I32, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "spx_autotune": (I32, [P, I32, I32, P, P, I32, P]),
    "spx_geom_factors": (I32, [P, P, P, P, P, P, P, P]),
    "spx_bwd_trans": (I32, [P, I32, P, P, P]),
    "spx_iproduct": (I32, [P, I32, P, P, P]),
    "spx_phys_deriv": (I32, [P, I32, P, P, P, P, P]),
    "spx_helmholtz": (I32, [P, I32, D, P, P, P, P, P]),
    "spx_helmholtz_adjoint": (I32, [P, P, P, P, P, P]),
    "spx_helmholtz_diag": (I32, [P, I32, D, P, P]),
    "spx_fwd_trans": (I32, [P, I32, P, P, P]),
    "spx_integral": (I32, [P, I32, P, P, P]),
    "spx_sensor": (I32, [P, P, P, P]),
    "spx_adapt_orders": (I32, [I64, P, P, D, D, I32, I32, P]),
    "spx_gather": (I32, [P, I32, P, I64, P, P, P]),
    "spx_assemble": (I32, [P, I32, P, I64, P, P, P]),
    "spx_dot": (I32, [P, I32, I64, P, P, P, P]),
    "spx_cg_workspace_bytes": (I32, [P, I64, C.POINTER(CgOpts), C.POINTER(C.c_size_t)]),
    "spx_cg_solve": (I32, [P, D, P, I64, P, P, P, C.c_size_t, C.POINTER(CgOpts), C.POINTER(CgResult), P]),
    "spx_cg_solve_noalloc": (I32, [P, D, P, I64, P, P, C.POINTER(CgOpts), C.POINTER(CgResult), P]),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"spx CUDA library not found at {LIB_PATH}; build it with "
                "`python -m paper_1906_03489_gb300.build` (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(SIGNATURES)


def check(status):
    if status != 0:
        raise SpxError(status, lib().spx_last_error().decode())
    return status
