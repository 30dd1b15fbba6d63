"""ctypes declarations of the C ABI in include/rr.h (marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librr.so")

c_i32, c_i64, c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
c_dbl, c_sz, c_vp = ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
c_i32p = ctypes.POINTER(ctypes.c_int32)


class RR:
    F64, F32, BF16, E4M3, F16 = 0, 1, 2, 3, 4
    MGS_L, MGS_R, CGS, CGS2, HESS_L, HESS_R = range(6)
    OK, ERR_ARG, ERR_CUDA, ERR_NOT_SPD, ERR_NO_CONV, ERR_TIMEOUT, ERR_WORKSPACE, ERR_NAN = range(8)
    DENSE, CSR, KERNEL = 0, 1, 2
    LARGEST, SMALLEST = 0, 1
    POWER, CHEBYSHEV = 0, 1
    NAMES = {0: "RR_OK", 1: "RR_ERR_ARG", 2: "RR_ERR_CUDA", 3: "RR_ERR_NOT_SPD",
             4: "RR_ERR_NO_CONV", 5: "RR_ERR_TIMEOUT", 6: "RR_ERR_WORKSPACE", 7: "RR_ERR_NAN"}


class RrError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{fn} returned {RR.NAMES.get(status, status)}" + (f": {detail}" if detail else ""))


class RrOperator(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("dtype", c_i32), ("m", c_i64), ("n", c_i64), ("ld", c_i64),
                ("nnz", c_i64), ("values", c_vp), ("row_ptr", c_vp), ("col_idx", c_vp), ("points_y", c_vp),
                ("kparams", c_dbl * 3)]


class RrParams(ctypes.Structure):
    _fields_ = [("k", c_i32), ("block", c_i32), ("filter", c_i32), ("degree", c_i32),
                ("max_sweeps", c_i32), ("which", c_i32), ("basis", c_i32), ("hessenberg", c_i32),
                ("refine", c_i32), ("phase1_sweeps", c_i32), ("tol", c_dbl),
                ("bounds", c_dbl * 2), ("v0", c_vp), ("profile", c_i32), ("hess_tol", c_dbl),
                ("seed", c_u64), ("refine_degree", c_i32)]


class RrBatchTuning(ctypes.Structure):
    _fields_ = [("branches", c_i32), ("max_splits", c_i32), ("order", c_i32), ("fixed_sweeps", c_i32)]


class RrInfo(ctypes.Structure):
    _fields_ = [("n_converged", c_i32), ("sweeps", c_i32), ("refine_sweeps", c_i32),
                ("cols_dropped", c_i32), ("max_res", c_dbl), ("res_history", c_dbl * 64),
                ("stage_ms", c_dbl * 8), ("stage_calls", c_i32 * 8), ("cond_G_est", c_dbl),
                ("cond_history", c_dbl * 64), ("tc_bytes", c_dbl), ("polish_sweeps", c_i32),
                ("tc_role_ms", c_dbl * 2), ("tc_role_bytes", c_dbl * 2), ("tc_role_flops", c_dbl * 2)]


_SIGS = {
    "rr_last_error": (ctypes.c_char_p, []),
    "rr_kernel_launches": (c_u64, []),
    "rr_workspace_size": (c_sz, [ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams), ctypes.c_int]),
    "rr_eig": (c_i32, [ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams), c_vp, c_vp, c_vp, c_sz,
                       ctypes.POINTER(RrInfo), c_vp]),
    "rr_svd": (c_i32, [ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams), c_vp, c_vp, c_vp, c_vp,
                       c_sz, ctypes.POINTER(RrInfo), c_vp]),
    "rr_batch_workspace_size": (c_sz, [c_i32, ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams)]),
    "rr_batch_svd": (c_i32, [c_i32, ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams), c_u64,
                             ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_vp,
                             c_sz, c_i32p, ctypes.POINTER(RrInfo), c_vp]),
    "rr_batch_svd_tuned": (c_i32, [c_i32, ctypes.POINTER(RrOperator), ctypes.POINTER(RrParams), c_u64,
                                   ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_vp,
                                   c_sz, ctypes.POINTER(RrBatchTuning), c_i32p, ctypes.POINTER(RrInfo), c_vp]),
    "rr_colscale_cast": (c_i32, [c_i64, c_i64, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_vp]),
    "rr_cast_operator": (c_i32, [c_i64, c_i64, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp]),
    "rr_split_operator": (c_i32, [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "rr_lift_workspace_size": (c_sz, [c_i64, c_i64, c_i64]),
    "rr_lift": (c_i32, [c_i64, c_i64, c_i32, c_vp, c_i64, c_i64, c_i32, c_vp, c_i64, c_i64, c_vp, c_i64, c_vp,
                        c_i64, c_vp, c_sz, c_vp]),
    "rr_gemm_lowp": (c_i32, [c_i32, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp,
                             c_i64, c_vp, c_vp]),
    "rr_gemm_lowp_split": (c_i32, [c_i64, c_i64, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_i64,
                                   c_vp, c_i64, c_vp, c_vp]),
    "rr_gemm_f64": (c_i32, [c_i32, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_i32,
                            c_vp]),
    "rr_gemm_f64_emulated_workspace_size": (c_sz, [c_i32, c_i64, c_i64, c_i64, c_i32]),
    "rr_gemm_f64_emulated": (c_i32, [c_i32, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64,
                                     c_i32, c_vp, c_sz, c_vp]),
    "rr_hessenberg_workspace_size": (c_sz, [c_i64, c_i64, c_i32]),
    "rr_hessenberg": (c_i32, [c_i32, c_i64, c_i64, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_dbl, c_vp,
                              c_sz, c_vp]),
    "rr_gram_workspace_size": (c_sz, [c_i64, c_i64, c_i64]),
    "rr_gram": (c_i32, [c_i64, c_i64, c_i64, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_i64, c_i32,
                        c_vp, c_sz, c_vp]),
    "rr_wait_selftest": (c_i32, [c_i32, c_i64, c_vp, c_vp]),
    "rr_hessenberg_blocked": (c_i32, [c_i64, c_i64, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_dbl, c_i32, c_vp,
                                      c_sz, c_vp]),
    "rr_krylov_hessenberg_workspace_size": (c_sz, [c_i64, c_i32, c_i32]),
    "rr_krylov_hessenberg": (c_i32, [c_i32, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp,
                                     c_vp, c_sz, c_vp]),
    "rr_krylov_workspace_size": (c_sz, [c_i64, c_i32, c_i32, c_i32]),
    "rr_krylov_eig": (c_i32, [ctypes.POINTER(RrOperator), c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp,
                              c_vp, c_sz, c_vp]),
    "rr_kernel_apply": (c_i32, [c_i32, ctypes.POINTER(RrOperator), c_i64, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64,
                                c_vp, c_i64, c_vp, c_vp]),
    "rr_basis_builder_workspace_size": (c_sz, [c_i32, c_i32, c_i64, c_i64]),
    "rr_basis_builder": (c_i32, [c_i32, c_i32, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "rr_gram_noalloc": (c_i32, [c_i64, c_i64, c_i64, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_i64,
                                c_i32, c_vp]),
    "rr_pencil_workspace_size": (c_sz, [c_i64, c_i64]),
    "rr_pencil_eig": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_i32p, c_vp]),
    "rr_pencil_svd": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_i32p,
                              c_vp]),
    "rr_csr_spmm": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64,
                            c_vp]),
    "rr_chebyshev_step": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_i64, c_dbl,
                                  c_dbl, c_dbl, c_vp, c_vp, c_i64, c_vp, c_i32, c_vp, c_i64, c_vp]),
    "rr_chebyshev_step_rows": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_i64, c_dbl, c_dbl,
                                       c_dbl, c_i32, c_vp, c_i64, c_vp]),
    "rr_quantize_e4m3": (c_i32, [c_i64, c_i64, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "rr_gemm_e4m3": (c_i32, [c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp]),
    "rr_conv3x3_forward": (c_i32, [c_i32, c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_i64, c_i32,
                                   c_vp, c_vp]),
    "rr_conv3x3_backward": (c_i32, [c_i32, c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                    c_vp]),
    "rr_relu_mask": (c_i32, [c_i64, c_vp, c_vp, c_vp]),
    "rr_procrustes_grad": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, ctypes.c_float, c_vp, c_vp, c_vp]),
    "rr_adam": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                        ctypes.c_float, c_i32, c_vp]),
    "rr_net_block": (c_i32, [c_i64, c_i32, c_vp, ctypes.c_float, c_vp, c_i64, c_vp]),
}

EXPORTED = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load librr.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(fn: str, status: int) -> int:
    if status != RR.OK:
        detail = lib().rr_last_error().decode() if status == RR.ERR_CUDA else ""
        raise RrError(fn, status, detail)
    return status
