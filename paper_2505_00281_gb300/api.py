"""Python binding of the C ABI (include/rr.h): argument marshalling only.

Tensors are PyTorch CUDA tensors used as device memory; every computation
runs in librr.so.  Matrices are column-major: a (rows x cols) tensor with
stride (1, ld).  ``fortran(t)`` returns such a copy.
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import RR, RrBatchTuning, RrError, RrInfo, RrOperator, RrParams, check, lib

__all__ = [
    "fortran", "ld_of", "dense_operator", "csr_operator", "kernel_operator", "rr_kernel_apply", "make_params", "rr_eig", "rr_svd",
    "rr_batch_svd", "rr_colscale_cast", "rr_cast_operator", "rr_split_operator", "rr_lift", "rr_gemm_lowp", "rr_gemm_f64",
    "rr_hessenberg", "rr_hessenberg_blocked", "rr_basis_builder", "rr_krylov_hessenberg", "rr_krylov_eig", "rr_wait_selftest", "rr_gram", "rr_gram_noalloc", "rr_pencil_eig", "rr_pencil_svd", "rr_csr_spmm",
    "rr_chebyshev_step", "rr_chebyshev_step_rows", "rr_quantize_e4m3", "rr_gemm_e4m3", "rr_conv3x3_forward", "rr_conv3x3_backward", "rr_relu_mask", "rr_procrustes_grad",
    "rr_adam", "rr_net_block", "RrParams", "RrOperator", "RrInfo", "DTYPES",
]

DTYPES = {torch.float64: RR.F64, torch.float32: RR.F32, torch.bfloat16: RR.BF16}
_BASIS = {"f64": RR.F64, "f32": RR.F32, "bf16": RR.BF16, "e4m3": RR.E4M3}


def fortran(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy (stride (1, rows)) of a 2-D tensor."""
    if t.dim() == 1:
        t = t[:, None]
    return t.t().contiguous().t()


def empty_f(rows: int, cols: int, dtype, device) -> torch.Tensor:
    """Uninitialised column-major (stride (1, rows)) tensor, allocated as such (no copy)."""
    return torch.empty(cols, rows, dtype=dtype, device=device).t()


def ld_of(t: torch.Tensor) -> int:
    if t.dim() == 1:
        return max(1, t.shape[0])
    if t.shape[1] == 1 or t.shape[0] == 0:
        return max(1, t.shape[0])
    if t.shape[0] == 1:
        return max(1, t.stride(1))
    if t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride (1, ld))")
    return t.stride(1)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def dense_operator(A: torch.Tensor) -> RrOperator:
    if A.dtype != torch.float64:
        raise ValueError("dense operator must be FP64")
    op = RrOperator(RR.DENSE, RR.F64, A.shape[0], A.shape[1], ld_of(A), 0, A.data_ptr(), None, None)
    op._keep = (A,)   # the struct holds raw pointers: keep the tensor alive with it
    return op


def csr_operator(row_ptr: torch.Tensor, col_idx: torch.Tensor, values: torch.Tensor) -> RrOperator:
    n = row_ptr.shape[0] - 1
    op = RrOperator(RR.CSR, RR.F32, n, n, n, values.shape[0], values.data_ptr(), row_ptr.data_ptr(),
                    col_idx.data_ptr())
    op._keep = (row_ptr, col_idx, values)
    return op


def kernel_operator(X: torch.Tensor, f: float, l: float, s: float = 0.0, Y: torch.Tensor = None) -> RrOperator:
    """The matrix-free Gaussian kernel operator A(i, j) = f (exp(-|x_i - y_j|^2 /
    (2 l^2)) + s [i == j]) over the rows of X (m x d FP64; Y n x d, or None for
    the square symmetric operator over X)."""
    if X.dtype != torch.float64 or (Y is not None and Y.dtype != torch.float64):
        raise ValueError("kernel points must be FP64")
    Xf = fortran(X)
    Yf = fortran(Y) if Y is not None else None
    n = Y.shape[0] if Y is not None else X.shape[0]
    op = RrOperator(RR.KERNEL, RR.F64, X.shape[0], n, ld_of(Xf), X.shape[1], Xf.data_ptr(), None, None,
                    Yf.data_ptr() if Yf is not None else None)
    op.kparams[0], op.kparams[1], op.kparams[2] = f, l, s
    op._keep = (Xf, Yf)
    return op


def rr_kernel_apply(op: RrOperator, X, trans=False, out_dtype=torch.float32, stream=None):
    """Y = op(A) X for a kernel operator (matrix-free)."""
    rows = op.n if trans else op.m
    Y = empty_f(rows, X.shape[1], out_dtype, X.device)
    check("rr_kernel_apply", lib().rr_kernel_apply(int(trans), ctypes.byref(op), X.shape[1], DTYPES[X.dtype], _p(X),
                                                   ld_of(X), DTYPES[out_dtype], _p(Y), ld_of(Y), None, 0, None,
                                                   _stream(stream)))
    return Y


def make_params(k, block, degree, max_sweeps, tol, basis="bf16", v0=None, filter=RR.POWER,
                which=RR.LARGEST, hessenberg=True, refine=True, phase1_sweeps=1, bounds=(0.0, 0.0),
                profile=False, hess_tol=0.0, seed=0, refine_degree=0):
    p = RrParams()
    p.k, p.block, p.filter, p.degree = k, block, filter, degree
    p.max_sweeps, p.which = max_sweeps, which
    p.basis = _BASIS[basis] if isinstance(basis, str) else basis
    p.hessenberg, p.refine, p.phase1_sweeps = int(hessenberg), int(refine), phase1_sweeps
    p.tol = tol
    p.bounds[0], p.bounds[1] = bounds
    p.v0 = None if v0 is None else v0.data_ptr()
    p.profile = int(profile)
    p.hess_tol = float(hess_tol)
    p.seed = int(seed)
    p.refine_degree = int(refine_degree)
    p._keep = (v0,)
    return p


def _info_dict(info: RrInfo, status: int):
    sweeps = info.sweeps
    return {"status": RR.NAMES.get(status, status), "n_converged": info.n_converged,
            "sweeps": sweeps, "refine_sweeps": info.refine_sweeps, "max_res": info.max_res,
            "res_history": [info.res_history[i] for i in range(min(sweeps, 64))],
            "stage_ms": [info.stage_ms[i] for i in range(8)],
            "stage_calls": [info.stage_calls[i] for i in range(8)],
            "cond_G_est": info.cond_G_est, "cols_dropped": info.cols_dropped, "tc_bytes": info.tc_bytes, "polish_sweeps": info.polish_sweeps,
            "tc_role_ms": list(info.tc_role_ms), "tc_role_bytes": list(info.tc_role_bytes),
            "tc_role_flops": list(info.tc_role_flops),
            "cond_history": [info.cond_history[i] for i in range(min(sweeps, 64))]}


def rr_eig(op: RrOperator, params: RrParams, n: int, device="cuda", stream=None, keep=()):
    """Wanted eigenpairs.  Returns (theta[k], X[n, k], info dict)."""
    L = lib()
    k = params.k
    theta = torch.empty(k, dtype=torch.float64, device=device)
    X = empty_f(n, k, torch.float64, device)
    wsb = L.rr_workspace_size(ctypes.byref(op), ctypes.byref(params), 0)
    if wsb == 0:
        raise RrError("rr_workspace_size", RR.ERR_ARG)
    ws = _ws(wsb, device)
    info = RrInfo()
    st = L.rr_eig(ctypes.byref(op), ctypes.byref(params), _p(theta), _p(X), _p(ws), ws.numel(),
                  ctypes.byref(info), _stream(stream))
    if st not in (RR.OK, RR.ERR_NO_CONV):
        check("rr_eig", st)
    return theta, X, _info_dict(info, st)


def rr_svd(op: RrOperator, params: RrParams, device="cuda", stream=None, ws=None):
    """Largest singular triplets.  Returns (sigma[k], U[m, k], V[n, k], info dict)."""
    L = lib()
    k, m, n = params.k, op.m, op.n
    sigma = torch.empty(k, dtype=torch.float64, device=device)
    U = empty_f(m, k, torch.float64, device)
    V = empty_f(n, k, torch.float64, device)
    wsb = L.rr_workspace_size(ctypes.byref(op), ctypes.byref(params), 1)
    if wsb == 0:
        raise RrError("rr_workspace_size", RR.ERR_ARG)
    if ws is None or ws.numel() < wsb:
        ws = _ws(wsb, device)
    info = RrInfo()
    st = L.rr_svd(ctypes.byref(op), ctypes.byref(params), _p(sigma), _p(U), _p(V), _p(ws), ws.numel(),
                  ctypes.byref(info), _stream(stream))
    if st not in (RR.OK, RR.ERR_NO_CONV):
        check("rr_svd", st)
    return sigma, U, V, _info_dict(info, st)


def rr_batch_svd(ops, params: RrParams, seed: int, device="cuda", stream=None, tuning=None):
    """Batched SVDs in one graph launch.  Returns (list of (sigma, U, V), statuses, infos).
    tuning: None (library defaults) or a dict with branches, max_splits, order and
    optionally fixed_sweeps (1: every problem runs max_sweeps sweeps; default 0:
    each problem stops at tol under device-side loop control)."""
    L = lib()
    cnt = len(ops)
    arr = (RrOperator * cnt)(*ops)
    k = params.k
    outs = [(torch.empty(k, dtype=torch.float64, device=device),
             empty_f(o.m, k, torch.float64, device),
             empty_f(o.n, k, torch.float64, device)) for o in ops]
    S = (ctypes.c_void_p * cnt)(*[o[0].data_ptr() for o in outs])
    U = (ctypes.c_void_p * cnt)(*[o[1].data_ptr() for o in outs])
    V = (ctypes.c_void_p * cnt)(*[o[2].data_ptr() for o in outs])
    wsb = L.rr_batch_workspace_size(cnt, arr, ctypes.byref(params))
    if wsb == 0:
        raise RrError("rr_batch_workspace_size", RR.ERR_ARG)
    ws = _ws(wsb, device)
    per = (ctypes.c_int32 * cnt)()
    infos = (RrInfo * cnt)()
    if tuning is None:
        st = L.rr_batch_svd(cnt, arr, ctypes.byref(params), seed, S, U, V, _p(ws), ws.numel(), per, infos,
                            _stream(stream))
    else:
        t = RrBatchTuning(int(tuning["branches"]), int(tuning["max_splits"]), int(tuning["order"]),
                          int(tuning.get("fixed_sweeps", 0)))
        st = L.rr_batch_svd_tuned(cnt, arr, ctypes.byref(params), seed, S, U, V, _p(ws), ws.numel(),
                                  ctypes.byref(t), per, infos, _stream(stream))
    if st not in (RR.OK, RR.ERR_NO_CONV):
        check("rr_batch_svd", st)
    return outs, [int(x) for x in per], [_info_dict(infos[i], per[i]) for i in range(cnt)]


# ---------------------------------------------------------------- stages
def rr_colscale_cast(X, dtype, stream=None):
    rows, cols = X.shape
    Y = empty_f(rows, cols, dtype, X.device)
    scale = torch.empty(cols, dtype=torch.float64, device=X.device)
    check("rr_colscale_cast", lib().rr_colscale_cast(rows, cols, _p(X), ld_of(X), DTYPES[dtype], _p(Y),
                                                      ld_of(Y), _p(scale), _stream(stream)))
    return Y, scale


def rr_cast_operator(A, dtype, row_copy=True, stream=None):
    m, n = A.shape
    col = empty_f(m, n, dtype, A.device)
    row = torch.empty(m * n, dtype=dtype, device=A.device) if row_copy else None
    check("rr_cast_operator", lib().rr_cast_operator(m, n, _p(A), ld_of(A), DTYPES[dtype], _p(col),
                                                      _p(row), _stream(stream)))
    return col, row


def rr_split_operator(A, row_copy=True, stream=None):
    """hi = bf16(A), lo = bf16(A - hi): (hi_col, hi_row, lo_col, lo_row); row copies flat or None."""
    m, n = A.shape
    hc = empty_f(m, n, torch.bfloat16, A.device)
    lc = empty_f(m, n, torch.bfloat16, A.device)
    hr = torch.empty(m * n, dtype=torch.bfloat16, device=A.device) if row_copy else None
    lr = torch.empty(m * n, dtype=torch.bfloat16, device=A.device) if row_copy else None
    check("rr_split_operator", lib().rr_split_operator(m, n, _p(A), ld_of(A), _p(hc), _p(hr), _p(lc), _p(lr),
                                                        _stream(stream)))
    return hc, hr, lc, lr


def rr_lift(S1, Y, S2=None, X=None, stream=None):
    """X = [S1 S2] Y (FP64 result; S1, S2 column-major FP64 / FP32 / BF16, Y FP64)."""
    n, p1 = S1.shape
    p2 = S2.shape[1] if S2 is not None else 0
    b = Y.shape[1]
    if X is None:
        X = empty_f(n, b, torch.float64, Y.device)
    L = lib()
    ws = _ws(L.rr_lift_workspace_size(n, b, p1 + p2), Y.device)
    check("rr_lift", L.rr_lift(n, b, DTYPES[S1.dtype], _p(S1), ld_of(S1), p1,
                               DTYPES[S2.dtype] if S2 is not None else 0, _p(S2), ld_of(S2) if S2 is not None else n,
                               p2, _p(Y), ld_of(Y), _p(X), ld_of(X), _p(ws), ws.numel(), _stream(stream)))
    return X


def rr_gemm_lowp(dtype, M, N, K, A_k, lda, B, ldb, C=None, R=None, coef=None, stream=None):
    if C is None:
        C = empty_f(M, N, torch.float32, B.device)
    check("rr_gemm_lowp", lib().rr_gemm_lowp(dtype, M, N, K, _p(A_k), lda, _p(B), ldb, _p(C), ld_of(C),
                                              _p(R), ld_of(R) if R is not None else 0, _p(coef),
                                              _stream(stream)))
    return C


def rr_gemm_lowp_split(M, N, K, A_hi, A_lo, lda, B_hi, B_lo, ldb, C=None, R=None, coef=None, stream=None):
    if C is None:
        C = empty_f(M, N, torch.float32, B_hi.device)
    check("rr_gemm_lowp_split", lib().rr_gemm_lowp_split(M, N, K, _p(A_hi), _p(A_lo), lda, _p(B_hi), _p(B_lo),
                                                          ldb, _p(C), ld_of(C), _p(R),
                                                          ld_of(R) if R is not None else 0, _p(coef),
                                                          _stream(stream)))
    return C


def rr_gemm_f64(trans, A, B, C=None, accumulate=False, stream=None):
    M = A.shape[1] if trans else A.shape[0]
    K = A.shape[0] if trans else A.shape[1]
    N = B.shape[1]
    if C is None:
        C = fortran(torch.zeros(M, N, dtype=torch.float64, device=B.device))
    check("rr_gemm_f64", lib().rr_gemm_f64(int(trans), M, N, K, _p(A), ld_of(A), _p(B), ld_of(B), _p(C),
                                            ld_of(C), int(accumulate), _stream(stream)))
    return C


def rr_gemm_f64_emulated(trans, A, B, slices=8, C=None, stream=None):
    M = A.shape[1] if trans else A.shape[0]
    K = A.shape[0] if trans else A.shape[1]
    N = B.shape[1]
    if C is None:
        C = empty_f(M, N, torch.float64, B.device)
    L = lib()
    ws = _ws(L.rr_gemm_f64_emulated_workspace_size(int(trans), M, N, K, slices), B.device)
    check("rr_gemm_f64_emulated", L.rr_gemm_f64_emulated(int(trans), M, N, K, _p(A), ld_of(A), _p(B),
                                                          ld_of(B), _p(C), ld_of(C), slices, _p(ws),
                                                          ws.numel(), _stream(stream)))
    return C


def rr_hessenberg(W, qtype=torch.bfloat16, tol=0.0, stream=None):
    """Algorithm 8 on W (FP32 or FP64, modified in place).  Returns (Q, piv, err)."""
    n, k = W.shape
    arith = DTYPES[W.dtype]
    Q = empty_f(n, k, qtype, W.device)
    piv = torch.empty(k, dtype=torch.int32, device=W.device)
    L = lib()
    wsb = L.rr_hessenberg_workspace_size(n, k, arith)
    ws = _ws(wsb, W.device)
    check("rr_hessenberg", L.rr_hessenberg(arith, n, k, _p(W), ld_of(W), DTYPES[qtype], _p(Q), ld_of(Q),
                                           _p(piv), tol, _p(ws), ws.numel(), _stream(stream)))
    err = ws[:4].view(torch.int32)
    return Q, piv, err


def rr_hessenberg_blocked(W, panel, qtype=torch.bfloat16, tol=0.0, stream=None):
    """Blocked Algorithm 8 on W (FP32, modified in place) in panels of `panel`
    columns.  Returns (Q, piv, err)."""
    n, k = W.shape
    Q = empty_f(n, k, qtype, W.device)
    piv = torch.empty(k, dtype=torch.int32, device=W.device)
    L = lib()
    ws = _ws(L.rr_hessenberg_workspace_size(n, k, RR.F32), W.device)
    check("rr_hessenberg_blocked", L.rr_hessenberg_blocked(n, k, _p(W), ld_of(W), DTYPES[qtype], _p(Q), ld_of(Q),
                                                           _p(piv), tol, int(panel), _p(ws), ws.numel(),
                                                           _stream(stream)))
    return Q, piv, ws[:4].view(torch.int32)


def rr_krylov_hessenberg(row_ptr, col_idx, values, v, k, dtype=torch.float64, stream=None):
    """Alg. 7 on a CSR operator.  Returns (V, AV, H, piv) on the device."""
    n = row_ptr.shape[0] - 1
    L = lib()
    V = empty_f(n, k, dtype, v.device)
    AV = empty_f(n, k, dtype, v.device)
    H = empty_f(k, k, torch.float64, v.device)
    piv = torch.empty(k, dtype=torch.int32, device=v.device)
    ws = _ws(L.rr_krylov_hessenberg_workspace_size(n, k, DTYPES[dtype]), v.device)
    check("rr_krylov_hessenberg", L.rr_krylov_hessenberg(DTYPES[dtype], n, k, _p(row_ptr), _p(col_idx), _p(values),
                                                         _p(v), _p(V), _p(AV), n, _p(H), _p(piv), _p(ws),
                                                         ws.numel(), _stream(stream)))
    return V, AV, H, piv


def rr_krylov_eig(op: RrOperator, v0, m, restarts, k, dtype=torch.float64, stream=None):
    """Alg. 7 + Alg. 3 with restarts.  Returns (theta[k], X[n, k], res[k])."""
    L = lib()
    n = op.n
    theta = torch.empty(k, dtype=torch.float64, device=v0.device)
    X = empty_f(n, k, torch.float64, v0.device)
    res = torch.empty(k, dtype=torch.float64, device=v0.device)
    wsb = L.rr_krylov_workspace_size(n, m, k, DTYPES[dtype])
    if wsb == 0:
        raise RrError("rr_krylov_workspace_size", RR.ERR_ARG)
    ws = _ws(wsb, v0.device)
    check("rr_krylov_eig", L.rr_krylov_eig(ctypes.byref(op), m, restarts, k, DTYPES[dtype], _p(v0), _p(theta), _p(X),
                                           _p(res), _p(ws), ws.numel(), _stream(stream)))
    return theta, X, res


BUILDERS = {"mgs_l": RR.MGS_L, "mgs_r": RR.MGS_R, "cgs": RR.CGS, "cgs2": RR.CGS2, "hess_l": RR.HESS_L,
            "hess_r": RR.HESS_R}


def rr_basis_builder(W, method, want_r=True, stream=None):
    """One of the comparator basis builders on W (FP64 / FP32 / FP16, modified
    in place into the basis Q).  Returns (Q, R or None, piv or None)."""
    n, k = W.shape
    m = BUILDERS[method] if isinstance(method, str) else method
    storage = {torch.float64: RR.F64, torch.float32: RR.F32, torch.float16: RR.F16}[W.dtype]
    L = lib()
    ws = _ws(L.rr_basis_builder_workspace_size(m, storage, n, k), W.device)
    hess = m in (RR.HESS_L, RR.HESS_R)
    R = fortran(torch.zeros(k, k, dtype=torch.float64, device=W.device)) if (want_r and not hess) else None
    piv = torch.empty(k, dtype=torch.int32, device=W.device) if hess else None
    check("rr_basis_builder", L.rr_basis_builder(m, storage, n, k, _p(W), ld_of(W), _p(R), _p(piv), _p(ws),
                                                 ws.numel(), _stream(stream)))
    return W, R, piv


def rr_gram(X, Y, G=None, accumulate=False, stream=None):
    n, p = X.shape
    q = Y.shape[1]
    if G is None:
        G = fortran(torch.zeros(p, q, dtype=torch.float64, device=X.device))
    L = lib()
    ws = _ws(L.rr_gram_workspace_size(n, p, q), X.device)
    check("rr_gram", L.rr_gram(n, p, q, DTYPES[X.dtype], _p(X), ld_of(X), DTYPES[Y.dtype], _p(Y), ld_of(Y),
                               _p(G), ld_of(G), int(accumulate), _p(ws), ws.numel(), _stream(stream)))
    return G


def rr_wait_selftest(mode, limit_ns, device="cuda", stream=None):
    """Run one of the library's bounded waits where nothing releases it;
    returns the status the kernel reported (RR.ERR_TIMEOUT expected)."""
    scratch = torch.empty(16, dtype=torch.uint8, device=device)
    return lib().rr_wait_selftest(int(mode), int(limit_ns), _p(scratch), _stream(stream))


def rr_gram_noalloc(X, Y, G=None, accumulate=False, stream=None):
    """rr_gram without a workspace: scratch is a fixed array inside the library."""
    n, p = X.shape
    q = Y.shape[1]
    if G is None:
        G = fortran(torch.zeros(p, q, dtype=torch.float64, device=X.device))
    check("rr_gram_noalloc", lib().rr_gram_noalloc(n, p, q, DTYPES[X.dtype], _p(X), ld_of(X), DTYPES[Y.dtype],
                                                    _p(Y), ld_of(Y), _p(G), ld_of(G), int(accumulate),
                                                    _stream(stream)))
    return G


def rr_pencil_eig(H, G, stream=None):
    b = H.shape[0]
    theta = torch.empty(b, dtype=torch.float64, device=H.device)
    Y = empty_f(b, b, torch.float64, H.device)
    L = lib()
    ws = _ws(L.rr_pencil_workspace_size(b, b), H.device)
    dropped = ctypes.c_int32(0)
    check("rr_pencil_eig", L.rr_pencil_eig(b, _p(H), _p(G), _p(theta), _p(Y), _p(ws), ws.numel(),
                                           ctypes.byref(dropped), _stream(stream)))
    return theta, Y, dropped.value


def rr_pencil_svd(B, Gu, Gv, stream=None):
    b1, b2 = B.shape
    r = min(b1, b2)
    s = torch.empty(r, dtype=torch.float64, device=B.device)
    Y = empty_f(b1, r, torch.float64, B.device)
    Z = empty_f(b2, r, torch.float64, B.device)
    L = lib()
    ws = _ws(L.rr_pencil_workspace_size(b1, b2), B.device)
    dropped = ctypes.c_int32(0)
    check("rr_pencil_svd", L.rr_pencil_svd(b1, b2, _p(B), _p(Gu), _p(Gv), _p(s), _p(Y), _p(Z), _p(ws),
                                           ws.numel(), ctypes.byref(dropped), _stream(stream)))
    return s, Y, Z, dropped.value


def rr_csr_spmm(row_ptr, col_idx, values, X, out_dtype=torch.float32, stream=None):
    n, b = X.shape
    Y = empty_f(n, b, out_dtype, X.device)
    check("rr_csr_spmm", lib().rr_csr_spmm(n, b, _p(row_ptr), _p(col_idx), _p(values), DTYPES[X.dtype],
                                           _p(X), ld_of(X), DTYPES[out_dtype], _p(Y), ld_of(Y),
                                           _stream(stream)))
    return Y


def rr_chebyshev_step(row_ptr, col_idx, values, Y_cur, Y_prev, alpha, c, beta, beta_col=None, R=None,
                      gamma=None, out_dtype=None, stream=None):
    n, b = Y_cur.shape
    out_dtype = out_dtype or Y_cur.dtype
    Yn = empty_f(n, b, out_dtype, Y_cur.device)
    check("rr_chebyshev_step", lib().rr_chebyshev_step(
        n, b, _p(row_ptr), _p(col_idx), _p(values), DTYPES[Y_cur.dtype], _p(Y_cur), _p(Y_prev),
        ld_of(Y_cur), alpha, c, beta, _p(beta_col), _p(R), ld_of(R) if R is not None else 0, _p(gamma),
        DTYPES[out_dtype], _p(Yn), ld_of(Yn), _stream(stream)))
    return Yn


def rr_chebyshev_step_rows(row_ptr, col_idx, values, Y_cur, Y_prev, b, alpha, c, beta, out_dtype=None,
                           stream=None):
    """Row-major step: Y_cur, Y_prev (n, ldr) contiguous, columns 0 .. b-1 used (pad columns too)."""
    n, ldr = Y_cur.shape
    out_dtype = out_dtype or Y_cur.dtype
    Yn = torch.empty(n, ldr, dtype=out_dtype, device=Y_cur.device)
    check("rr_chebyshev_step_rows", lib().rr_chebyshev_step_rows(
        n, b, _p(row_ptr), _p(col_idx), _p(values), DTYPES[Y_cur.dtype], _p(Y_cur), _p(Y_prev), ldr, alpha, c,
        beta, DTYPES[out_dtype], _p(Yn), ldr, _stream(stream)))
    return Yn


def rr_quantize_e4m3(X, by_rows=False, stream=None):
    """E4M3 copy of the FP64 column-major X with power-of-two scales per column
    (Q column-major, (rows, ldq) uint8 view) or per row (Q row-major).
    Returns (Q uint8 tensor, inv_scale FP32).  ld is rounded up to 16 bytes."""
    rows, cols = X.shape
    inner = cols if by_rows else rows
    ldq = -(-max(inner, 1) // 16) * 16
    outer = rows if by_rows else cols
    Q = torch.zeros(outer, ldq, dtype=torch.uint8, device=X.device)   # each line contiguous
    inv = torch.empty(outer, dtype=torch.float32, device=X.device)
    scratch = torch.empty(max(rows, cols, 1), dtype=torch.int64, device=X.device)
    check("rr_quantize_e4m3", lib().rr_quantize_e4m3(rows, cols, _p(X), ld_of(X), int(by_rows), _p(Q), ldq,
                                                     _p(inv), _p(scratch), _stream(stream)))
    return Q, inv


def rr_gemm_e4m3(M, N, K, A_q, a_scale, B_q, b_scale, stream=None):
    """C (M x N FP32, column-major) = diag(a_scale) A_q^T B_q diag(b_scale); A_q (M, lda) and
    B_q (N, ldb) uint8 tensors whose lines are the K-contiguous rows of A and columns of B."""
    C = empty_f(M, N, torch.float32, A_q.device)
    check("rr_gemm_e4m3", lib().rr_gemm_e4m3(M, N, K, _p(A_q), A_q.stride(0), _p(a_scale), _p(B_q), B_q.stride(0),
                                             _p(b_scale), _p(C), ld_of(C), _stream(stream)))
    return C


def _nchw(t):
    if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 4:
        raise ValueError("expected a contiguous FP32 (N, C, H, W) tensor")
    return t


def rr_conv3x3_forward(x, w, b, relu=False, add=None, y=None, stream=None):
    """y = [relu](conv3x3(x, w) + b [+ add]); `add` is (N, O, H, W) or a view with that shape."""
    N, C, H, W = _nchw(x).shape
    O = w.shape[0]
    if y is None:
        y = torch.empty(N, O, H, W, dtype=torch.float32, device=x.device)
    nstride = add.stride(0) if add is not None else 0
    check("rr_conv3x3_forward", lib().rr_conv3x3_forward(N, C, H, W, O, _p(x), _p(w), _p(b), _p(add), nstride,
                                                         int(relu), _p(y), _stream(stream)))
    return y


def rr_conv3x3_backward(x, w, g, dw, db, need_dx=True, stream=None):
    """Adds dL/dw, dL/db into dw, db; returns dL/dx (or None)."""
    N, C, H, W = _nchw(x).shape
    O = w.shape[0]
    dx = torch.empty_like(x) if need_dx else None
    check("rr_conv3x3_backward", lib().rr_conv3x3_backward(N, C, H, W, O, _p(x), _p(w), _p(_nchw(g)), _p(dx),
                                                           _p(dw), _p(db), _stream(stream)))
    return dx


def rr_relu_mask(g, act, stream=None):
    check("rr_relu_mask", lib().rr_relu_mask(g.numel(), _p(g), _p(act), _stream(stream)))
    return g


def rr_procrustes_grad(out, Vstar, U, Wm, scale, grad=None, loss=None, stream=None):
    """out: network output (k, n) rows = channels (any contiguous view); returns (grad like out, loss[1] FP64)."""
    k = Vstar.shape[1]
    n = Vstar.shape[0]
    grad = torch.empty_like(out) if grad is None else grad
    loss = torch.zeros(1, dtype=torch.float64, device=out.device) if loss is None else loss
    check("rr_procrustes_grad", lib().rr_procrustes_grad(n, k, _p(out), _p(Vstar), _p(U), _p(Wm),
                                                         float(scale), _p(grad), _p(loss), _stream(stream)))
    return grad, loss


def rr_adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    check("rr_adam", lib().rr_adam(p.numel(), _p(p), _p(g), _p(m), _p(v), float(lr), float(b1), float(b2),
                                   float(eps), int(t), _stream(stream)))


def rr_net_block(out, scale, V, stream=None):
    """V[:, :k] = scale * out, out the (k, n) channel-major network output."""
    k = out.shape[0] if out.dim() == 2 else out.shape[-3]
    n = V.shape[0]
    check("rr_net_block", lib().rr_net_block(n, k, _p(out), float(scale), _p(V), ld_of(V), _stream(stream)))
    return V
