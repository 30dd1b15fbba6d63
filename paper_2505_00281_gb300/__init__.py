"""GB300 (sm_103a) orthogonalization-free Rayleigh-Ritz library.

The compute path is the CUDA library ``librr.so`` (C ABI declared in
``include/rr.h``); this package only marshals arguments to it.  Importing
the package does not load the library; the first call does, and raises if the
library is missing.  There is no CPU fallback.
"""
from ._lib import RR, RrError, lib  # noqa: F401
from .api import (  # noqa: F401
    rr_eig, rr_svd, rr_batch_svd, rr_colscale_cast, rr_cast_operator, rr_split_operator, rr_lift, rr_gemm_lowp, rr_gemm_lowp_split,
    rr_gemm_f64, rr_gemm_f64_emulated, rr_hessenberg, rr_hessenberg_blocked, rr_basis_builder, rr_krylov_hessenberg, rr_krylov_eig, rr_gram, rr_gram_noalloc, rr_pencil_eig, rr_pencil_svd, rr_csr_spmm,
    rr_chebyshev_step, rr_chebyshev_step_rows, rr_quantize_e4m3, rr_gemm_e4m3, rr_conv3x3_forward, rr_conv3x3_backward, rr_relu_mask, rr_procrustes_grad, rr_adam,
    rr_net_block, fortran, RrParams, RrOperator, RrInfo,
)
