"""GB300 (sm_103a) implementation of the hot path of PowerLU (Zhang &
Mascagni, arXiv 2002.07138): the v passes over A, the FP64 LU / QR steps
between them, the blocked rank determination and the LU tail, behind the C
ABI of include/powerlu.h (libpowerlu.so).  This package is the thin Python
binding of that library; it needs the library to be built and never falls
back to another implementation.
"""
from ._binding import (  # noqa: F401
    lib, LIB_PATH, Context, PLUError, plu_matrix, plu_report, as_plu_matrix, colmajor_empty,
    plu_gaussian, plu_pass, plu_lu_reorth, plu_getrf, plu_qr, plu_cholqr1, plu_norm2, plu_rank,
    plu_powerlu, plu_powerlu_fp, plu_randlu, plu_singlepass, plu_batched, plu_batched_tiles,
    plu_set_batched_tile, plu_batched_splitk, plu_set_batched_tune_file,
    plu_batch_problem,
    plu_csr, CsrMatrix, plu_spmm, plu_powerlu_csr, plu_powerlu_fp_csr,
    PREC, STATUS,
    SIGNATURES,
    STREAM_OMEGA_N, STREAM_OMEGA_M, STREAM_OMEGA_SP,
    PLU_FP64, PLU_TF32, PLU_BF16, PLU_FP8_E4M3, PLU_FP32, PLU_TF32X3, PLU_F64, PLU_F32,
)
