"""FP64 CPU oracle of the randomized LU algorithms of Zhang & Mascagni,
"Pass-Efficient Randomized LU Algorithms for Computing Low-Rank Matrix
Approximation" (arXiv 2002.07138).

TEST INFRASTRUCTURE ONLY.  Nothing in the library path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2002_07138_gb300``); each side implements
the Philox4x32-10 counter generator and the Gaussian transform on its own.

Every routine is written in the paper's order and notation, in float64, with
numpy primitives (matmul, argmax, norms) as steps and no blocking or fusion:

* ``philox``    -- Philox4x32-10 (Salmon et al., SC'11), the counter generator.
* ``gaussian``  -- the Gaussian test matrices Omega drawn by Algorithms rsvd,
                   bpowerlu, gpowerlu and singlepasslu (Box-Muller on Philox).
* ``lu``        -- partial-pivoting LU, MATLAB ``lu`` semantics (Sec. 2).
* ``qr``        -- economy Householder QR with R_ii >= 0 (Sec. 2, ``qr``).
* ``powerlu``   -- Algorithms gpowerlu, bpowerlu, adaptivewithoutupdating
                   (+ the precise-rank variant of Sec. 6.4), powerlufp,
                   rlu + basicpoweriteration and singlepasslu.
* ``sparse``    -- products with a sparse A in CSR (the sprand experiment
                   of Sec. 6), as passes the algorithms above accept.
* ``metrics``   -- relative Frobenius error (Eq. error), Eckart-Young optimum
                   (Eq. ey) and principal angles.

Parity status of each function is stated in its docstring; all are pinned by
the ``-m "not gpu"`` tests except where a docstring says "parity unpinned".
"""
from .philox import philox4x32_10, STREAM_OMEGA_N, STREAM_OMEGA_M, STREAM_OMEGA_SP
from .gaussian import ln_pos, sincos_turn, gaussian_matrix
from .lu import getrf, lu_permuted_L, lu_full
from .qr import qr_economy
from .powerlu import (gpowerlu, powerlu, adaptive_rank, adaptive_rank_restart, Remainder,
                      RESTART_STREAM_STRIDE, rank_scan, powerlu_fp, randlu,
                      basic_power_iteration_lu, singlepass, PassCounter)
from .sparse import csr_mul, csr_tmul, SparsePassCounter
from .metrics import (rel_lu_error, eckart_young_error, eckart_young_rank,
                      max_principal_sine)

__all__ = [
    "philox4x32_10", "STREAM_OMEGA_N", "STREAM_OMEGA_M", "STREAM_OMEGA_SP",
    "ln_pos", "sincos_turn", "gaussian_matrix",
    "getrf", "lu_permuted_L", "lu_full", "qr_economy",
    "gpowerlu", "powerlu", "adaptive_rank", "adaptive_rank_restart", "Remainder",
    "RESTART_STREAM_STRIDE", "rank_scan", "powerlu_fp", "randlu",
    "basic_power_iteration_lu", "singlepass", "PassCounter",
    "csr_mul", "csr_tmul", "SparsePassCounter",
    "rel_lu_error", "eckart_young_error", "eckart_young_rank", "max_principal_sine",
]
