"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds none of PowerLU's arithmetic: it only builds test matrices
A = U diag(sigma) V^T with U, V orthonormal factors of seeded Gaussian
matrices -- the construction of the paper's accuracy experiments (Sec. 6.2,
"Matrix Type 1/2/3") -- plus the workload descriptions of the benchmark
configurations.  Random draws here use numpy's PCG64 (CPU) or torch's
Philox (CUDA) generators, never the generator of the method's Omega.

Matrices are returned column-major (Fortran order): numpy arrays with
order='F', or torch tensors of shape (m, n) and strides (1, m).
"""
import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# singular value profiles
# --------------------------------------------------------------------------
def sigma_profile(name, count, k=None):
    """Singular values sigma_1..sigma_count of the named profile.

    type1: 1/i^2 (Sec. 6.2, slow decay)       type2: exp(-i/7) (fast decay)
    type3: 1e-4 + 1/(1 + exp(i - 30)) (S-shaped)
    exp20: exp(-i/20)        pow15: i^-1.5        inv: 1/i
    gap400: 1/i for i <= 400, 0.01/i beyond (a 100x gap at i = 400)
    expk:  exp(-i/k)
    """
    i = np.arange(1, count + 1, dtype=np.float64)
    if name == "type1":
        return 1.0 / i ** 2
    if name == "type2":
        return np.exp(-i / 7.0)
    if name == "type3":
        return 1e-4 + np.exp(-np.logaddexp(0.0, i - 30.0))   # 1/(1 + e^(i-30))
    if name == "exp20":
        return np.exp(-i / 20.0)
    if name == "pow15":
        return i ** -1.5
    if name == "inv":
        return 1.0 / i
    if name == "gap400":
        return np.where(i <= 400, 1.0 / i, 0.01 / i)
    if name == "expk":
        return np.exp(-i / float(k))
    if name == "flat12":           # well-conditioned, sigma in [1, 2]
        return np.linspace(2.0, 1.0, count)
    raise ValueError(name)


# --------------------------------------------------------------------------
# CPU (numpy) generators, float64
# --------------------------------------------------------------------------
def orthonormal_np(rows, cols, rng):
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def svd_matrix_np(m, n, sigma, seed, noise=0.0):
    """A = U diag(sigma) V^T (+ noise * N(0,1) entries), float64, Fortran order."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = orthonormal_np(m, r, rng)
    V = orthonormal_np(n, r, rng)
    A = (U * np.asarray(sigma)[None, :]) @ V.T
    if noise:
        A = A + noise * rng.standard_normal((m, n))
    return np.asfortranarray(A)


def rank_k_matrix_np(m, n, k, seed):
    """Exact rank-k A = B C with Gaussian B (m x k), C (k x n)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, k))
    C = rng.standard_normal((k, n))
    return np.asfortranarray(B @ C)


def gaussian_np(m, n, seed):
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((m, n)))


# --------------------------------------------------------------------------
# torch generators (CPU or CUDA), for sizes numpy cannot build quickly
# --------------------------------------------------------------------------
def colmajor(t):
    """Column-major copy of a 2-D torch tensor: shape (m, n), strides (1, m)."""
    return t.t().contiguous().t()


def _preload_torch_linalg():
    """Load torch's CUDA linear-algebra library by absolute path (its lazy
    load by name fails under some profilers' injected environments)."""
    import ctypes
    import os
    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        try:
            ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def svd_matrix_torch(m, n, sigma, seed, device="cuda", dtype=None, noise=0.0,
                     work_dtype=None):
    """A = U diag(sigma) V^T built with torch (QR of seeded Gaussians) on
    ``device``; returned column-major in ``dtype``."""
    import torch
    if str(device).startswith("cuda"):
        _preload_torch_linalg()
    dtype = dtype or torch.float32
    work_dtype = work_dtype or (torch.float64 if max(m, n) <= 4096 else torch.float32)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    r = len(sigma)
    s = torch.as_tensor(np.asarray(sigma), device=device, dtype=work_dtype)

    def orth(rows, cols):
        G = torch.randn(rows, cols, generator=g, device=device, dtype=work_dtype)
        Q, R = torch.linalg.qr(G)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1
        Q.mul_(d[None, :])
        return Q

    U = orth(m, r)
    V = orth(n, r)
    U.mul_(s[None, :])
    # build A^T row-major = A column-major, so the result needs no transpose copy
    At = V @ U.t()                                       # n x m, contiguous
    del U, V
    if noise:
        At.add_(torch.randn(n, m, generator=g, device=device, dtype=work_dtype),
                alpha=float(noise))
    At = At.to(dtype)
    return At.t()                                        # (m, n), strides (1, m)


# --------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    m: int
    n: int
    sigma: str
    k: int = 0
    l: int = 0
    v: int = 2
    storage: str = "f64"          # dtype A is stored in
    noise: float = 0.0
    eps: float = 0.0
    b: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    def sigma_values(self):
        return sigma_profile(self.sigma, min(self.m, self.n))

    def build(self, device="cpu"):
        """Column-major A: numpy float64 on 'cpu', torch tensor on CUDA."""
        sig = self.sigma_values()
        if device == "cpu":
            A = svd_matrix_np(self.m, self.n, sig, self.seed, noise=self.noise)
            return A if self.storage == "f64" else np.asfortranarray(A.astype(np.float32))
        import torch
        dt = torch.float64 if self.storage == "f64" else torch.float32
        return svd_matrix_torch(self.m, self.n, sig, self.seed, device=device, dtype=dt,
                                noise=self.noise)


# The five configurations of the paper's hot path (sizes in the spirit of
# Sec. 6: square dense matrices up to 32k, l = k + 10 or k + 20).
PLAIN_2000x1500 = Workload("plain_fp64_2000x1500_k20_l25_v2", 2000, 1500, "type1",
                           k=20, l=25, v=2, storage="f64")
FIXED_RANK_8192 = Workload("fixed_rank_8192_k100_l110", 8192, 8192, "exp20",
                           k=100, l=110, v=3, storage="f32",
                           noise=1e-6 / math.sqrt(8192))
MIXED_32768 = Workload("mixed_32768_k256_l276_v3", 32768, 32768, "pow15",
                       k=256, l=276, v=3, storage="f32")
# the mixed-precision recipe at a quarter of the size (A is 1.07 GB, still
# larger than L2): the case the kernel profiles are captured on
MIXED_16384 = Workload("mixed_16384_k256_l276_v3", 16384, 16384, "pow15",
                       k=256, l=276, v=3, storage="f32")
FIXED_PREC_20000x10000 = Workload("fixed_prec_20000x10000_eps1e-3_b32_l512_v4",
                                  20000, 10000, "gap400", l=512, v=4,
                                  storage="f32", eps=1e-3, b=32)


def batched_problems(count=512, seed=0):
    """Problem sizes of the batched workload: m log-uniform in [256, 4096],
    n log-uniform in [128, m], k uniform in [8, 64], l = k + 10, v in {2, 3}
    half and half, sigma_i = exp(-i/k)."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        m = int(round(math.exp(rng.uniform(math.log(256), math.log(4096)))))
        n = int(round(math.exp(rng.uniform(math.log(128), math.log(m)))))
        k = int(rng.integers(8, 65))
        l = k + 10
        if l >= min(m, n):
            l = min(m, n) - 1
            k = min(k, l)
        v = 2 if i % 2 == 0 else 3
        probs.append(dict(m=m, n=n, k=k, l=l, v=v, seed=int(seed * 100003 + i)))
    return probs


# --------------------------------------------------------------------------
# sparse matrices (the sparse runtime experiment of Sec. 6: MATLAB sprand)
# --------------------------------------------------------------------------
def sprand_csr(m, n, density, seed):
    """A seeded stand-in for MATLAB's sprand(m, n, density): about
    density * m * n nonzeros at uniformly random positions, values uniform on
    [0, 1).  Positions are drawn with replacement and repeats dropped, so
    each (i, j) appears once and nnz is slightly below round(density m n).
    Returns the CSR of A: (row_ptr int64 (m + 1), col_idx int32, val float64),
    columns sorted within each row."""
    rng = np.random.default_rng(seed)
    want = int(round(density * m * n))
    lin = np.unique(rng.integers(0, m * n, size=want, dtype=np.int64))
    rows = lin // n
    cols = (lin - rows * n).astype(np.int32)
    val = rng.random(lin.size)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return row_ptr, cols, val


def csr_transpose(m, n, row_ptr, col_idx, val):
    """The CSR of A^T (n x m) from the CSR of A (m x n): a stable reordering
    of the same entries by column.  Returns (t_row_ptr, t_col_idx, t_val)."""
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    order = np.argsort(col_idx, kind="stable")
    t_row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(col_idx, minlength=n), out=t_row_ptr[1:])
    return t_row_ptr, rows[order].astype(np.int32), val[order]


def csr_to_dense(m, n, row_ptr, col_idx, val):
    """The dense m x n A (Fortran order) of a CSR whose positions are unique."""
    A = np.zeros((m, n), order="F")
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    A[rows, col_idx] = val
    return A


def dense_to_csr(A):
    """CSR of the nonzeros of a dense array, row by row (format conversion)."""
    m, n = A.shape
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), np.asarray(A)[rows, cols].astype(np.float64)


def sparse_rank_r(m, n, r, seed, frac=0.15):
    """A dense array holding a sparse matrix of exact rank r: the sum of r
    outer products of Gaussian vectors whose entries are kept with
    probability frac."""
    rng = np.random.default_rng(seed)
    A = np.zeros((m, n), order="F")
    for _ in range(r):
        u = rng.standard_normal(m) * (rng.random(m) < frac)
        v = rng.standard_normal(n) * (rng.random(n) < frac)
        A += np.outer(u, v)
    return A
