"""ctypes binding of libpowerlu.so (include/powerlu.h), argument marshalling only.

The C entry points are exposed under their own names (``lib().plu_powerlu``
...).  The wrappers below take torch CUDA tensors (column-major views: shape
(rows, cols), stride (1, ld)), pass their device pointers and the current
torch stream to the library, and turn non-OK statuses into exceptions.
Every step of the computation runs in the library's kernels; there is no
other code path: if the library is not built, importing raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpowerlu.so")

PLU_FP64, PLU_TF32, PLU_BF16, PLU_FP8_E4M3, PLU_FP32, PLU_TF32X3 = 0, 1, 2, 3, 4, 5
PLU_F64, PLU_F32 = 0, 1
STATUS = {0: "PLU_OK", 1: "PLU_EINVAL", 2: "PLU_ENOMEM", 3: "PLU_ECUDA", 4: "PLU_ENUMERIC",
          5: "PLU_ETIMEOUT", 6: "PLU_TOL_NOT_MET", 7: "PLU_EUNSUPPORTED", 8: "PLU_EINDEX"}
PREC = {"fp64": PLU_FP64, "tf32": PLU_TF32, "bf16": PLU_BF16, "fp8": PLU_FP8_E4M3,
        "fp32": PLU_FP32, "tf32x3": PLU_TF32X3}

STREAM_OMEGA_N, STREAM_OMEGA_M, STREAM_OMEGA_SP = 1, 2, 3

c_i64, c_i32, c_u64, c_u32, c_int, c_dbl, c_vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                                  ctypes.c_uint32, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_void_p)


class plu_matrix(ctypes.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("ld", c_i64), ("dtype", c_i32), ("data", c_vp)]


class plu_csr(ctypes.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("nnz", c_i64), ("row_ptr", c_vp), ("col_idx", c_vp),
                ("val", c_vp), ("t_row_ptr", c_vp), ("t_col_idx", c_vp), ("t_val", c_vp)]


class plu_report(ctypes.Structure):
    _fields_ = [("ms_total", c_dbl), ("ms_passes", c_dbl), ("passes", c_i32), ("rank", c_i32),
                ("indicator", c_dbl), ("normA2", c_dbl), ("info1", c_i32), ("info2", c_i32),
                ("flops_passes", c_dbl), ("bytes_passes", c_dbl), ("launches", c_i32),
                ("rounds", c_i32), ("ms_phase", c_dbl * 8)]

    PHASES = ("sketch", "power_passes", "reorth", "qr", "last_pass", "rank", "tail_lu",
              "tail_products")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_phase"}
        d["ms_phase"] = {nm: float(self.ms_phase[i]) for i, nm in enumerate(self.PHASES)}
        return d


class plu_batch_problem(ctypes.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("ld", c_i64), ("dtype", c_i32), ("A", c_vp),
                ("k", c_i32), ("l", c_i32), ("v", c_i32), ("algo", c_i32), ("seed", c_u64),
                ("p", c_vp), ("q", c_vp), ("L", c_vp), ("ldL", c_i64), ("U", c_vp), ("ldU", c_i64)]


# C signatures: name -> (restype, argtypes)
SIGNATURES = {
    "plu_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_vp]),
    "plu_destroy": (None, [c_vp]),
    "plu_last_error": (ctypes.c_char_p, [c_vp]),
    "plu_set_stream": (c_int, [c_vp, c_vp]),
    "plu_set_async": (c_int, [c_vp, c_int]),
    "plu_check": (c_int, [c_vp]),
    "plu_set_wait_budget": (c_int, [c_vp, c_i64]),
    "plu_set_lu_updates": (c_int, [c_vp, c_int]),
    "plu_gaussian": (c_int, [c_vp, c_i64, c_i64, c_u64, c_u32, c_vp, c_i64]),
    "plu_pass": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_int, c_vp, c_i64, c_int, c_int,
                         c_vp, c_i64]),
    "plu_lu_reorth": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64]),
    "plu_getrf": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "plu_qr": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_i64]),
    "plu_cholqr1": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_i64, c_int]),
    "plu_rank": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64, c_dbl, c_dbl, c_int, c_int,
                         ctypes.POINTER(c_int), ctypes.POINTER(c_dbl)]),
    "plu_norm2": (c_int, [c_vp, ctypes.POINTER(plu_matrix), ctypes.POINTER(c_dbl)]),
    "plu_powerlu": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_int, c_int, c_int, c_u64, c_int,
                            c_vp, c_vp, c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(plu_report)]),
    "plu_randlu": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_int, c_int, c_int, c_u64, c_int,
                           c_vp, c_vp, c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(plu_report)]),
    "plu_powerlu_fp": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_dbl, c_int, c_int, c_int, c_int,
                               c_u64, c_int, ctypes.POINTER(c_int), c_vp, c_vp, c_vp, c_i64, c_vp,
                               c_i64, ctypes.POINTER(plu_report)]),
    "plu_powerlu_fp_restart": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_dbl, c_int, c_int, c_int,
                                       c_int, c_int, c_u64, c_int, ctypes.POINTER(c_int), c_vp,
                                       c_vp, c_vp, c_i64, c_vp, c_i64,
                                       ctypes.POINTER(plu_report)]),
    "plu_singlepass": (c_int, [c_vp, ctypes.POINTER(plu_matrix), c_int, c_u64, c_int, c_vp, c_vp,
                               c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(plu_report)]),
    "plu_spmm": (c_int, [c_vp, ctypes.POINTER(plu_csr), c_int, c_vp, c_i64, c_int, c_vp, c_i64]),
    "plu_powerlu_csr": (c_int, [c_vp, ctypes.POINTER(plu_csr), c_int, c_int, c_int, c_u64, c_vp,
                                c_vp, c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(plu_report)]),
    "plu_powerlu_fp_csr": (c_int, [c_vp, ctypes.POINTER(plu_csr), c_dbl, c_int, c_int, c_int,
                                   c_int, c_int, c_u64, ctypes.POINTER(c_int), c_vp, c_vp, c_vp,
                                   c_i64, c_vp, c_i64, ctypes.POINTER(plu_report)]),
    "plu_lu_reorth_static": (c_int, [c_vp, c_i64, c_int, c_vp, c_i64, ctypes.c_char_p,
                                     ctypes.c_size_t]),
    "plu_set_batched_tile": (c_int, [c_vp, c_int, c_int]),
    "plu_batched_tiles": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int,
                                  ctypes.POINTER(c_int)]),
    "plu_batched_splitk": (c_int, [c_vp, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int)]),
    "plu_set_batched_tune_file": (c_int, [c_vp, ctypes.c_char_p]),
    "plu_batched": (c_int, [c_vp, ctypes.POINTER(plu_batch_problem), c_int, c_int,
                            ctypes.POINTER(plu_report)]),
}

_lib = None


def lib():
    """The loaded library (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpowerlu.so is not built (run __graft_entry__.build()); "
                              "there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PLUError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__("%s: %s" % (self.name, msg))


# ----------------------------------------------------------------- helpers
def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ld(t):
    """Leading dimension of a column-major 2-D tensor view."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError("expected a column-major tensor (stride(0) == 1)")
    return max(t.stride(1), t.shape[0], 1)


def colmajor_empty(rows, cols, dtype=None, device="cuda"):
    torch = _torch()
    dtype = dtype or torch.float64
    return torch.empty(cols, rows, dtype=dtype, device=device).t()


def as_plu_matrix(A):
    torch = _torch()
    dt = {torch.float64: PLU_F64, torch.float32: PLU_F32}.get(A.dtype)
    if dt is None:
        raise ValueError("A must be float32 or float64")
    return plu_matrix(A.shape[0], A.shape[1], _ld(A), dt, A.data_ptr())


class Context:
    """plu_ctx bound to a device and (by default) torch's current stream."""

    def __init__(self, device=0, stream=None):
        torch = _torch()
        self._h = c_vp()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        st = lib().plu_create(ctypes.byref(self._h), int(device), c_vp(stream))
        if st != 0:
            raise PLUError(st, "plu_create failed")
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().plu_destroy(self._h)
            self._h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st, allow=()):
        if st != 0 and st not in allow:
            raise PLUError(st, lib().plu_last_error(self._h).decode())
        return st

    def set_stream(self, stream):
        return self.check(lib().plu_set_stream(self._h, c_vp(stream)))

    def set_wait_budget(self, spins):
        return self.check(lib().plu_set_wait_budget(self._h, int(spins)))

    def set_lu_updates(self, mode):
        """-1: default, 0: FP64 FMAs, 1: tensor-core digit products."""
        return self.check(lib().plu_set_lu_updates(self._h, int(mode)))


# ------------------------------------------------------------ entry points
def plu_gaussian(ctx, rows, cols, seed, stream_id, out=None):
    out = out if out is not None else colmajor_empty(rows, cols)
    ctx.check(lib().plu_gaussian(ctx.handle, rows, cols, seed, stream_id, _ptr(out), _ld(out)))
    return out


def plu_pass(ctx, A, trans, X, prec="fp64", out=None):
    M = A.shape[1] if trans else A.shape[0]
    cols = X.shape[1]
    out = out if out is not None else colmajor_empty(M, cols)
    Am = as_plu_matrix(A)
    ctx.check(lib().plu_pass(ctx.handle, ctypes.byref(Am), int(trans), _ptr(X), _ld(X), cols,
                             PREC[prec], _ptr(out), _ld(out)))
    return out


def plu_lu_reorth(ctx, X):
    ctx.check(lib().plu_lu_reorth(ctx.handle, X.shape[0], X.shape[1], _ptr(X), _ld(X)))
    return X


def plu_getrf(ctx, X):
    """[L, U, P] = lu(X); X is destroyed.  Returns (perm, L, U, info)."""
    torch = _torch()
    rows, cols = X.shape
    perm = torch.empty(rows, dtype=torch.int32, device=X.device)
    L = colmajor_empty(rows, cols, device=X.device)
    U = colmajor_empty(cols, cols, device=X.device)
    info = torch.zeros(1, dtype=torch.int32, device=X.device)
    ctx.check(lib().plu_getrf(ctx.handle, rows, cols, _ptr(X), _ld(X), _ptr(perm), _ptr(L),
                              _ld(L), _ptr(U), _ld(U), _ptr(info)))
    return perm, L, U, int(info.item())


def plu_qr(ctx, X, want_r=False):
    R = colmajor_empty(X.shape[1], X.shape[1], device=X.device) if want_r else None
    ctx.check(lib().plu_qr(ctx.handle, X.shape[0], X.shape[1], _ptr(X), _ld(X), _ptr(R),
                           _ld(R) if R is not None else 0))
    return (X, R) if want_r else X


def plu_set_batched_tile(ctx, bm=0, bn=0):
    """Fix the batched GEMM tile shape (bm x bn); (0, 0) restores the autotuner."""
    ctx.check(lib().plu_set_batched_tile(ctx.handle, bm, bn))


def plu_batched_tiles(ctx):
    """Tile shapes (rows, columns) the autotuner chose for the grouped GEMM
    launches of the last plu_batched call, in launch order."""
    n = c_int()
    ctx.check(lib().plu_batched_tiles(ctx.handle, None, None, 0, ctypes.byref(n)))
    bm = (c_int * max(n.value, 1))()
    bn = (c_int * max(n.value, 1))()
    ctx.check(lib().plu_batched_tiles(ctx.handle, bm, bn, n.value, ctypes.byref(n)))
    return [(bm[i], bn[i]) for i in range(n.value)]


def plu_batched_splitk(ctx):
    """K-chunk length of each grouped GEMM launch of the last plu_batched call
    (0: no split-K), in launch order."""
    n = c_int()
    ctx.check(lib().plu_batched_splitk(ctx.handle, None, 0, ctypes.byref(n)))
    kc = (c_int * max(n.value, 1))()
    ctx.check(lib().plu_batched_splitk(ctx.handle, kc, n.value, ctypes.byref(n)))
    return [kc[i] for i in range(n.value)]


def plu_set_batched_tune_file(ctx, path):
    """Persist the batched autotuner's choices in the text file `path`
    (None turns it off)."""
    ctx.check(lib().plu_set_batched_tune_file(
        ctx.handle, None if path is None else str(path).encode()))


def plu_cholqr1(ctx, X, tc=True):
    """One CholeskyQR round in place (X <- X R^-1); tc: FP64-accurate products
    on the BF16 tensor cores.  Returns (X, R)."""
    R = colmajor_empty(X.shape[1], X.shape[1], device=X.device)
    ctx.check(lib().plu_cholqr1(ctx.handle, X.shape[0], X.shape[1], _ptr(X), _ld(X), _ptr(R),
                                _ld(R), int(bool(tc))))
    return X, R


def plu_norm2(ctx, A):
    Am = as_plu_matrix(A)
    out = c_dbl()
    ctx.check(lib().plu_norm2(ctx.handle, ctypes.byref(Am), ctypes.byref(out)))
    return out.value


def plu_rank(ctx, G, normA2, eps, b, precise=False):
    k = c_int()
    E = c_dbl()
    st = ctx.check(lib().plu_rank(ctx.handle, G.shape[0], G.shape[1], _ptr(G), _ld(G),
                                  float(normA2), float(eps), int(b), int(bool(precise)),
                                  ctypes.byref(k), ctypes.byref(E)), allow=(6,))
    return k.value, E.value, st == 0


def plu_powerlu(ctx, A, k, l, v, seed=0, prec="fp64"):
    """Fixed rank.  Returns (p, q, L, U, report dict)."""
    torch = _torch()
    m, n = A.shape
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, k, device=A.device)
    U = colmajor_empty(k, n, device=A.device)
    rep = plu_report()
    Am = as_plu_matrix(A)
    ctx.check(lib().plu_powerlu(ctx.handle, ctypes.byref(Am), k, l, v, seed, PREC[prec], _ptr(p),
                                _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U), ctypes.byref(rep)))
    return p, q, L, U, rep.as_dict()


def plu_randlu(ctx, A, k, l, piter, seed=0, prec="fp64"):
    """RandLU with `piter` power iterations (2 piter + 2 passes over A).
    Returns (p, q, L, U, report dict) as plu_powerlu."""
    torch = _torch()
    m, n = A.shape
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, k, device=A.device)
    U = colmajor_empty(k, n, device=A.device)
    rep = plu_report()
    Am = as_plu_matrix(A)
    ctx.check(lib().plu_randlu(ctx.handle, ctypes.byref(Am), k, l, piter, seed, PREC[prec],
                               _ptr(p), _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U),
                               ctypes.byref(rep)))
    return p, q, L, U, rep.as_dict()


def plu_powerlu_fp(ctx, A, eps, b, l, v, seed=0, prec="fp64", precise=False, max_rounds=1):
    """Fixed precision (max_rounds > 1: with the restart on the remainder,
    plu_powerlu_fp_restart).  Returns (k, p, q, L[:, :k], U[:k], met, report dict)."""
    torch = _torch()
    m, n = A.shape
    K = l * max_rounds
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, K, device=A.device)
    U = colmajor_empty(K, n, device=A.device)
    rep = plu_report()
    k = c_int()
    Am = as_plu_matrix(A)
    if max_rounds == 1:
        st = ctx.check(lib().plu_powerlu_fp(ctx.handle, ctypes.byref(Am), float(eps), b, l, v,
                                            int(bool(precise)), seed, PREC[prec], ctypes.byref(k),
                                            _ptr(p), _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U),
                                            ctypes.byref(rep)), allow=(6,))
    else:
        st = ctx.check(lib().plu_powerlu_fp_restart(
            ctx.handle, ctypes.byref(Am), float(eps), b, l, v, int(bool(precise)), max_rounds,
            seed, PREC[prec], ctypes.byref(k), _ptr(p), _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U),
            ctypes.byref(rep)), allow=(6,))
    kk = k.value
    return kk, p, q, L[:, :kk], U[:kk, :], st == 0, rep.as_dict()


def plu_singlepass(ctx, A, k, seed=0, prec="fp64"):
    """Single pass (Alg. singlepasslu).  Returns (p, q, L, U, report dict)."""
    torch = _torch()
    m, n = A.shape
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, k, device=A.device)
    U = colmajor_empty(k, n, device=A.device)
    rep = plu_report()
    Am = as_plu_matrix(A)
    ctx.check(lib().plu_singlepass(ctx.handle, ctypes.byref(Am), k, seed, PREC[prec], _ptr(p),
                                   _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U), ctypes.byref(rep)))
    return p, q, L, U, rep.as_dict()


def plu_batched(ctx, problems, prec="fp32"):
    """Batched factorisation.  `problems`: list of dicts with A (column-major
    CUDA tensor), k, l, v, algo (0 PowerLU, 1 single pass), seed.  Returns
    (list of (p, q, L, U), report dict)."""
    torch = _torch()
    arr = (plu_batch_problem * len(problems))()
    outs = []
    for i, pr in enumerate(problems):
        A = pr["A"]
        m, n = A.shape
        k = pr["k"]
        p = torch.empty(m, dtype=torch.int32, device=A.device)
        q = torch.empty(n, dtype=torch.int32, device=A.device)
        L = colmajor_empty(m, k, device=A.device)
        U = colmajor_empty(k, n, device=A.device)
        Am = as_plu_matrix(A)
        arr[i] = plu_batch_problem(m, n, Am.ld, Am.dtype, A.data_ptr(), k, pr.get("l", k),
                                   pr.get("v", 2), pr.get("algo", 0), pr.get("seed", 0),
                                   p.data_ptr(), q.data_ptr(), L.data_ptr(), _ld(L), U.data_ptr(),
                                   _ld(U))
        outs.append((p, q, L, U))
    rep = plu_report()
    ctx.check(lib().plu_batched(ctx.handle, arr, len(problems), PREC[prec], ctypes.byref(rep)))
    return outs, rep.as_dict()


# ------------------------------------------------------------- sparse A
class CsrMatrix:
    """A sparse m x n A on the device as plu_csr wants it: the CSR of A and
    the CSR of A^T (int64 row pointers, int32 column indices, float64
    values, all CUDA tensors).  Holds the tensors so they outlive the calls."""

    def __init__(self, m, n, row_ptr, col_idx, val, t_row_ptr, t_col_idx, t_val):
        torch = _torch()
        want = ((row_ptr, torch.int64, m + 1), (col_idx, torch.int32, None),
                (val, torch.float64, None), (t_row_ptr, torch.int64, n + 1),
                (t_col_idx, torch.int32, None), (t_val, torch.float64, None))
        for t, dt, size in want:
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.dim() != 1:
                raise ValueError("CSR arrays must be contiguous 1-D CUDA tensors "
                                 "(int64 row pointers, int32 indices, float64 values)")
            if size is not None and t.numel() != size:
                raise ValueError("row pointer arrays need m + 1 and n + 1 entries")
        nnz = val.numel()
        if col_idx.numel() != nnz or t_col_idx.numel() != nnz or t_val.numel() != nnz:
            raise ValueError("A and A^T must have the same number of nonzeros")
        self.m, self.n, self.nnz = int(m), int(n), int(nnz)
        self.shape = (self.m, self.n)
        self.device = val.device
        self.tensors = (row_ptr, col_idx, val, t_row_ptr, t_col_idx, t_val)
        self.struct = plu_csr(self.m, self.n, self.nnz, *(t.data_ptr() for t in self.tensors))


def plu_spmm(ctx, A, trans, X, out=None):
    """Y = A X (trans 0) or A^T X (trans 1) for a CsrMatrix A, FP64."""
    M = A.n if trans else A.m
    cols = X.shape[1]
    out = out if out is not None else colmajor_empty(M, cols, device=X.device)
    ctx.check(lib().plu_spmm(ctx.handle, ctypes.byref(A.struct), int(trans), _ptr(X), _ld(X), cols,
                             _ptr(out), _ld(out)))
    return out


def plu_powerlu_csr(ctx, A, k, l, v, seed=0):
    """Fixed rank on a CsrMatrix A (FP64 sparse passes).  Returns
    (p, q, L, U, report dict) as plu_powerlu."""
    torch = _torch()
    m, n = A.shape
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, k, device=A.device)
    U = colmajor_empty(k, n, device=A.device)
    rep = plu_report()
    ctx.check(lib().plu_powerlu_csr(ctx.handle, ctypes.byref(A.struct), k, l, v, seed, _ptr(p),
                                    _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U), ctypes.byref(rep)))
    return p, q, L, U, rep.as_dict()


def plu_powerlu_fp_csr(ctx, A, eps, b, l, v, seed=0, precise=False, max_rounds=1):
    """Fixed precision on a CsrMatrix A.  Returns
    (k, p, q, L[:, :k], U[:k], met, report dict) as plu_powerlu_fp."""
    torch = _torch()
    m, n = A.shape
    K = l * max_rounds
    p = torch.empty(m, dtype=torch.int32, device=A.device)
    q = torch.empty(n, dtype=torch.int32, device=A.device)
    L = colmajor_empty(m, K, device=A.device)
    U = colmajor_empty(K, n, device=A.device)
    rep = plu_report()
    k = c_int()
    st = ctx.check(lib().plu_powerlu_fp_csr(
        ctx.handle, ctypes.byref(A.struct), float(eps), b, l, v, int(bool(precise)), max_rounds,
        seed, ctypes.byref(k), _ptr(p), _ptr(q), _ptr(L), _ld(L), _ptr(U), _ld(U),
        ctypes.byref(rep)), allow=(6,))
    kk = k.value
    return kk, p, q, L[:, :kk], U[:kk, :], st == 0, rep.as_dict()
