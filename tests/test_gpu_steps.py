"""GPU parity of each step of the hot path against the FP64 oracle, through
the C ABI (libpowerlu.so).  Sizes span several 64-row tiles and ragged
tails; FP64 steps are compared at ~1e-12 relative, integer outputs
(permutations) bit for bit, the Gaussian sketch bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2002_07138_gb300 as plu

pytestmark = pytest.mark.gpu


def dev(X, dtype=torch.float64):
    """Column-major CUDA copy of a numpy matrix."""
    X = np.asarray(X)
    out = plu.colmajor_empty(X.shape[0], X.shape[1], dtype=dtype)
    out.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return out


def host(T):
    return T.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------- a1
@pytest.mark.parametrize("rows,cols,seed,sid", [(2000, 25, 0, 1), (1500, 25, 0, 2), (7, 5, 3, 2),
                                                 (1001, 33, (1 << 40) + 5, 3), (1, 1, 9, 1)])
def test_gaussian_bit_identical(ctx, rows, cols, seed, sid):
    ref = oracle.gaussian_matrix(rows, cols, seed, sid)
    got = plu.plu_gaussian(ctx, rows, cols, seed, sid)
    assert np.array_equal(host(got), ref)


@pytest.mark.parametrize("rows", [33, 34])     # one entry per thread / one pair per thread
def test_gaussian_with_leading_dimension(ctx, rows):
    buf = plu.colmajor_empty(40, 6)
    buf.fill_(7.0)
    view = buf[:rows, :]
    plu.plu_gaussian(ctx, rows, 6, 11, 1, out=view)
    assert np.array_equal(host(buf[:rows]), oracle.gaussian_matrix(rows, 6, 11, 1))
    assert torch.all(buf[rows:] == 7.0)


# --------------------------------------------------------------- a2/a4/a6
@pytest.mark.parametrize("m,n,cols", [(1000, 777, 25), (333, 1201, 70), (64, 64, 64), (2000, 1500, 1)])
@pytest.mark.parametrize("trans", [0, 1])
def test_pass_fp64(ctx, m, n, cols, trans):
    A = synth.gaussian_np(m, n, 1)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 2)
    ref = A @ X if trans == 0 else A.T @ X
    got = host(plu.plu_pass(ctx, dev(A), trans, dev(X), "fp64"))
    assert rel(got, ref) < 1e-13


@pytest.mark.parametrize("trans", [0, 1])
def test_pass_fp64_with_f32_matrix_and_ld(ctx, trans):
    m, n, cols = 517, 300, 19
    big = plu.colmajor_empty(600, n, dtype=torch.float32)
    big.copy_(torch.from_numpy(synth.gaussian_np(600, n, 3).astype(np.float32)))
    A = big[:m, :]
    X = synth.gaussian_np(n if trans == 0 else m, cols, 4)
    A64 = host(A)
    ref = A64 @ X if trans == 0 else A64.T @ X
    got = host(plu.plu_pass(ctx, A, trans, dev(X), "fp64"))
    assert rel(got, ref) < 1e-13


@pytest.mark.parametrize("trans", [0, 1])
def test_pass_fp32(ctx, trans):
    m, n, cols = 1500, 1100, 40
    A32 = synth.gaussian_np(m, n, 5).astype(np.float32)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 6)
    Xr = X.astype(np.float32).astype(np.float64)
    A64 = A32.astype(np.float64)
    ref = A64 @ Xr if trans == 0 else A64.T @ Xr
    got = host(plu.plu_pass(ctx, dev(A32, torch.float32), trans, dev(X), "fp32"))
    assert rel(got, ref) < 2e-6


# ------------------------------------------------------------------- a3
@pytest.mark.parametrize("rows,cols", [(2000, 25), (1500, 110), (777, 64), (300, 300), (65, 3)])
def test_lu_reorth(ctx, rows, cols):
    X = synth.gaussian_np(rows, cols, rows + cols)
    ref = oracle.lu_permuted_L(X)
    got = host(plu.plu_lu_reorth(ctx, dev(X)))
    assert rel(got, ref) < 1e-12


# ------------------------------------------------------------------- a8
@pytest.mark.parametrize("rows,cols", [(2000, 20), (1500, 100), (513, 64), (64, 64), (10000, 7)])
def test_getrf(ctx, rows, cols):
    X = synth.gaussian_np(rows, cols, 7 * rows + cols)
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(ctx, dev(X))
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < 1e-12
    assert rel(host(gU), U) < 1e-12
    assert ginfo == info == 0


def test_getrf_tie_rule_matches_lapack_order(ctx):
    """Exact-arithmetic integer panels with tied pivot magnitudes: the GPU's
    virtual pivoting must pick the same rows as the oracle's row swaps."""
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 20:
        X = rng.integers(-1, 2, size=(12, 5)).astype(np.float64)
        X[:, 0] = rng.choice([-2.0, 2.0], size=12)          # every row ties in column 0
        perm, L, U, info = oracle.getrf(X)
        # keep panels whose elimination is exact (dyadic pivots only)
        piv = np.abs(np.diag(U))
        if not np.all((piv == 0) | (np.log2(np.where(piv == 0, 1, piv)) % 1 == 0)):
            continue
        if not np.array_equal(X[perm], L @ U):
            continue
        gp, gL, gU, ginfo = plu.plu_getrf(ctx, dev(X))
        assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
        assert np.array_equal(host(gL), L) and np.array_equal(host(gU), U)
        assert ginfo == info
        checked += 1


def test_getrf_zero_column(ctx):
    X = synth.gaussian_np(300, 8, 1)
    X[:, 3] = 0.0
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(ctx, dev(X))
    assert info == 4 and ginfo == 4
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < 1e-12 and rel(host(gU), U) < 1e-12


# ------------------------------------------------------------------- a5
@pytest.mark.parametrize("rows,cols", [(1500, 25), (8192, 110), (700, 64), (333, 333)])
def test_qr(ctx, rows, cols):
    X = synth.gaussian_np(rows, cols, rows) * np.logspace(0, -3, cols)[None, :]
    Q, R = oracle.qr_economy(X)
    gQ, gR = plu.plu_qr(ctx, dev(X), want_r=True)
    gQ, gR = host(gQ), host(gR)
    assert np.max(np.abs(gQ.T @ gQ - np.eye(cols))) < 1e-13
    assert rel(gQ, Q) < 1e-11
    assert rel(gR, R) < 1e-11


# ------------------------------------------------------------------- a7
@pytest.mark.parametrize("precise", [False, True])
def test_rank_scan(ctx, precise):
    sig = synth.sigma_profile("type2", 400)
    A = synth.svd_matrix_np(500, 400, sig, seed=6)
    V = oracle.gpowerlu(A, 200, 4, seed=1)
    G = A @ V
    nA2 = float(np.sum(A * A))
    for eps in (1e-2, 1e-4, 1e-6):
        k, E, met = oracle.rank_scan(G, nA2, eps, 10, precise)
        gk, gE, gmet = plu.plu_rank(ctx, dev(G), nA2, eps, 10, precise)
        assert (gk, gmet) == (k, met)
        assert abs(gE - E) <= 1e-12 * nA2


def test_norm2(ctx):
    A = synth.gaussian_np(1234, 567, 8)
    assert abs(plu.plu_norm2(ctx, dev(A)) - float(np.sum(A * A))) <= 1e-12 * np.sum(A * A)
    A32 = A.astype(np.float32)
    ref = float(np.sum(A32.astype(np.float64) ** 2))
    assert abs(plu.plu_norm2(ctx, dev(A32, torch.float32)) - ref) <= 1e-12 * ref


# --------------------------------------------------- failure detection
def test_barrier_timeout_is_reported_and_context_survives(ctx):
    """A one-spin wait budget makes the grid barriers of the panel LU give up:
    the call returns PLU_ETIMEOUT and the next call on the context works."""
    X = dev(synth.gaussian_np(20000, 16, 3))
    ctx.set_wait_budget(1)
    try:
        with pytest.raises(plu.PLUError) as ei:
            plu.plu_lu_reorth(ctx, X)
        assert ei.value.name == "PLU_ETIMEOUT"
    finally:
        ctx.set_wait_budget(-1)
    Y = synth.gaussian_np(2000, 16, 4)
    assert rel(host(plu.plu_lu_reorth(ctx, dev(Y))), oracle.lu_permuted_L(Y)) < 1e-12


def test_invalid_arguments_launch_nothing(ctx):
    A = dev(synth.gaussian_np(50, 40, 1))
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_powerlu(ctx, A, 10, 9, 2)            # l < k
    assert ei.value.name == "PLU_EINVAL"
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_powerlu(ctx, A, 5, 10, 1)            # v < 2
    assert ei.value.name == "PLU_EINVAL"
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_powerlu(ctx, A, 5, 40, 2)            # l >= min(m, n)
    assert ei.value.name == "PLU_EINVAL"


def _fp64_values_for_rounding(rng, n):
    """FP64 values whose FP32 rounding exercises every case: random
    magnitudes over the normal FP32 range, exact ties between neighbouring
    floats and values one double ulp either side, the binade edges, values
    that round up into the next binade, near the largest float (below the
    halfway point to infinity), around the smallest normal, subnormal
    results and zeros."""
    f = (rng.standard_normal(n) * np.exp2(rng.integers(-120, 120, size=n))).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf), dtype=np.float32)
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2.0          # exact ties
    up = np.nextafter(mid, np.inf)
    dn = np.nextafter(mid, -np.inf)
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edges = np.array([1.0, -1.0, 2.0 - 2.0 ** -30, 1.0 + 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52,
                      fmax, fmax * (1 + 2.0 ** -25) - 2.0 ** 100, -fmax, tiny, tiny * (1 - 2.0 ** -30),
                      tiny * (1 + 2.0 ** -30), tiny / 3.0, -tiny / 7.0, 2.0 ** -150, 2.0 ** -149,
                      0.0, -0.0, 3.0e-42, 1e-300])
    v = np.concatenate([f.astype(np.float64), mid, up, dn, -mid, edges])
    return v[np.isfinite(v.astype(np.float32))]


@pytest.mark.parametrize("trans", [0, 1])
def test_fp32_pass_rounds_fp64_operands_to_nearest(ctx, trans):
    """FP32 passes round FP64 operands to FP32 as IEEE round-to-nearest-even
    does (the library forms the rounding on the integer pipe): with X's
    columns unit vectors, Y holds the rounded entries of A bit for bit."""
    rng = np.random.default_rng(17)
    vals = _fp64_values_for_rounding(rng, 4000)
    m, n = 384, 96
    A = np.resize(vals, m * n).reshape(n, m).T.copy()
    A[:, 0] = np.resize(vals[::-1], m)
    js = [0, 1, 5, 47, 95] if trans == 0 else [0, 3, 200, 383]
    K = n if trans == 0 else m
    X = np.zeros((K, len(js)))
    for c, j in enumerate(js):
        X[j, c] = 1.0
    got = host(plu.plu_pass(ctx, dev(A), trans, dev(X), "fp32"))
    sel = A[:, js] if trans == 0 else A[js, :].T
    # + 0.0: the product adds the one nonzero term to a +0 accumulator, so a
    # rounded -0 comes out as +0
    want = sel.astype(np.float32).astype(np.float64) + 0.0
    bad = np.flatnonzero(got.view(np.int64) != want.view(np.int64))
    assert bad.size == 0, (sel.ravel()[bad[:5]], got.ravel()[bad[:5]], want.ravel()[bad[:5]])


# ------------------------------------------- a2/a4/a6 on tensor cores (TF32)
def tf32_trunc(a):
    """float32 -> TF32 by dropping the 13 low mantissa bits (what the MMA reads)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def tf32_rna(a):
    """float32 -> TF32, round to nearest, ties away from zero."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


@pytest.mark.parametrize("m,n,cols", [(1000, 777, 25), (2048, 1536, 276), (300, 257, 1),
                                      (512, 8192, 110), (4096, 1024, 512), (132, 4100, 48)])
@pytest.mark.parametrize("trans", [0, 1])
def test_pass_tf32_matches_tf32_operands(ctx, m, n, cols, trans):
    """The tensor-core pass equals the FP64 product of the TF32 operands the
    MMA consumes (A truncated, X rounded) up to FP32 accumulation error."""
    A32 = synth.gaussian_np(m, n, 11).astype(np.float32)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 12)
    At = tf32_trunc(A32).astype(np.float64)
    Xr = tf32_rna(X.astype(np.float32)).astype(np.float64)
    ref = At @ Xr if trans == 0 else At.T @ Xr
    got = host(plu.plu_pass(ctx, dev(A32, torch.float32), trans, dev(X), "tf32"))
    K = n if trans == 0 else m
    assert rel(got, ref) < 4e-7 * np.sqrt(K / 32.0) + 1e-6


@pytest.mark.parametrize("trans", [0, 1])
def test_pass_tf32_leading_dimension_and_fallback(ctx, trans):
    m, n, cols = 600, 500, 40
    X = synth.gaussian_np(n if trans == 0 else m, cols, 14)
    Xr = tf32_rna(X.astype(np.float32)).astype(np.float64)
    for ld in (604, 601):                    # 601: not a multiple of 4 -> SIMT FP32 kernel
        big = plu.colmajor_empty(ld, n, dtype=torch.float32)
        big.copy_(torch.from_numpy(synth.gaussian_np(ld, n, 13).astype(np.float32)))
        A = big[:m, :]
        A32 = host(A).astype(np.float32)
        got = host(plu.plu_pass(ctx, A, trans, dev(X), "tf32"))
        if ld % 4 == 0:
            At = tf32_trunc(A32).astype(np.float64)
            ref = At @ Xr if trans == 0 else At.T @ Xr
            assert rel(got, ref) < 2e-6
        else:
            A64 = A32.astype(np.float64)
            Xf = X.astype(np.float32).astype(np.float64)
            ref = A64 @ Xf if trans == 0 else A64.T @ Xf
            assert rel(got, ref) < 2e-6


def test_pass_tf32_rejects_fp64_matrix(ctx):
    A = dev(synth.gaussian_np(100, 80, 1))
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_pass(ctx, A, 0, dev(synth.gaussian_np(80, 4, 2)), "tf32")
    assert ei.value.name == "PLU_EUNSUPPORTED"


@pytest.mark.parametrize("rows,cols", [(4096, 512), (2000, 276)])
def test_qr_wide_sketch_cooperative_cholesky(ctx, rows, cols):
    """Sketch widths of the mixed and fixed-precision workloads go through the
    multi-CTA blocked Cholesky."""
    X = synth.gaussian_np(rows, cols, cols) * np.logspace(0, -2, cols)[None, :]
    Q, R = oracle.qr_economy(X)
    gQ, gR = plu.plu_qr(ctx, dev(X), want_r=True)
    gQ, gR = host(gQ), host(gR)
    assert np.max(np.abs(gQ.T @ gQ - np.eye(cols))) < 1e-13
    assert rel(gQ, Q) < 1e-11
    assert rel(gR, R) < 1e-11


@pytest.mark.parametrize("rows,cols", [(32768, 276), (20000, 512)])
def test_lu_reorth_full_size_panels(ctx, rows, cols):
    """Panels of the 32768^2 mixed and 20000 x 10000 fixed-precision workloads."""
    X = synth.gaussian_np(rows, cols, rows + cols)
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(ctx, dev(X))
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < 1e-12
    assert rel(host(gU), U) < 1e-12


# ------------------------------------- a2/a4 on tensor cores (BF16, FP8-E4M3)
def bf16_rne(a):
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def e4m3_rne(x):
    """Round float64 values to FP8-E4M3 (round to nearest even, saturate at 448)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)                       # subnormal spacing 2^-9 below 2^-6
    sp = 2.0 ** (e - 3)
    q = np.round(a / sp) * sp                     # numpy rounds half to even
    return np.sign(x) * np.minimum(q, 448.0)


def fp8_reference(A32, X, trans):
    """The FP8 pass as the library defines it: rank-1 128x128 tile scales
    s_r (rows) and s_c (columns), A/(s_r s_c) and the scaled small operand
    rounded to E4M3, FP32 scales applied in FP64."""
    m, n = A32.shape
    RB, CB = (m + 127) // 128, (n + 127) // 128
    amax = np.zeros((RB, CB), dtype=np.float32)
    for rb in range(RB):
        for cb in range(CB):
            amax[rb, cb] = np.max(np.abs(A32[rb * 128:(rb + 1) * 128, cb * 128:(cb + 1) * 128]))
    s_r = np.max(amax, axis=1).astype(np.float32)
    s_r[s_r == 0] = 1
    s_c = (np.max(amax / s_r[:, None], axis=0) / np.float32(448)).astype(np.float32)
    s_c[s_c == 0] = 1
    rows_s = np.repeat(s_r, 128)[:m]
    cols_s = np.repeat(s_c, 128)[:n]
    Aq = e4m3_rne((A32 / (rows_s[:, None] * cols_s[None, :]).astype(np.float32)).astype(np.float32))
    fold = (cols_s if trans == 0 else rows_s).astype(np.float64)
    outs = (rows_s if trans == 0 else cols_s).astype(np.float64)
    Z = X * fold[:, None]
    cs = (np.max(np.abs(Z), axis=0) / 448.0).astype(np.float32).astype(np.float64)
    cs[cs == 0] = 1
    Zq = e4m3_rne((Z / cs[None, :]).astype(np.float32).astype(np.float64))
    Y = (Aq @ Zq if trans == 0 else Aq.T @ Zq) * outs[:, None] * cs[None, :]
    return Y


@pytest.mark.parametrize("m,n,cols", [(1000, 777, 25), (2048, 1536, 276), (300, 4100, 48)])
@pytest.mark.parametrize("trans", [0, 1])
def test_pass_bf16_matches_bf16_operands(ctx, m, n, cols, trans):
    A32 = synth.gaussian_np(m, n, 21).astype(np.float32)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 22)
    Ab = bf16_rne(A32).astype(np.float64)
    Xb = bf16_rne(X.astype(np.float32)).astype(np.float64)
    ref = Ab @ Xb if trans == 0 else Ab.T @ Xb
    got = host(plu.plu_pass(ctx, dev(A32, torch.float32), trans, dev(X), "bf16"))
    assert rel(got, ref) < 2e-6


@pytest.mark.parametrize("m,n,cols", [(1000, 777, 25), (2048, 1536, 276), (300, 4100, 48)])
@pytest.mark.parametrize("trans", [0, 1])
def test_pass_fp8_matches_fp8_operands(ctx, m, n, cols, trans):
    rng = np.random.default_rng(23)
    A32 = (synth.gaussian_np(m, n, 23) * rng.uniform(0.1, 10.0, size=(1, n))).astype(np.float32)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 24)
    ref = fp8_reference(A32, X, trans)
    got = host(plu.plu_pass(ctx, dev(A32, torch.float32), trans, dev(X), "fp8"))
    assert rel(got, ref) < 2e-5
    exact = A32.astype(np.float64) @ X if trans == 0 else A32.astype(np.float64).T @ X
    assert rel(got, exact) < 0.1


def _cholqr1(ctx, X, tc):
    Xd = plu.colmajor_empty(X.shape[0], X.shape[1])
    Xd.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    Q, R = plu.plu_cholqr1(ctx, Xd, tc=tc)
    return Q.cpu().numpy(), R.cpu().numpy()


@pytest.mark.parametrize("rows,cols", [(4096, 200), (3000, 256), (1000, 37), (6000, 512)])
def test_cholqr1_tensor_core_products_match_fp64(ctx, rows, cols):
    """One CholeskyQR round with X^T X and X R^-1 as exact slice products on
    the BF16 tensor cores: the same R and Q as the FP64 round to ~1e-14
    (well-conditioned X), and R^T R = X^T X to FP64 accuracy."""
    X = np.random.default_rng(rows + cols).standard_normal((rows, cols))
    Qt, Rt = _cholqr1(ctx, X, True)
    Qf, Rf = _cholqr1(ctx, X, False)
    assert np.linalg.norm(Rt - Rf) <= 1e-13 * np.linalg.norm(Rf)
    assert np.linalg.norm(Qt - Qf) <= 1e-13 * np.linalg.norm(Qf)
    G = X.T @ X
    assert np.linalg.norm(np.triu(Rt).T @ np.triu(Rt) - G) <= 1e-14 * np.linalg.norm(G)


def test_cholqr1_tensor_core_products_row_and_column_scales(ctx):
    """Rows spanning 2^-8 .. 2^8 and columns 10^-1 .. 10^1: per-row slices of
    X and per-column slices of R^-1 keep every row of Q = X R^-1 as accurate,
    relative to that row, as the FP64 round (Q R reproduces X row by row), and
    the Gram matrix to FP64 accuracy."""
    rng = np.random.default_rng(7)
    rows, cols = 5000, 120
    X = rng.standard_normal((rows, cols))
    X *= np.exp2(rng.integers(-8, 9, size=rows))[:, None]
    X *= 10.0 ** rng.uniform(-1, 1, size=cols)[None, :]
    Qt, Rt = _cholqr1(ctx, X, True)
    Qf, Rf = _cholqr1(ctx, X, False)
    Rt = np.triu(Rt)
    G = X.T @ X
    assert np.linalg.norm(Rt.T @ Rt - G) <= 1e-13 * np.linalg.norm(G)
    resid_t = np.linalg.norm(Qt @ Rt - X, axis=1) / np.linalg.norm(X, axis=1)
    resid_f = np.linalg.norm(Qf @ np.triu(Rf) - X, axis=1) / np.linalg.norm(X, axis=1)
    assert resid_t.max() <= 10 * resid_f.max() + 1e-13


def test_cholqr1_tensor_core_rejects_wide_x(ctx):
    X = plu.colmajor_empty(2000, 600)
    X.normal_()
    with pytest.raises(plu.PLUError):
        plu.plu_cholqr1(ctx, X, tc=True)


@pytest.mark.parametrize("tc", [True, False])
def test_cholqr1_reports_non_finite_input(ctx, tc):
    """A NaN in X reaches the Cholesky through either form of the products
    (the tensor-core slices of a non-finite line are NaN) and is reported."""
    X = np.random.default_rng(9).standard_normal((2000, 64))
    X[123, 7] = np.nan
    with pytest.raises(plu.PLUError):
        _cholqr1(ctx, X, tc)
