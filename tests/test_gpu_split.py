"""GPU parity of the split-precision tensor-core pass (PLU_TF32X3): Y = op(A) X
over an FP32 A with FP32-accurate products, the pass the mixed modes take
for the products that enter the result to first order (the last pass of
Alg. bpowerlu, RandLU's B pass, the passes of Alg. singlepasslu on request).

Two checks per shape: (1) against the FP64 sum of the three TF32 products the
kernel forms from the split operands (A = A_hi + A_lo, X = X_hi + X_lo, each
part the round-to-nearest TF32 value), which leaves only the FP32
accumulation; (2) against the exact FP64 product of the FP32 A and the FP64
X, where it must sit at FP32-level error, far below the plain TF32 pass."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2002_07138_gb300 as plu

pytestmark = pytest.mark.gpu


def dev(X, dtype=torch.float64):
    X = np.asarray(X)
    out = plu.colmajor_empty(X.shape[0], X.shape[1], dtype=dtype)
    out.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return out


def host(T):
    return T.double().cpu().numpy()


def dev_f32(X):
    """FP32 column-major CUDA view of X with ld rounded up to a multiple of 4,
    so the tensor maps take it (rows past m are outside the view)."""
    X = np.asarray(X, dtype=np.float32)
    m = X.shape[0]
    big = plu.colmajor_empty((m + 3) // 4 * 4, X.shape[1], dtype=torch.float32)
    A = big[:m, :]
    A.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return A


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tf32_rna(a):
    """float32 -> TF32, round to nearest, ties away from zero."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def split(a32):
    """(hi, lo) as float64: hi = TF32(a), lo = TF32(a - hi), a - hi exact in FP32."""
    hi = tf32_rna(a32)
    lo = tf32_rna((a32 - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


SHAPES = [(1000, 777, 25), (2048, 1536, 276), (300, 257, 1), (512, 8192, 110),
          (4096, 1024, 512), (132, 4100, 48), (129, 33, 17), (3001, 2003, 256)]


@pytest.mark.parametrize("m,n,cols", SHAPES)
@pytest.mark.parametrize("trans", [0, 1])
def test_pass_tf32x3_matches_split_operands(ctx, m, n, cols, trans):
    A32 = synth.gaussian_np(m, n, 21).astype(np.float32)
    X = synth.gaussian_np(n if trans == 0 else m, cols, 22)
    Ah, Al = split(A32)
    Xh, Xl = split(X.astype(np.float32))
    op = (lambda M: M) if trans == 0 else (lambda M: M.T)
    model = op(Ah) @ Xh + op(Al) @ Xh + op(Ah) @ Xl
    Ad = dev_f32(A32)
    got = host(plu.plu_pass(ctx, Ad, trans, dev(X), "tf32x3"))
    K = n if trans == 0 else m
    assert rel(got, model) < 4e-7 * np.sqrt(K / 32.0) + 1e-6
    # against the exact product: FP32-level, orders of magnitude below TF32
    exact = op(A32.astype(np.float64)) @ X
    e3 = rel(got, exact)
    assert e3 < 4e-7 * np.sqrt(K / 32.0) + 2e-6
    if K >= 256:
        e1 = rel(host(plu.plu_pass(ctx, Ad, trans, dev(X), "tf32")), exact)
        assert e3 < e1 / 50, (e3, e1)


@pytest.mark.parametrize("trans", [0, 1])
def test_pass_tf32x3_elementwise_bound(ctx, trans):
    """Every entry within the worst-case bound of the split and the FP32
    accumulation, relative to (|A| |X|)_ij: 4 * 2^-22 for the dropped and
    rounded remainders plus 2^-22 per accumulation step (K / 8 MMA slices)."""
    m, n, cols = 2500, 1800, 64
    rng = np.random.default_rng(5)
    A32 = (rng.standard_normal((m, n)) * np.exp2(rng.integers(-8, 9, size=(m, 1)))).astype(np.float32)
    X = rng.standard_normal((n if trans == 0 else m, cols))
    op = (lambda M: M) if trans == 0 else (lambda M: M.T)
    exact = op(A32.astype(np.float64)) @ X
    absb = np.abs(op(A32.astype(np.float64))) @ np.abs(X)
    got = host(plu.plu_pass(ctx, dev_f32(A32), trans, dev(X), "tf32x3"))
    K = n if trans == 0 else m
    bound = (4 + K / 8 + 16) * 2.0 ** -22
    assert np.all(np.abs(got - exact) <= bound * absb)


@pytest.mark.parametrize("trans", [0, 1])
def test_pass_tf32x3_leading_dimension_and_fallback(ctx, trans):
    """A sub-matrix view (ld > m) through the tensor maps, and an ld that is
    not a multiple of 4 (no TMA) through the FP32 SIMT kernel."""
    m, n, cols = 600, 500, 40
    X = synth.gaussian_np(n if trans == 0 else m, cols, 14)
    for ld in (604, 601):
        big = plu.colmajor_empty(ld, n, dtype=torch.float32)
        big.copy_(torch.from_numpy(synth.gaussian_np(ld, n, 13).astype(np.float32)))
        A = big[:m, :]
        A64 = host(A)
        exact = A64 @ X if trans == 0 else A64.T @ X
        got = host(plu.plu_pass(ctx, A, trans, dev(X), "tf32x3"))
        assert rel(got, exact) < 2e-6


def test_pass_tf32x3_rejects_fp64_matrix(ctx):
    A = dev(synth.gaussian_np(100, 80, 1))
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_pass(ctx, A, 0, dev(synth.gaussian_np(80, 4, 2)), "tf32x3")
    assert ei.value.name == "PLU_EUNSUPPORTED"


@pytest.mark.parametrize("trans,cols", [(0, 256), (1, 276)])
def test_pass_tf32x3_full_size(ctx, trans, cols):
    """The 32768 x 32768 FP32 matrix of the mixed-precision workload (the
    last pass Y = A V_k takes 256 columns, the passes 276): sampled rows of Y
    against the FP64 products of those rows, computed on the GPU in FP64."""
    N = 32768
    g = torch.Generator(device="cuda").manual_seed(3)
    A = plu.colmajor_empty(N, N, dtype=torch.float32)
    A.copy_(torch.randn(N, N, device="cuda", generator=g, dtype=torch.float32).t())
    X = plu.colmajor_empty(N, cols)
    X.copy_(torch.randn(N, cols, device="cuda", generator=g, dtype=torch.float64))
    Y = plu.plu_pass(ctx, A, trans, X, "tf32x3")
    rows = torch.tensor(np.random.default_rng(1).choice(N, 96, replace=False), device="cuda")
    Ad = A.index_select(0, rows).double() if trans == 0 else A.index_select(1, rows).t().double()
    ref = Ad @ X
    err = float(torch.linalg.norm(Y.index_select(0, rows) - ref) / torch.linalg.norm(ref))
    assert err < 4e-7 * np.sqrt(N / 32.0) + 2e-6
    del A, X, Y, Ad, ref
    torch.cuda.empty_cache()


def test_singlepass_tf32x3_error_matches_fp64(ctx):
    """Alg. singlepasslu with FP32-accurate split passes: its error within
    1.1x of the FP64 single pass on the same Omega (the single pass has no
    re-orthogonalising step, so the pass rounding enters G and H directly)."""
    sig = synth.sigma_profile("type1", 3000)
    A = synth.svd_matrix_np(6000, 3000, sig, seed=7)
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    gp, gq, gL, gU, _ = plu.plu_singlepass(ctx, dev(A64h), 30, seed=1, prec="fp64")
    e64 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    gp, gq, gL, gU, _ = plu.plu_singlepass(ctx, dev(A32, torch.float32), 30, seed=1,
                                           prec="tf32x3")
    e3 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert e3 <= 1.1 * e64, (e3, e64)
