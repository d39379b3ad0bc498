"""GPU parity of the panel LU with tensor-core trailing updates (the lu of
Alg. gpowerlu and the getrf steps of Alg. bpowerlu, as the mixed-precision
modes run them) against the oracle's partial-pivoting LU, through the C ABI
with the context's LU update mode set to the tensor cores.

The updates are FP64-accurate sums of exact FP16 digit products, so on
random panels the pivots equal the oracle's and the factors agree to the
same 1e-12 as the FP64-FMA kernel; on panels whose elimination is exact in
binary arithmetic the factors are bit-identical."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2002_07138_gb300 as plu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tctx(built_lib):
    c = plu.Context(0)
    c.set_lu_updates(1)
    yield c
    torch.cuda.synchronize()
    c.close()


def dev(X):
    X = np.asarray(X, dtype=np.float64)
    out = plu.colmajor_empty(X.shape[0], X.shape[1])
    out.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return out


def host(T):
    return T.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_getrf(tctx, X, tol=1e-12):
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(tctx, dev(X))
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < tol
    assert rel(host(gU), U) < tol
    assert ginfo == info
    return perm, L, U


# one leaf; several leaves with a ragged last one; ragged 128-row tiles; an
# update wider than one launch's 256 columns (two and three launches)
@pytest.mark.parametrize("rows,cols", [(2000, 20), (1500, 100), (513, 64), (64, 64), (10000, 7),
                                       (3001, 70), (5000, 290), (1031, 600)])
def test_getrf_tc(tctx, rows, cols):
    check_getrf(tctx, synth.gaussian_np(rows, cols, 11 * rows + cols))


@pytest.mark.parametrize("rows,cols", [(2000, 25), (1500, 110), (777, 64), (300, 300), (4100, 97)])
def test_lu_reorth_tc(tctx, rows, cols):
    X = synth.gaussian_np(rows, cols, rows + 3 * cols)
    ref = oracle.lu_permuted_L(X)
    got = host(plu.plu_lu_reorth(tctx, dev(X)))
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("rows,cols", [(32768, 276), (32768, 256), (20000, 512)])
def test_getrf_tc_full_size_panels(tctx, rows, cols):
    """The panels of the 32768^2 mixed workload (the m x l sketch and the
    m x k Y of the tail) and of the 20000 x 10000 fixed-precision workload."""
    check_getrf(tctx, synth.gaussian_np(rows, cols, rows + cols))


def test_getrf_tc_scaled_rows_and_columns(tctx):
    """Rows and columns scaled by powers of two spread over 2^-60 .. 2^60:
    the digits are cut relative to each multiplier row's and each U12
    column's own exponent."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3000, 96))
    X *= np.exp2(rng.integers(-60, 61, size=3000)).astype(np.float64)[:, None]
    X *= np.exp2(rng.integers(-60, 61, size=96)).astype(np.float64)[None, :]
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(tctx, dev(X))
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < 1e-12
    # U's rows live on very different scales: compare each row on its own
    gU = host(gU)
    for r in range(U.shape[0]):
        assert np.linalg.norm(gU[r] - U[r]) <= 1e-12 * np.linalg.norm(U[r])


def exact_panel(rng, r, rows, dup=0):
    """X (rows x r) with X[Pi] = [L0; L1] U0: a unit diagonal, dyadic
    multipliers |l| <= 1/2 elsewhere, small-integer U0 with power-of-two
    diagonal, so partial pivoting is exact in binary arithmetic; plus `dup`
    copies (half of them negated) of diagonal rows, which tie with their
    originals exactly when their column comes up."""
    L0 = np.tril(rng.integers(-2, 3, size=(rows, r)).astype(np.float64) / 4.0, -1)
    L0[:r, :r] += np.eye(r)
    U0 = np.triu(rng.integers(-8, 9, size=(r, r)).astype(np.float64), 1)
    U0 += np.diag(rng.choice([-64.0, 64.0, -32.0, 32.0], size=r))
    Xs = L0 @ U0
    if dup:
        src = rng.choice(r, size=dup, replace=False)
        sign = np.where(np.arange(dup) % 2 == 0, 1.0, -1.0)
        Xs = np.vstack([Xs, Xs[src] * sign[:, None]])
    X = np.empty_like(Xs)
    X[rng.permutation(Xs.shape[0])] = Xs
    return X


def test_getrf_tc_exact_panel_is_bit_identical(tctx):
    """On a panel whose elimination is exact in binary arithmetic (see
    exact_panel) L and U are bit-identical to the oracle's, across three
    tensor-core updates."""
    X = exact_panel(np.random.default_rng(21), 96, 900)
    perm, L, U, info = oracle.getrf(X)
    assert np.array_equal(X[perm], L @ U)
    gp, gL, gU, ginfo = plu.plu_getrf(tctx, dev(X))
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert np.array_equal(host(gL), L)
    assert np.array_equal(host(gU), U)


def test_getrf_tc_tie_rule(tctx):
    """Tied pivot magnitudes (duplicated and negated rows) on exact panels
    with several leaves: the row first in the current order must win, as in
    LAPACK (rows in place on the GPU, row swaps in the oracle)."""
    for seed in range(4):
        X = exact_panel(np.random.default_rng(100 + seed), 70, 500, dup=40)
        perm, L, U, info = oracle.getrf(X)
        assert np.array_equal(X[perm], L @ U)
        gp, gL, gU, ginfo = plu.plu_getrf(tctx, dev(X))
        assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
        assert np.array_equal(host(gL), L) and np.array_equal(host(gU), U)
        assert ginfo == info


@pytest.mark.parametrize("zc", [3, 40])
def test_getrf_tc_zero_column(tctx, zc):
    X = synth.gaussian_np(700, 70, 5)
    X[:, zc] = 0.0
    perm, L, U, info = oracle.getrf(X)
    gp, gL, gU, ginfo = plu.plu_getrf(tctx, dev(X))
    assert info == zc + 1 and ginfo == zc + 1
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), perm)
    assert rel(host(gL), L) < 1e-12 and rel(host(gU), U) < 1e-12


def test_getrf_tc_reports_non_finite(tctx):
    X = synth.gaussian_np(900, 80, 6)
    X[400, 50] = np.nan
    with pytest.raises(plu.PLUError):
        plu.plu_getrf(tctx, dev(X))
    # the context keeps working
    check_getrf(tctx, synth.gaussian_np(600, 40, 7))


@pytest.mark.parametrize("v", [2, 3, 4])
def test_powerlu_fp64_with_tc_lu_matches_oracle(tctx, v):
    """Whole PowerLU (every pass FP64) with every panel LU on the tensor-core
    path: identical p, q and factors within 1e-10 of the oracle."""
    m, n, k, l = 2000, 1500, 20, 25
    A = synth.svd_matrix_np(m, n, synth.sigma_profile("type1", n), seed=0)
    p, q, L, U = oracle.powerlu(A, k, l, v, seed=0)
    gp, gq, gL, gU, rep = plu.plu_powerlu(tctx, dev(A), k, l, v, seed=0, prec="fp64")
    assert np.array_equal(gp.cpu().numpy(), p) and np.array_equal(gq.cpu().numpy(), q)
    assert rel(host(gL), L) < 1e-10 and rel(host(gU), U) < 1e-10


def test_lu_update_mode_is_validated(tctx):
    with pytest.raises(plu.PLUError):
        tctx.set_lu_updates(2)
    tctx.set_lu_updates(1)
