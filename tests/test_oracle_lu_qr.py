"""Pins of the oracle's partial-pivoting LU and economy QR."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import getrf, lu_permuted_L, qr_economy


def exact_lu(X):
    """Partial-pivoting elimination in exact rational arithmetic on the
    float64 values of X: pivot = largest |a_ij| among the rows from j down in
    the current (swapped) order, first one on ties; zero columns skipped."""
    m, n = X.shape
    A = [[Fraction(float(X[i, j])) for j in range(n)] for i in range(m)]
    perm = list(range(m))
    r = min(m, n)
    ties = 0
    for j in range(r):
        best = j
        for i in range(j + 1, m):
            if abs(A[i][j]) > abs(A[best][j]):
                best = i
        ties += sum(1 for i in range(j, m) if i != best and abs(A[i][j]) == abs(A[best][j])
                    and A[best][j] != 0)
        if A[best][j] != 0:
            A[j], A[best] = A[best], A[j]
            perm[j], perm[best] = perm[best], perm[j]
            for i in range(j + 1, m):
                A[i][j] = A[i][j] / A[j][j]
        for i in range(j + 1, m):
            for c in range(j + 1, n):
                A[i][c] -= A[i][j] * A[j][c]
    L = [[(A[i][j] if j < i else (Fraction(1) if i == j else Fraction(0))) for j in range(r)]
         for i in range(m)]
    U = [[(A[i][j] if j >= i else Fraction(0)) for j in range(n)] for i in range(r)]
    return perm, L, U, ties


def _tof(M):
    return np.array([[float(x) for x in row] for row in M])


@pytest.mark.parametrize("seed", range(6))
def test_getrf_matches_exact_rational_random(seed):
    X = np.random.default_rng(seed).standard_normal((8, 6))
    perm, L, U, info = getrf(X)
    eperm, eL, eU, _ = exact_lu(X)
    assert list(perm) == eperm
    assert info == 0
    assert np.max(np.abs(L - _tof(eL))) <= 1e-15 * 8
    assert np.max(np.abs(U - _tof(eU))) <= 1e-15 * 8 * np.max(np.abs(X))


def _dyadic_tie_matrices(count, m=8, n=6):
    """Small-integer matrices whose exact elimination has only power-of-two
    pivots (so float64 elimination is exact) and at least two pivot ties."""
    rng = np.random.default_rng(7)
    out = []
    tries = 0
    while len(out) < count and tries < 200000:
        tries += 1
        X = rng.integers(-2, 3, size=(m, n)).astype(np.float64)
        perm, L, U, ties = exact_lu(X)
        piv = [U[j][j] for j in range(min(m, n))]
        ok = all(p == 0 or (abs(p).numerator & (abs(p).numerator - 1) == 0
                            and abs(p).denominator & (abs(p).denominator - 1) == 0) for p in piv)
        if ok and ties >= 2:
            out.append(X)
    return out


def test_getrf_tie_rule_exact():
    mats = _dyadic_tie_matrices(12)
    assert len(mats) == 12
    for X in mats:
        perm, L, U, info = getrf(X)
        eperm, eL, eU, _ = exact_lu(X)
        assert list(perm) == eperm
        assert np.array_equal(L, _tof(eL)) and np.array_equal(U, _tof(eU))


def test_getrf_zero_column_and_rank_deficient():
    X = np.random.default_rng(3).standard_normal((8, 6))
    X[:, 2] = 0.0
    perm, L, U, info = getrf(X)
    assert info == 3
    assert np.allclose(X[perm], L @ U, atol=1e-14)
    # rank-2 panel: later columns eliminate to (near) zero; P X = L U still holds
    B = np.random.default_rng(4).standard_normal((10, 2))
    X = B @ np.random.default_rng(5).standard_normal((2, 5))
    perm, L, U, info = getrf(X)
    assert np.allclose(X[perm], L @ U, atol=1e-13)
    assert np.max(np.abs(L)) <= 1.0


def test_getrf_matches_lapack_pivots():
    X = np.random.default_rng(11).standard_normal((2000, 25))
    perm, L, U, info = getrf(X)
    P, Ls, Us = scipy.linalg.lu(X)
    sperm = np.argmax(P, axis=0)          # X = P Ls Us -> X[sperm] = Ls Us
    assert np.array_equal(perm, sperm)
    assert np.max(np.abs(L - Ls)) < 1e-13
    assert np.max(np.abs(U - Us)) < 1e-13
    assert np.max(np.abs(L)) <= 1.0


def test_getrf_multipliers_scale_by_reciprocal_like_lapack():
    """MATLAB's lu is LAPACK getrf, whose getf2 / getrf2 scale the pivot
    column by 1 / u_jj (|u_jj| normal): one elimination step matches LAPACK
    bit for bit, and the plain quotient differs in many entries."""
    X = np.random.default_rng(21).standard_normal((5000, 1))
    perm, L, U, _ = getrf(X)
    _, Ls, _ = scipy.linalg.lu(X)
    assert np.array_equal(L[:, 0], Ls[:, 0])
    assert np.sum(X[perm, 0] / X[perm[0], 0] != L[:, 0]) > 100
    # a subnormal pivot is divided, not inverted (1 / u would overflow)
    Y = np.array([[4e-320], [2e-320], [1e-320]])
    perm, L, U, _ = getrf(Y)
    assert np.array_equal(L[:, 0], Y[perm, 0] / Y[perm[0], 0])


def test_permuted_L_rows_align():
    X = np.random.default_rng(12).standard_normal((50, 7))
    Lp = lu_permuted_L(X)
    perm, L, U, _ = getrf(X)
    assert np.allclose(Lp @ U, X, atol=1e-13)          # P^T L U = X
    assert np.array_equal(Lp[perm], L)
    # wide input (more columns than rows) keeps r = m
    Xw = np.random.default_rng(13).standard_normal((4, 9))
    perm, L, U, _ = getrf(Xw)
    assert L.shape == (4, 4) and U.shape == (4, 9)
    assert np.allclose(Xw[perm], L @ U, atol=1e-13)


@pytest.mark.parametrize("shape", [(40, 7), (300, 25), (9, 9)])
def test_qr_economy(shape):
    X = np.random.default_rng(shape[0]).standard_normal(shape)
    Q, R = qr_economy(X)
    n, l = shape
    assert Q.shape == (n, l) and R.shape == (l, l)
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) < 1e-14
    assert np.max(np.abs(Q @ R - X)) < 1e-13
    assert np.all(np.diag(R) >= 0) and np.allclose(R, np.triu(R))
    Qn, Rn = np.linalg.qr(X)
    s = np.sign(np.diag(Rn))
    assert np.max(np.abs(Q - Qn * s[None, :])) < 1e-12


def test_qr_ill_conditioned_columns():
    rng = np.random.default_rng(21)
    X = rng.standard_normal((200, 12)) * np.logspace(0, -8, 12)[None, :]
    Q, R = qr_economy(X)
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) < 1e-14
    assert np.max(np.abs(Q @ R - X)) < 1e-14
