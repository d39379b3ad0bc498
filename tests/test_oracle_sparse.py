"""Pins of the oracle's sparse products (the sprand experiment of Sec. 6) and
of PowerLU / PowerLU_FP run on them: brute force on a hand-written matrix,
the dense product of the same matrix, scipy.sparse, and a sparse matrix of
exact rank r that PowerLU must reproduce to rounding."""
import numpy as np
import pytest

import synth
from oracle import (csr_mul, csr_tmul, SparsePassCounter, PassCounter, powerlu, powerlu_fp,
                    rel_lu_error)


def test_brute_force_8x6():
    """A hand-written 8 x 6 matrix with an empty row and an empty column:
    each product entry summed by explicit loops."""
    A = np.zeros((8, 6))
    A[0, 1], A[0, 5] = 2.0, -1.0
    A[2, 0], A[2, 3], A[2, 4] = 0.5, 3.0, -4.0
    A[3, 3] = 7.0
    A[5, 0], A[5, 1], A[5, 5] = -2.5, 1.5, 0.25
    A[7, 4] = 6.0
    rp, ci, val = synth.dense_to_csr(A)
    assert rp[1] - rp[0] == 2 and rp[2] == rp[1]          # row 1 empty
    X = np.arange(18, dtype=float).reshape(6, 3) - 4.0
    Z = np.arange(24, dtype=float).reshape(8, 3) * 0.5 - 1.0
    Y = csr_mul(8, rp, ci, val, X)
    T = csr_tmul(6, rp, ci, val, Z)
    for i in range(8):
        for c in range(3):
            s = 0.0
            for j in range(6):
                s += A[i, j] * X[j, c]
            assert Y[i, c] == s
    for j in range(6):
        for c in range(3):
            s = 0.0
            for i in range(8):
                s += A[i, j] * Z[i, c]
            assert T[j, c] == s
    assert np.all(T[2] == 0.0)                             # column 2 empty


@pytest.mark.parametrize("m,n,density", [(300, 200, 0.02), (157, 411, 0.05), (64, 64, 0.003)])
def test_products_match_dense(m, n, density):
    rp, ci, val = synth.sprand_csr(m, n, density, seed=m + n)
    A = synth.csr_to_dense(m, n, rp, ci, val)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, 7))
    Z = rng.standard_normal((m, 5))
    scale = np.abs(A).sum() + 1.0
    assert np.max(np.abs(csr_mul(m, rp, ci, val, X) - A @ X)) < 1e-14 * scale
    assert np.max(np.abs(csr_tmul(n, rp, ci, val, Z) - A.T @ Z)) < 1e-14 * scale


def test_products_match_scipy():
    sp = pytest.importorskip("scipy.sparse")
    m, n = 500, 350
    rp, ci, val = synth.sprand_csr(m, n, 0.01, seed=9)
    S = sp.csr_matrix((val, ci, rp), shape=(m, n))
    X = np.random.default_rng(2).standard_normal((n, 11))
    Z = np.random.default_rng(3).standard_normal((m, 4))
    np.testing.assert_allclose(csr_mul(m, rp, ci, val, X), S @ X, rtol=0, atol=1e-13)
    np.testing.assert_allclose(csr_tmul(n, rp, ci, val, Z), S.T @ Z, rtol=0, atol=1e-13)


def test_unsorted_columns_same_product():
    m, n = 120, 90
    rp, ci, val = synth.sprand_csr(m, n, 0.1, seed=4)
    rng = np.random.default_rng(5)
    ci2, val2 = ci.copy(), val.copy()
    for i in range(m):
        s, e = rp[i], rp[i + 1]
        perm = rng.permutation(e - s) + s
        ci2[s:e], val2[s:e] = ci[perm], val[perm]
    X = rng.standard_normal((n, 3))
    np.testing.assert_allclose(csr_mul(m, rp, ci2, val2, X), csr_mul(m, rp, ci, val, X),
                               rtol=0, atol=1e-13)


def test_selected_rows_match_full_product():
    m, n = 260, 190
    rp, ci, val = synth.sprand_csr(m, n, 0.05, seed=12)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((n, 5))
    Z = rng.standard_normal((m, 5))
    sel_r = np.array([259, 0, 17, 133, 17 + 1])
    sel_c = np.array([5, 189, 0, 77])
    np.testing.assert_array_equal(csr_mul(m, rp, ci, val, X, rows=sel_r),
                                  csr_mul(m, rp, ci, val, X)[sel_r])
    np.testing.assert_array_equal(csr_tmul(n, rp, ci, val, Z, rows=sel_c),
                                  csr_tmul(n, rp, ci, val, Z)[sel_c])


def test_empty_matrix():
    rp = np.zeros(11, dtype=np.int64)
    e = np.zeros(0, dtype=np.int32)
    ev = np.zeros(0)
    assert np.all(csr_mul(10, rp, e, ev, np.ones((7, 3))) == 0.0)
    assert np.all(csr_tmul(7, rp, e, ev, np.ones((10, 3))) == 0.0)
    assert SparsePassCounter(10, 7, rp, e, ev).frob2() == 0.0


def test_transpose_generator_consistent():
    m, n = 210, 130
    rp, ci, val = synth.sprand_csr(m, n, 0.04, seed=8)
    trp, tci, tval = synth.csr_transpose(m, n, rp, ci, val)
    A = synth.csr_to_dense(m, n, rp, ci, val)
    np.testing.assert_array_equal(synth.csr_to_dense(n, m, trp, tci, tval), A.T)
    # the CSR of A^T used as an A gives A^T X by the row rule
    X = np.random.default_rng(0).standard_normal((m, 4))
    np.testing.assert_allclose(csr_mul(n, trp, tci, tval, X), csr_tmul(n, rp, ci, val, X),
                               rtol=0, atol=1e-13)


def test_sprand_density_and_range():
    m, n, d = 2000, 1500, 0.003
    rp, ci, val = synth.sprand_csr(m, n, d, seed=0)
    nnz = int(rp[-1])
    assert abs(nnz - d * m * n) < 0.01 * d * m * n
    assert np.all(np.diff(rp) >= 0) and ci.min() >= 0 and ci.max() < n
    assert val.min() >= 0.0 and val.max() < 1.0
    lin = np.repeat(np.arange(m), np.diff(rp)) * n + ci
    assert np.unique(lin).size == nnz


@pytest.mark.parametrize("v", [2, 3, 4])
def test_powerlu_sparse_equals_dense(v):
    """PowerLU on the sparse passes is PowerLU on the dense A: same pivots,
    factors equal to rounding, exactly v passes (Sec. 3.3)."""
    m, n = 400, 300
    rp, ci, val = synth.sprand_csr(m, n, 0.02, seed=v)
    A = synth.csr_to_dense(m, n, rp, ci, val)
    S = SparsePassCounter(m, n, rp, ci, val)
    p, q, L, U = powerlu(S, 12, 16, v, seed=7)
    assert S.passes == v
    pd, qd, Ld, Ud = powerlu(PassCounter(A), 12, 16, v, seed=7)
    np.testing.assert_array_equal(p, pd)
    np.testing.assert_array_equal(q, qd)
    assert np.linalg.norm(L - Ld) <= 1e-12 * np.linalg.norm(Ld)
    assert np.linalg.norm(U - Ud) <= 1e-12 * np.linalg.norm(Ud)


@pytest.mark.parametrize("v", [2, 3])
def test_powerlu_sparse_exact_rank(v):
    """A sparse A of exact rank r is reproduced to rounding at k = r."""
    m, n, r = 350, 260, 6
    A = synth.sparse_rank_r(m, n, r, seed=11)
    rp, ci, val = synth.dense_to_csr(A)
    assert rp[-1] < 0.2 * m * n
    p, q, L, U = powerlu(SparsePassCounter(m, n, rp, ci, val), r, r + 4, v, seed=2)
    assert rel_lu_error(A, p, q, L, U) < 1e-12


def test_powerlu_fp_sparse_finds_rank():
    """Alg. powerlufp on a sparse rank-r A stops at k = r (b = 1, the
    indicator E drops to rounding once r columns are taken)."""
    m, n, r = 300, 240, 5
    A = synth.sparse_rank_r(m, n, r, seed=13)
    rp, ci, val = synth.dense_to_csr(A)
    S = SparsePassCounter(m, n, rp, ci, val)
    assert abs(S.frob2() - np.sum(A * A)) <= 1e-12 * np.sum(A * A)
    k, p, q, L, U, E, met = powerlu_fp(S, 1e-6, 1, 20, 3, seed=4)
    assert met and k == r
    assert rel_lu_error(A, p, q, L, U) < 1e-10


def test_powerlu_fp_restart_sparse_equals_dense():
    """The restart on the remainder (two rounds) gives the same rank, pivots
    and factors on the sparse passes as on the dense A."""
    m, n = 300, 220
    rp, ci, val = synth.sprand_csr(m, n, 0.03, seed=21)
    A = synth.csr_to_dense(m, n, rp, ci, val)
    S = SparsePassCounter(m, n, rp, ci, val)
    ks, ps, qs, Ls, Us, Es, mets = powerlu_fp(S, 0.05, 4, 12, 3, seed=8, max_rounds=2)
    kd, pd, qd, Ld, Ud, Ed, metd = powerlu_fp(PassCounter(A), 0.05, 4, 12, 3, seed=8,
                                                max_rounds=2)
    assert ks == kd == 24 and not mets and not metd
    np.testing.assert_array_equal(ps, pd)
    np.testing.assert_array_equal(qs, qd)
    assert np.linalg.norm(Ls - Ld) <= 1e-12 * np.linalg.norm(Ld)
    assert np.linalg.norm(Us - Ud) <= 1e-12 * np.linalg.norm(Ud)
    assert abs(Es - Ed) <= 1e-10 * S.frob2()
