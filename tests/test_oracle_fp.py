"""Pins of the oracle's blocked adaptive rank determination
(Alg. adaptivewithoutupdating, the precise variant of Sec. 6.4) and
PowerLU_FP (Alg. powerlufp)."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import (gpowerlu, adaptive_rank, powerlu_fp, rel_lu_error, eckart_young_rank,
                    eckart_young_error)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_indicator_equals_explicit_updating():
    """Thms. thm:22 and errorerror: the blocked loop A^(i) = A^(i-1) -
    A^(i-1) V_i V_i^T (Eqs. b1-b2) gives A^(i) = A (I - P_i) with P_i a
    projector, and ||A^(i)||_F^2 = ||A||_F^2 - sum_{j<=i} ||A V_j||_F^2."""
    sig = synth.sigma_profile("type1", 200)
    A = synth.svd_matrix_np(300, 200, sig, seed=3)
    b, l = 5, 40
    V = gpowerlu(A, l, 4, seed=2)
    Ai = A.copy()
    nA2 = np.sum(A * A)
    acc = 0.0
    P = np.zeros((200, 200))
    for i in range(l // b):
        Vi = V[:, i * b:(i + 1) * b]
        Ai = Ai - Ai @ Vi @ Vi.T
        P = P + Vi @ Vi.T
        assert np.max(np.abs(P @ P - P)) < 1e-13
        assert np.max(np.abs(Ai - A @ (np.eye(200) - P))) < 1e-13
        acc += np.sum((A @ Vi) ** 2)
        explicit = np.sum(Ai * Ai)
        assert abs(explicit - (nA2 - acc)) <= 1e-12 * nA2


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_svd_ranks.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, eps, svd, fp, b = line.split()
                rows.append((t, float(eps), int(svd), int(fp), int(b)))
    return rows


@pytest.mark.parametrize("row", _table1())
def test_table1_truncated_svd_ranks(row):
    """Table 1: optimal ranks of the n = 8000 matrix types from their
    singular values (Eq. ey)."""
    t, eps, svd_rank, _, _ = row
    assert eckart_young_rank(synth.sigma_profile(t, 8000), eps) == svd_rank


def test_blocked_rank_stops_at_first_block_and_precise_refines():
    sig = synth.sigma_profile("type2", 400)
    A = synth.svd_matrix_np(500, 400, sig, seed=6)
    eps, b, l, v = 1e-4, 10, 200, 4
    kopt = eckart_young_rank(sig, eps)
    k, V, G, E, met = adaptive_rank(A, eps, b, l, v, seed=1)
    assert met and k % b == 0
    nA2 = np.sum(A * A)
    # first block meeting the test
    Es = nA2 - np.cumsum(np.sum(G * G, axis=0))
    assert Es[k - 1] <= eps ** 2 * nA2 < Es[k - b - 1]
    assert kopt <= k <= kopt + b
    kp, _, _, Ep, metp = adaptive_rank(A, eps, b, l, v, seed=1, precise=True)
    assert metp and kp <= k and kp >= kopt
    assert Es[kp - 1] <= eps ** 2 * nA2 < Es[kp - 2]
    assert abs(Ep - Es[kp - 1]) <= 1e-12 * nA2


def test_partial_last_block_and_tolerance_not_met():
    sig = synth.sigma_profile("type1", 100)
    A = synth.svd_matrix_np(120, 100, sig, seed=7)
    k, V, G, E, met = adaptive_rank(A, 1e-12, 7, 30, 3, seed=2)
    assert not met and k == 30
    kf, p, q, L, U, Ef, metf = powerlu_fp(A, 1e-12, 7, 30, 3, seed=2)
    assert not metf and kf == 30 and L.shape == (120, 30)


@pytest.mark.parametrize("precise", [False, True])
def test_powerlu_fp_error_meets_tolerance(precise):
    """Alg. powerlufp: the factorisation error equals the indicator
    sqrt(E)/||A||_F (Thm. errorindicator) and meets eps."""
    sig = synth.sigma_profile("type3", 300)
    A = synth.svd_matrix_np(400, 300, sig, seed=8)
    eps = 1e-2
    k, p, q, L, U, E, met = powerlu_fp(A, eps, 8, 80, 4, seed=5, precise=precise)
    assert met
    err = rel_lu_error(A, p, q, L, U)
    ind = math.sqrt(max(E, 0.0) / np.sum(A * A))
    assert err <= eps * (1 + 1e-8)
    assert abs(err - ind) <= 1e-7
    kopt = eckart_young_rank(sig, eps)
    assert k >= kopt
    assert err >= eckart_young_error(sig, k) * (1 - 1e-9)


@pytest.mark.slow
def test_table1_powerlu_fp_rank_type2_n2000():
    """Table 1 in miniature (n = 2000, type 2, eps = 1e-4 and 1e-5, b = 10,
    v = 4, l = 50 b): the PowerLU_FP rank sits within one block above the
    optimum, as the paper reports for n = 8000 (66 vs 65, 82 vs 81)."""
    sig = synth.sigma_profile("type2", 2000)
    A = synth.svd_matrix_np(2000, 2000, sig, seed=10)
    for eps in (1e-4, 1e-5):
        kopt = eckart_young_rank(sig, eps)
        k, *_ = adaptive_rank(A, eps, 10, 500, 4, seed=3, precise=True)
        assert kopt <= k <= kopt + 10


# ---- the restart of the Remark after Alg. adaptivewithoutupdating
def _restart_case():
    sig = 1.0 / np.arange(1, 201)
    A = synth.svd_matrix_np(300, 200, sig, seed=21)
    return A, sig


def test_remainder_operator_equals_explicit_remainder():
    """A_r X and A_r^T Z through G = A W equal the explicit A - A W W^T."""
    from oracle import Remainder, PassCounter
    A, _ = _restart_case()
    W = gpowerlu(A, 24, 3, seed=4)                       # orthonormal n x 24
    Ac = PassCounter(A)
    R = Remainder(Ac, W, A @ W)
    Ar = A - A @ W @ W.T
    X = synth.gaussian_np(200, 7, 5)
    Z = synth.gaussian_np(300, 7, 6)
    assert np.abs(R.mul(X) - Ar @ X).max() <= 1e-12 * np.abs(Ar @ X).max()
    assert np.abs(R.tmul(Z) - Ar.T @ Z).max() <= 1e-12 * np.abs(Ar.T @ Z).max()
    assert Ac.passes == 2


@pytest.mark.parametrize("v", [3, 4])
def test_restart_reaches_tolerance_with_orthonormal_union(v):
    """With l too small for eps, later rounds on the remainder reach it: the
    union of the rounds' bases is orthonormal, the carried-over indicator E
    equals the explicit residual ||A - A W W^T||_F^2 (Thm. errorindicator),
    the factors meet eps, and each round reads A v times."""
    from oracle import adaptive_rank_restart, PassCounter, eckart_young_rank
    A, sig = _restart_case()
    eps, b, l = 0.05, 8, 24
    r_svd = eckart_young_rank(sig, eps)
    assert r_svd > l                                      # one round cannot succeed
    Ac = PassCounter(A)
    k, W, G, E, met, rounds = adaptive_rank_restart(Ac, eps, b, l, v, seed=2, max_rounds=6)
    assert met and rounds >= 2 and k >= r_svd and k <= rounds * l
    assert Ac.passes == rounds * v
    assert np.abs(W.T @ W - np.eye(k)).max() <= 1e-10
    assert np.abs(G - A @ W).max() <= 1e-10 * np.abs(G).max()
    resid = np.sum((A - A @ W @ W.T) ** 2)
    assert abs(E - resid) <= 1e-9 * np.sum(A * A)
    kk, p, q, L, U, E2, met2 = powerlu_fp(A, eps, b, l, v, seed=2, max_rounds=6)
    assert kk == k and met2
    assert rel_lu_error(A, p, q, L, U) <= eps


def test_restart_single_round_is_the_plain_algorithm():
    """max_rounds = 1 is Alg. adaptivewithoutupdating itself: not met, k = l."""
    from oracle import adaptive_rank_restart
    A, _ = _restart_case()
    k, W, G, E, met, rounds = adaptive_rank_restart(A, 0.05, 8, 24, 3, seed=2, max_rounds=1)
    k1, V1, G1, E1, met1 = adaptive_rank(A, 0.05, 8, 24, 3, seed=2)
    assert (k, met, rounds) == (24, False, 1) and (k1, met1) == (24, False)
    assert np.array_equal(W, V1) and np.array_equal(G, G1) and E == E1
