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
