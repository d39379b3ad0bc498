"""Pins of the RandLU tail in the oracle (Alg. rlu steps 4-7 and
Eq. pseudoinverse), after the range finder of Alg. basicpoweriteration.

The tail forms B = L_y^+ P A, factors Q B^T = L' U', and returns
L = L_y U'^T, U = L'^T.  In exact arithmetic this gives
L U = (L_y L_y^+ P A) Q^T, where L_y L_y^+ is the orthogonal projector onto
range(L_y).  The tests below check that identity with the projector built
from numpy's QR (not from the oracle's normal-equations pseudoinverse), the
structure of the two factors, and exact reconstruction of a rank-k A.  Each
of them fails when P A is replaced by A, when U'^T and L'^T trade places or
lose a transpose, or when the pseudoinverse is formed wrongly.
"""
import numpy as np
import pytest

import synth
from oracle import basic_power_iteration_lu, randlu, rel_lu_error, eckart_young_error


def _is_perm(p, n):
    return sorted(int(x) for x in p) == list(range(n))


@pytest.fixture(scope="module")
def exact_rank20():
    return synth.rank_k_matrix_np(2000, 1500, 20, seed=31)


@pytest.mark.parametrize("p", [0, 1])
def test_randlu_exact_rank_reconstruction(exact_rank20, p):
    """A = B C of rank 20 (2000 x 1500), k = 20, l = 25: range(L_y) holds
    range(P A), so the tail reproduces A up to rounding (Alg. rlu)."""
    A = exact_rank20
    P, Q, L, U = randlu(A, 20, 25, p, seed=4)
    assert _is_perm(P, A.shape[0]) and _is_perm(Q, A.shape[1])
    assert L.shape == (2000, 20) and U.shape == (20, 1500)
    assert np.linalg.norm(A[P][:, Q] - L @ U) <= 1e-13 * np.linalg.norm(A)


@pytest.fixture(scope="module")
def well_conditioned():
    sig = synth.sigma_profile("flat12", 200)          # sigma in [1, 2]
    return synth.svd_matrix_np(300, 200, sig, seed=12)


@pytest.mark.parametrize("k,l,p", [(16, 16, 0), (16, 16, 1), (10, 16, 1)])
def test_randlu_tail_is_projection(well_conditioned, k, l, p):
    """L U = (Pi P A) Q^T with Pi the orthogonal projector onto range(L_y(:, 1:k))
    (Eq. pseudoinverse: L_y^+ = (L_y^T L_y)^{-1} L_y^T, so L_y L_y^+ = Pi)."""
    A = well_conditioned
    P, Q, L, U = randlu(A, k, l, p, seed=8)
    perm, Ly, _ = basic_power_iteration_lu(A, l, p, seed=8)
    assert np.array_equal(perm, P)
    Qy, _ = np.linalg.qr(Ly[:, :k])
    PA = A[perm, :]
    target = (Qy @ (Qy.T @ PA))[:, Q]
    assert np.linalg.norm(L @ U - target) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("p", [0, 1])
def test_randlu_factor_structure(well_conditioned, p):
    """U = L'^T is unit upper trapezoidal with |u_ij| <= 1 (partial pivoting
    in lu(B^T)); L = L_y U'^T is lower trapezoidal (L_y unit lower
    trapezoidal, U'^T lower triangular) with the diagonal of U'."""
    A = well_conditioned
    k, l = 12, 16
    P, Q, L, U = randlu(A, k, l, p, seed=21)
    assert np.all(np.tril(U, -1) == 0.0)
    assert np.array_equal(np.diag(U), np.ones(k))
    assert np.max(np.abs(U)) <= 1.0
    assert np.all(np.triu(L, 1) == 0.0)
    perm, Ly, _ = basic_power_iteration_lu(A, l, p, seed=21)
    # U'^T = L_y(1:k, 1:k)^{-1} L(1:k, 1:k) is lower triangular (L_y is unit
    # lower), and it shares its diagonal with L
    Lb = np.linalg.solve(Ly[:k, :k], L[:k, :k])
    assert np.max(np.abs(np.triu(Lb, 1))) <= 1e-12 * np.max(np.abs(Lb))
    assert np.allclose(np.diag(L), np.diag(Lb), rtol=1e-12, atol=0.0)


def test_randlu_error_above_optimum():
    """The relative error of the rank-k factors is at least the Eckart-Young
    optimum of the known spectrum and within a small factor of it."""
    n = 200
    sig = synth.sigma_profile("type2", n)
    A = synth.svd_matrix_np(300, n, sig, seed=3)
    k, l = 15, 25
    P, Q, L, U = randlu(A, k, l, 1, seed=6)
    err = rel_lu_error(A, P, Q, L, U)
    opt = eckart_young_error(sig, k)
    assert opt * (1 - 1e-9) <= err <= 1.5 * opt
