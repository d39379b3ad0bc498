"""Pins of the oracle's PowerLU (Alg. bpowerlu + Alg. gpowerlu), RandLU
(Alg. rlu + Alg. basicpoweriteration) and single-pass LU (Alg. singlepasslu)
against closed forms, theorems and invariants of the paper."""
import math

import numpy as np
import pytest

import synth
from oracle import (gpowerlu, powerlu, randlu, singlepass, PassCounter, gaussian_matrix,
                    STREAM_OMEGA_N, STREAM_OMEGA_M, STREAM_OMEGA_SP, rel_lu_error,
                    eckart_young_error, max_principal_sine)
from oracle.powerlu import singlepass_streamed_GH


def _is_perm(p, n):
    return sorted(int(x) for x in p) == list(range(n))


@pytest.fixture(scope="module")
def flatA():
    sig = synth.sigma_profile("flat12", 150)
    return synth.svd_matrix_np(200, 150, sig, seed=5)


@pytest.mark.parametrize("v", [2, 3, 4, 5, 6])
def test_reorthogonalisation_keeps_range(flatA, v):
    """Remark after Alg. rlu: re-orthogonalisation does not change the range
    in exact arithmetic: V spans (A^T A)^p A^T Omega (v even) or
    (A^T A)^p Omega (v odd), p = floor((v-1)/2)."""
    A = flatA
    m, n = A.shape
    l, seed = 10, 17
    V = gpowerlu(A, l, v, seed)
    assert np.max(np.abs(V.T @ V - np.eye(l))) < 1e-13
    p = (v - 1) // 2
    if v % 2 == 0:
        Y = A.T @ gaussian_matrix(m, l, seed, STREAM_OMEGA_M)
    else:
        Y = gaussian_matrix(n, l, seed, STREAM_OMEGA_N)
    for _ in range(p):
        Y = A.T @ (A @ Y)
    assert max_principal_sine(V, Y) < 1e-12


@pytest.mark.parametrize("v", [2, 3, 4, 5, 6, 7])
def test_pass_count_is_v(v):
    """Generalised PowerLU reads A exactly v times (Sec. 3.3)."""
    A = PassCounter(synth.gaussian_np(60, 40, 1))
    powerlu(A, 5, 8, v, seed=3)
    assert A.passes == v


@pytest.mark.parametrize("p", [0, 1, 2])
def test_randlu_pass_count(p):
    """RandLU accesses A 2p + 2 times (Sec. 3.2)."""
    A = PassCounter(synth.gaussian_np(60, 40, 1))
    randlu(A, 5, 8, p, seed=3)
    assert A.passes == 2 * p + 2


@pytest.fixture(scope="module")
def type2A():
    return synth.svd_matrix_np(300, 200, synth.sigma_profile("type2", 200), seed=9)


@pytest.mark.parametrize("v", [2, 3, 4])
def test_powerlu_closed_form_and_structure(type2A, v):
    """Eqs. plu-powerlufinal: L U = P (A V_k V_k^T) Q^T exactly; L1, L2 unit
    lower trapezoidal with |entries| <= 1; U = L2^T unit upper."""
    A = type2A
    m, n = A.shape
    k, l = 12, 18
    p, q, L, U, V, info = powerlu(A, k, l, v, seed=1, return_basis=True)
    assert info == (0, 0)
    assert _is_perm(p, m) and _is_perm(q, n)
    assert L.shape == (m, k) and U.shape == (k, n)
    Vk = V[:, :k]
    AVV = A @ Vk @ Vk.T
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(AVV[p][:, q] - L @ U) <= 1e-13 * nrm
    assert np.allclose(np.triu(L, 1), 0.0)              # L lower trapezoidal
    assert np.allclose(np.tril(U, -1), 0.0)             # U upper trapezoidal
    assert np.allclose(np.diag(U), 1.0) and np.max(np.abs(U)) <= 1.0 + 1e-15
    # Thm. errorindicator: ||A - A Vk Vk^T||_F^2 = ||A||_F^2 - ||A Vk||_F^2
    err = rel_lu_error(A, p, q, L, U)
    ind = math.sqrt(max(nrm ** 2 - np.linalg.norm(A @ Vk) ** 2, 0.0)) / nrm
    assert abs(err - ind) <= 1e-6 * ind + 1e-13
    # never better than Eckart-Young (Eq. ey)
    assert err >= eckart_young_error(synth.sigma_profile("type2", 200), k) * (1 - 1e-9)


@pytest.mark.parametrize("v", [2, 3])
def test_exact_rank_k_reconstruction(v):
    A = synth.rank_k_matrix_np(2000, 1500, 20, seed=4)
    p, q, L, U = powerlu(A, 20, 25, v, seed=0)
    assert rel_lu_error(A, p, q, L, U) <= 1e-13


def test_powerlu_reaches_optimum_on_config_sizes():
    """Plain FP64 workload (2000 x 1500, sigma = 1/i^2, k=20, l=25, v=2): the
    error lies between the Eckart-Young optimum 5.98e-3 and the expected
    Frobenius error of a sketch with no power step, sqrt(1 + k/(q-1)) times
    the optimum (q = l - k), with 20% slack for a single draw."""
    w = synth.PLAIN_2000x1500
    A = w.build("cpu")
    p, q, L, U = powerlu(A, w.k, w.l, w.v, seed=0)
    err = rel_lu_error(A, p, q, L, U)
    opt = eckart_young_error(w.sigma_values(), w.k)
    assert abs(opt - 5.98e-3) < 5e-5
    q = w.l - w.k
    assert opt * (1 - 1e-9) <= err < 1.2 * math.sqrt(1 + w.k / (q - 1)) * opt


def test_theorem_randlu_powerlu_same_range(type2A):
    """Thm. acc:t: with k = l, the same Omega and exact arithmetic,
    Range(P_r^T L_r) = Range(P_p^T L_p) for RandLU(p) and PowerLU(v = 2p+1)."""
    A = type2A
    l = 12
    for p in (1, 2):
        pr, qr_, Lr, Ur = randlu(A, l, l, p, seed=6)
        pp, qp, Lp, Up = powerlu(A, l, l, 2 * p + 1, seed=6)
        Xr = np.empty_like(Lr)
        Xr[pr] = Lr
        Xp = np.empty_like(Lp)
        Xp[pp] = Lp
        assert max_principal_sine(Xr, Xp) < 1e-10


def _bound(sig, k, q, e):
    """Thm. approxlu / approxlu2 with exponent e = 2p (odd v) or 2p+1 (even v);
    reading: [(1 + sqrt(k/(q-1))) s_{k+1}^e + e sqrt(k+q)/q (sum_{j>k} s_j^{2e})^{1/2}]^{1/e}."""
    t1 = (1 + math.sqrt(k / (q - 1))) * sig[k] ** e
    t2 = math.e * math.sqrt(k + q) / q * math.sqrt(np.sum(sig[k:] ** (2 * e)))
    return (t1 + t2) ** (1.0 / e)


@pytest.mark.parametrize("v", [3, 4])
def test_expected_error_bound(v):
    """Thms. approxlu (odd v) and approxlu2 (even v): mean over 20 draws of
    ||A - A V V^T||_2 stays below the bound."""
    sig = synth.sigma_profile("type1", 120)
    A = synth.svd_matrix_np(150, 120, sig, seed=2)
    k, q = 8, 4
    p = (v - 1) // 2
    e = 2 * p if v % 2 else 2 * p + 1
    errs = []
    for s in range(20):
        V = gpowerlu(A, k + q, v, seed=100 + s)
        errs.append(np.linalg.norm(A - A @ V @ V.T, 2))
    assert np.mean(errs) <= _bound(sig, k, q, e)
    assert np.min(errs) >= sig[k + q] * (1 - 1e-9)


def test_singlepass_identities():
    """Alg. singlepasslu: H = A A^T Omega; the column-streaming sweep of
    Sec. 5 gives the same G and H; and in exact arithmetic
    L U = P (A P_G) Q^T with P_G the orthogonal projector onto range(G),
    G = A^T Omega (from P H = L1 U1, G^{T dagger} = G (G^T G)^-1 and
    Q G^{T dagger} U1^T = L2 U2), so the error is ||A - A P_G||_F."""
    sig = synth.sigma_profile("type2", 200)
    A = synth.svd_matrix_np(300, 200, sig, seed=8)
    k = 15
    Om = gaussian_matrix(300, k, 4, STREAM_OMEGA_SP)
    G, H = singlepass_streamed_GH(A, Om)
    assert np.max(np.abs(G - A.T @ Om)) < 1e-12
    assert np.max(np.abs(H - A @ (A.T @ Om))) < 1e-12
    Ac = PassCounter(A)
    p, q, L, U = singlepass(Ac, k, seed=4)
    assert Ac.passes == 1
    assert _is_perm(p, 300) and _is_perm(q, 200)
    assert np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.tril(U, -1), 0.0)
    assert np.allclose(np.diag(U), 1.0) and np.max(np.abs(U)) <= 1.0 + 1e-15
    Qg, _ = np.linalg.qr(A.T @ Om)
    APG = A @ Qg @ Qg.T
    nrm = np.linalg.norm(A)
    assert np.linalg.norm(APG[p][:, q] - L @ U) <= 1e-12 * nrm
    err = rel_lu_error(A, p, q, L, U)
    assert abs(err - np.linalg.norm(A - APG) / nrm) <= 1e-10
    assert err >= eckart_young_error(sig, k) * (1 - 1e-9)
