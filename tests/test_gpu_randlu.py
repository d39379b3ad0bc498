"""GPU parity of RandLU with power iteration (Alg. rlu with
Alg. basicpoweriteration, the comparison method of the paper) against the
FP64 oracle on the same seeded inputs and the same Philox sketch: FP64 path
-> identical p and q, L and U within 1e-9 relative; TF32 passes -> error
within 1.1x of the FP64 path's."""
import math

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def lu_err(A, res):
    gp, gq, gL, gU = res[:4]
    return oracle.rel_lu_error(A, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))


@pytest.fixture(scope="module")
def plain_case():
    w = synth.PLAIN_2000x1500
    return w, w.build("cpu")


@pytest.mark.parametrize("piter", [0, 1, 2])
def test_randlu_fp64_parity_plain_config(ctx, plain_case, piter):
    """2000 x 1500, sigma_i = 1/i^2, k = 20, l = 25: the oracle's pivots
    exactly, L and U within 1e-9; 2 piter + 2 passes."""
    w, A = plain_case
    p, q, L, U = oracle.randlu(A, w.k, w.l, piter, seed=0)
    gp, gq, gL, gU, rep = plu.plu_randlu(ctx, dev(A), w.k, w.l, piter, seed=0, prec="fp64")
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), np.asarray(p))
    assert np.array_equal(gq.cpu().numpy().astype(np.int64), np.asarray(q))
    assert rel(host(gL), L) < 1e-9
    assert rel(host(gU), U) < 1e-9
    assert rep["passes"] == 2 * piter + 2
    err = lu_err(A, (gp, gq, gL, gU))
    assert err >= oracle.eckart_young_error(w.sigma_values(), w.k) * (1 - 1e-9)
    assert abs(err - oracle.rel_lu_error(A, p, q, L, U)) <= 1e-9 * err + 1e-15


@pytest.mark.parametrize("m,n,k,l,piter", [(1000, 700, 13, 20, 1), (700, 1000, 31, 40, 2),
                                           (517, 517, 64, 70, 0), (3000, 257, 5, 6, 1)])
def test_randlu_fp64_ragged_shapes(ctx, m, n, k, l, piter):
    sig = synth.sigma_profile("type2", min(m, n))
    A = synth.svd_matrix_np(m, n, sig, seed=m + n)
    p, q, L, U = oracle.randlu(A, k, l, piter, seed=3)
    gp, gq, gL, gU, _ = plu.plu_randlu(ctx, dev(A), k, l, piter, seed=3, prec="fp64")
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), np.asarray(p))
    assert np.array_equal(gq.cpu().numpy().astype(np.int64), np.asarray(q))
    assert rel(host(gL), L) < 1e-9
    assert rel(host(gU), U) < 1e-9


def test_randlu_structure(ctx, plain_case):
    """U = L'^T is unit upper triangular with |u_ij| <= 1; p, q permutations."""
    w, A = plain_case
    gp, gq, gL, gU, _ = plu.plu_randlu(ctx, dev(A), w.k, w.l, 1, seed=5)
    U = host(gU)
    assert np.allclose(np.diag(U[:, :w.k]), 1.0)
    assert np.all(np.abs(np.tril(U[:, :w.k], -1)) == 0.0)
    assert np.max(np.abs(U)) <= 1.0 + 1e-12
    assert sorted(gp.cpu().tolist()) == list(range(A.shape[0]))
    assert sorted(gq.cpu().tolist()) == list(range(A.shape[1]))


def test_randlu_exact_rank_k(ctx):
    A = synth.rank_k_matrix_np(2000, 1500, 20, seed=4)
    for piter in (0, 1):
        res = plu.plu_randlu(ctx, dev(A), 20, 25, piter, seed=0)
        assert lu_err(A, res) <= 1e-13


def test_randlu_tf32_error_within_1p1_of_fp64(ctx):
    sig = synth.sigma_profile("exp20", 2048)
    A = synth.svd_matrix_np(2048, 2048, sig, seed=1, noise=1e-6 / math.sqrt(2048))
    e64 = lu_err(A, plu.plu_randlu(ctx, dev(A), 100, 110, 1, seed=2, prec="fp64"))
    res = plu.plu_randlu(ctx, dev(A, torch.float32), 100, 110, 1, seed=2, prec="tf32")
    assert lu_err(A, res) <= 1.1 * e64


def test_randlu_rejects_bad_arguments(ctx):
    A = dev(np.random.default_rng(0).standard_normal((64, 48)))
    with pytest.raises(plu.PLUError):
        plu.plu_randlu(ctx, A, 10, 8, 1)            # k > l
    with pytest.raises(plu.PLUError):
        plu.plu_randlu(ctx, A, 4, 8, -1)            # piter < 0
    with pytest.raises(plu.PLUError):
        plu.plu_randlu(ctx, A, 4, 48, 0)            # l >= min(m, n)
