"""GPU parity of the sparse path (the sprand experiment of Sec. 6) against
the oracle through the C ABI: plu_spmm element by element (CSR-order sums:
within a few ulps of the row's absolute sum), PowerLU and PowerLU_FP on a
sparse A with identical pivots and factors within 1e-10, the out-of-range
index status, and sampled rows of a full-size 32000 x 32000 product."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2002_07138_gb300 as plu

pytestmark = pytest.mark.gpu


def dev(X):
    X = np.asarray(X, dtype=np.float64)
    out = plu.colmajor_empty(X.shape[0], X.shape[1])
    out.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return out


def host(T):
    return T.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_device(m, n, rp, ci, val):
    trp, tci, tval = synth.csr_transpose(m, n, rp, ci, val)
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rp, ci, val, trp, tci, tval)]
    return plu.CsrMatrix(m, n, *t)


def check_spmm(ctx, m, n, rp, ci, val, cols, seed):
    S = to_device(m, n, rp, ci, val)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, cols))
    Z = rng.standard_normal((m, cols))
    Y = host(plu.plu_spmm(ctx, S, 0, dev(X)))
    T = host(plu.plu_spmm(ctx, S, 1, dev(Z)))
    # bound of the rounding: sum |a| |x| over the row, times a few ulps
    aval = np.abs(val)
    bY = oracle.csr_mul(m, rp, ci, aval, np.abs(X))
    bT = oracle.csr_tmul(n, rp, ci, aval, np.abs(Z))
    eY = np.abs(Y - oracle.csr_mul(m, rp, ci, val, X))
    eT = np.abs(T - oracle.csr_tmul(n, rp, ci, val, Z))
    rows_nnz = np.diff(rp)[:, None] + 1
    cols_nnz = np.bincount(ci, minlength=n)[:, None] + 1
    assert np.all(eY <= 2.3e-16 * rows_nnz * bY), float(np.max(eY / (bY + 1e-300)))
    assert np.all(eT <= 2.3e-16 * cols_nnz * bT), float(np.max(eT / (bT + 1e-300)))


@pytest.mark.parametrize("m,n,density,cols", [
    (3000, 2500, 0.003, 200),       # several CTAs, ragged last CTA, sprand density
    (1000, 777, 0.02, 300),         # two column chunks, the second ragged
    (777, 1000, 0.02, 257),         # odd width: padded row-major copy
    (64, 96, 0.1, 1),               # one column
    (33, 4000, 0.05, 64),           # many nonzeros per row, 33 rows
])
def test_spmm_parity(ctx, m, n, density, cols):
    rp, ci, val = synth.sprand_csr(m, n, density, seed=m ^ n)
    check_spmm(ctx, m, n, rp, ci, val, cols, seed=cols)


def test_spmm_empty_rows_and_unsorted_columns(ctx):
    m, n = 500, 420
    rp, ci, val = synth.sprand_csr(m, n, 0.004, seed=3)
    assert np.any(np.diff(rp) == 0)                      # empty rows present
    rng = np.random.default_rng(1)
    ci, val = ci.copy(), val.copy()
    for i in range(m):
        s, e = rp[i], rp[i + 1]
        perm = rng.permutation(e - s) + s
        ci[s:e], val[s:e] = ci[perm], val[perm]
    check_spmm(ctx, m, n, rp, ci, val, 40, seed=2)


def test_spmm_zero_matrix(ctx):
    m, n = 70, 50
    S = to_device(m, n, np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    Y = plu.plu_spmm(ctx, S, 0, dev(np.ones((n, 9))))
    T = plu.plu_spmm(ctx, S, 1, dev(np.ones((m, 9))))
    assert torch.all(Y == 0) and torch.all(T == 0)


def test_spmm_bad_index_reports_and_context_survives(ctx):
    """A column index outside [0, n) or a row pointer beyond nnz is skipped
    by the kernel's own checks and reported as PLU_EINDEX."""
    m, n = 200, 150
    rp, ci, val = synth.sprand_csr(m, n, 0.05, seed=5)
    bad = ci.copy()
    bad[7] = n + 5
    bad[11] = -1
    trp, tci, tval = synth.csr_transpose(m, n, rp, ci, val)
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
         for a in (rp, bad, val, trp, tci, tval)]
    S = plu.CsrMatrix(m, n, *t)
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_spmm(ctx, S, 0, dev(np.ones((n, 4))))
    assert ei.value.name == "PLU_EINDEX"
    rp2 = rp.copy()
    rp2[m] = rp[m] + 1000                                 # last row runs past nnz
    t2 = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
          for a in (rp2, ci, val, trp, tci, tval)]
    with pytest.raises(plu.PLUError) as ei:
        plu.plu_spmm(ctx, plu.CsrMatrix(m, n, *t2), 0, dev(np.ones((n, 4))))
    assert ei.value.name == "PLU_EINDEX"
    # the context is usable and the status cleared
    check_spmm(ctx, m, n, rp, ci, val, 8, seed=1)


@pytest.mark.parametrize("v", [2, 3, 4])
def test_powerlu_csr_parity(ctx, v):
    """3000 x 2500 sprand at 0.3% density, k = 20, l = 25."""
    m, n, k, l = 3000, 2500, 20, 25
    rp, ci, val = synth.sprand_csr(m, n, 0.003, seed=20 + v)
    ref = oracle.powerlu(oracle.SparsePassCounter(m, n, rp, ci, val), k, l, v, seed=0)
    gp, gq, gL, gU, rep = plu.plu_powerlu_csr(ctx, to_device(m, n, rp, ci, val), k, l, v, seed=0)
    assert np.array_equal(gp.cpu().numpy(), ref[0])
    assert np.array_equal(gq.cpu().numpy(), ref[1])
    assert rel(host(gL), ref[2]) < 1e-10
    assert rel(host(gU), ref[3]) < 1e-10
    assert rep["passes"] == v
    assert rep["flops_passes"] == pytest.approx(2.0 * rp[-1] * (l * (v - 1) + k))


@pytest.mark.parametrize("v", [2, 3])
def test_powerlu_csr_exact_rank(ctx, v):
    m, n, r = 1200, 900, 7
    A = synth.sparse_rank_r(m, n, r, seed=31)
    rp, ci, val = synth.dense_to_csr(A)
    gp, gq, gL, gU, _ = plu.plu_powerlu_csr(ctx, to_device(m, n, rp, ci, val), r, r + 5, v,
                                             seed=3)
    err = oracle.rel_lu_error(A, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert err < 1e-12


def test_powerlu_fp_csr_parity(ctx):
    m, n, r = 1500, 1100, 9
    A = synth.sparse_rank_r(m, n, r, seed=41)
    A += synth.csr_to_dense(m, n, *synth.sprand_csr(m, n, 0.003, seed=42)) * 1e-9
    rp, ci, val = synth.dense_to_csr(A)
    S = oracle.SparsePassCounter(m, n, rp, ci, val)
    # b = 1: the rank stops at r, before the noise-level columns
    k, p, q, L, U, E, met = oracle.powerlu_fp(S, 1e-6, 1, 40, 3, seed=5)
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp_csr(ctx, to_device(m, n, rp, ci, val),
                                                           1e-6, 1, 40, 3, seed=5)
    assert gk == k == r and gmet and met
    assert np.array_equal(gp.cpu().numpy(), p) and np.array_equal(gq.cpu().numpy(), q)
    assert rel(host(gL), L) < 1e-10 and rel(host(gU), U) < 1e-10
    assert rep["normA2"] == pytest.approx(S.frob2(), rel=1e-13)


def test_powerlu_fp_csr_restart_parity(ctx):
    """Two restart rounds on a sprand A whose tolerance l columns cannot meet."""
    m, n = 1400, 1000
    rp, ci, val = synth.sprand_csr(m, n, 0.01, seed=50)
    S = oracle.SparsePassCounter(m, n, rp, ci, val)
    k, p, q, L, U, E, met = oracle.powerlu_fp(S, 0.05, 4, 16, 3, seed=6, max_rounds=2)
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp_csr(
        ctx, to_device(m, n, rp, ci, val), 0.05, 4, 16, 3, seed=6, max_rounds=2)
    assert gk == k == 32 and not met and not gmet
    assert np.array_equal(gp.cpu().numpy(), p) and np.array_equal(gq.cpu().numpy(), q)
    assert rel(host(gL), L) < 1e-10 and rel(host(gU), U) < 1e-10


@pytest.fixture(scope="module")
def full_sprand():
    n = 32000
    rp, ci, val = synth.sprand_csr(n, n, 0.003, seed=0)
    return n, rp, ci, val


def test_spmm_full_size_sampled(ctx, full_sprand):
    """The 32000 x 32000 sprand matrix at 0.3% density with l = 200 columns,
    as the bench runs it: 300 sampled rows of A X and of A^T X against the
    oracle's definition."""
    n, rp, ci, val = full_sprand
    S = to_device(n, n, rp, ci, val)
    X = torch.randn(n, 200, dtype=torch.float64, generator=torch.Generator().manual_seed(3))
    Xd = plu.colmajor_empty(n, 200)
    Xd.copy_(X)
    Xh = X.numpy()
    sel = np.random.default_rng(4).choice(n, 300, replace=False)
    sel[0], sel[1] = 0, n - 1
    for trans in (0, 1):
        Y = host(plu.plu_spmm(ctx, S, trans, Xd))[sel]
        f = oracle.csr_tmul if trans else oracle.csr_mul
        ref = f(n, rp, ci, val, Xh, rows=sel)
        bound = f(n, rp, ci, np.abs(val), np.abs(Xh), rows=sel)
        assert np.all(np.abs(Y - ref) <= 2.3e-16 * 200 * bound)


def sparse_rel_error(m, rp, ci, val, p, q, L, U):
    """||A - P^T L U Q||_F / ||A||_F for a sparse A without forming L U:
    ||A||^2 is the sum of the squared values, <A, P^T L U Q> a k-length dot
    product per nonzero (row pinv[i] of L, column qinv[j] of U), and
    ||L U||^2 = trace((L^T L)(U U^T)).  CUDA tensors; rp, ci, val the CSR."""
    dev = L.device
    rpt = torch.as_tensor(rp, device=dev)
    cit = torch.as_tensor(ci, device=dev).long()
    vt = torch.as_tensor(val, device=dev)
    pinv = torch.empty_like(p.long())
    pinv[p.long()] = torch.arange(m, device=dev)
    qinv = torch.empty_like(q.long())
    qinv[q.long()] = torch.arange(q.numel(), device=dev)
    rows = torch.repeat_interleave(torch.arange(m, device=dev), rpt[1:] - rpt[:-1])
    normA2 = float((vt * vt).sum())
    inner = 0.0
    step = 1 << 19
    for s0 in range(0, vt.numel(), step):
        r = pinv[rows[s0:s0 + step]]
        c = qinv[cit[s0:s0 + step]]
        inner += float((vt[s0:s0 + step] * (L[r] * U[:, c].t()).sum(1)).sum())
    normLU2 = float(((L.t() @ L) * (U @ U.t())).sum())
    return max(normA2 - 2.0 * inner + normLU2, 0.0) ** 0.5 / normA2 ** 0.5


def test_powerlu_csr_full_size(ctx, full_sprand):
    """PowerLU on the full-size sprand A (k = l = 200, v = 4): valid
    permutations, finite factors, 4 passes, and the relative error (formed
    from the nonzeros) equal to that of the dense FP64 path on the same
    matrix, whose pivots it shares."""
    n, rp, ci, val = full_sprand
    S = to_device(n, n, rp, ci, val)
    k = l = 200
    gp, gq, gL, gU, rep = plu.plu_powerlu_csr(ctx, S, k, l, 4, seed=0)
    p, q = gp.cpu().numpy(), gq.cpu().numpy()
    assert np.array_equal(np.sort(p), np.arange(n)) and np.array_equal(np.sort(q), np.arange(n))
    assert torch.isfinite(gL).all() and torch.isfinite(gU).all()
    assert rep["passes"] == 4
    err = sparse_rel_error(n, rp, ci, val, gp, gq, gL, gU)
    # the same algorithm with dense FP64 passes over the densified A
    Ad = plu.colmajor_empty(n, n)
    Ad.zero_()
    rows = torch.repeat_interleave(torch.arange(n), torch.from_numpy(np.diff(rp)))
    Ad.index_put_((rows.cuda(), torch.from_numpy(ci).long().cuda()), torch.from_numpy(val).cuda())
    dp, dq, dL, dU, _ = plu.plu_powerlu(ctx, Ad, k, l, 4, seed=0, prec="fp64")
    del Ad
    torch.cuda.empty_cache()
    assert np.array_equal(dp.cpu().numpy(), p) and np.array_equal(dq.cpu().numpy(), q)
    err_dense = sparse_rel_error(n, rp, ci, val, dp, dq, dL, dU)
    assert 0.0 < err < 1.0
    assert abs(err - err_dense) <= 1e-9 * err_dense
