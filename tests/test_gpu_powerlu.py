"""GPU parity of the whole algorithms (PowerLU fixed rank, PowerLU_FP fixed
precision) against the FP64 oracle on the same seeded inputs and the same
Philox sketch: FP64 path -> identical p and q, L and U within 1e-10
relative (Frobenius, per factor); FP32 passes -> error within 1.1x of FP64."""
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


def check_parity(A, got, ref, tol=1e-10):
    gp, gq, gL, gU = got
    p, q, L, U = ref
    assert np.array_equal(gp.cpu().numpy().astype(np.int64), np.asarray(p))
    assert np.array_equal(gq.cpu().numpy().astype(np.int64), np.asarray(q))
    assert rel(host(gL), L) < tol
    assert rel(host(gU), U) < tol


@pytest.fixture(scope="module")
def plain_case():
    w = synth.PLAIN_2000x1500
    return w, w.build("cpu")


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_powerlu_fp64_plain_config(ctx, plain_case, v):
    """2000 x 1500, sigma_i = 1/i^2, k = 20, l = 25, seed 0."""
    w, A = plain_case
    ref = oracle.powerlu(A, w.k, w.l, v, seed=0)
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A), w.k, w.l, v, seed=0, prec="fp64")
    check_parity(A, (gp, gq, gL, gU), ref)
    assert rep["passes"] == v
    err = oracle.rel_lu_error(A, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert err >= oracle.eckart_young_error(w.sigma_values(), w.k) * (1 - 1e-9)


@pytest.mark.parametrize("m,n,k,l,v", [(1000, 700, 13, 20, 3), (700, 1000, 31, 40, 4),
                                       (517, 517, 64, 70, 2), (3000, 257, 5, 6, 5)])
def test_powerlu_fp64_ragged_shapes(ctx, m, n, k, l, v):
    sig = synth.sigma_profile("type2", min(m, n))
    A = synth.svd_matrix_np(m, n, sig, seed=m + n)
    ref = oracle.powerlu(A, k, l, v, seed=3)
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A), k, l, v, seed=3, prec="fp64")
    check_parity(A, (gp, gq, gL, gU), ref)


def test_powerlu_exact_rank_k(ctx):
    A = synth.rank_k_matrix_np(2000, 1500, 20, seed=4)
    for v in (2, 3):
        gp, gq, gL, gU, _ = plu.plu_powerlu(ctx, dev(A), 20, 25, v, seed=0)
        err = oracle.rel_lu_error(A, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
        assert err <= 1e-13


def test_powerlu_fp32_passes_error_within_1p1_of_fp64(ctx):
    sig = synth.sigma_profile("exp20", 2048)
    A = synth.svd_matrix_np(2048, 2048, sig, seed=1, noise=1e-6 / math.sqrt(2048))
    A32 = dev(A.astype(np.float32), torch.float32)
    A64h = A.astype(np.float32).astype(np.float64)
    errs = {}
    for prec, Ad in (("fp64", dev(A64h)), ("fp32", A32)):
        gp, gq, gL, gU, _ = plu.plu_powerlu(ctx, Ad, 100, 110, 3, seed=0, prec=prec)
        errs[prec] = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert errs["fp32"] <= 1.1 * errs["fp64"]


@pytest.mark.parametrize("precise", [False, True])
def test_powerlu_fp_parity(ctx, precise):
    sig = synth.sigma_profile("type2", 800)
    A = synth.svd_matrix_np(1000, 800, sig, seed=12)
    eps, b, l, v = 1e-4, 10, 120, 4
    k, p, q, L, U, E, met = oracle.powerlu_fp(A, eps, b, l, v, seed=2, precise=precise)
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, dev(A), eps, b, l, v, seed=2,
                                                       prec="fp64", precise=precise)
    assert (gk, gmet) == (k, met)
    check_parity(A, (gp, gq, gL, gU), (p, q, L, U))
    nA2 = float(np.sum(A * A))
    assert abs(rep["normA2"] - nA2) <= 1e-12 * nA2
    assert abs(rep["indicator"] - math.sqrt(max(E, 0) / nA2)) <= 1e-8
    # ||A||_F^2 comes from the first pass: A is read exactly v times
    assert rep["passes"] == v


@pytest.mark.parametrize("v,precise", [(3, False), (4, True)])
def test_powerlu_fp_restart_parity(ctx, v, precise):
    """The restart of the Remark after Alg. adaptivewithoutupdating: l too
    small for eps, later rounds on the remainder A - A W W^T reach it.  FP64
    path: the same rank, rounds, pivots and factors as the oracle."""
    sig = 1.0 / np.arange(1, 601)
    A = synth.svd_matrix_np(900, 600, sig, seed=31)
    eps, b, l, rounds = 0.06, 8, 40, 6
    k, p, q, L, U, E, met = oracle.powerlu_fp(A, eps, b, l, v, seed=5, precise=precise,
                                              max_rounds=rounds)
    assert met and k > l
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, dev(A), eps, b, l, v, seed=5,
                                                       prec="fp64", precise=precise,
                                                       max_rounds=rounds)
    assert (gk, gmet) == (k, met)
    assert rep["rounds"] >= 2 and rep["passes"] == rep["rounds"] * v
    check_parity(A, (gp, gq, gL, gU), (p, q, L, U), tol=1e-9)
    assert oracle.rel_lu_error(A, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU)) <= eps
    nA2 = float(np.sum(A * A))
    assert abs(rep["indicator"] - math.sqrt(max(E, 0) / nA2)) <= 1e-8


def test_powerlu_fp_restart_tf32_meets_tolerance(ctx):
    """The restart in the TF32 mode: same rank as FP64, error within eps and
    within 1.1x of the FP64 path."""
    sig = 1.0 / np.arange(1, 1025)
    A = synth.svd_matrix_np(2048, 1024, sig, seed=32)
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    eps, b, l, v, rounds = 0.05, 16, 96, 3, 6
    res = {}
    for prec, Ad in (("fp64", dev(A64h)), ("tf32", dev(A32, torch.float32))):
        gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, Ad, eps, b, l, v, seed=7,
                                                           prec=prec, max_rounds=rounds)
        assert gmet and rep["rounds"] >= 2
        res[prec] = (gk, oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(),
                                             host(gL), host(gU)))
    assert res["tf32"][0] == res["fp64"][0]
    assert res["tf32"][1] <= eps and res["tf32"][1] <= 1.1 * res["fp64"][1]


def test_powerlu_fp_tolerance_not_met(ctx):
    sig = synth.sigma_profile("type1", 300)
    A = synth.svd_matrix_np(400, 300, sig, seed=3)
    k, p, q, L, U, E, met = oracle.powerlu_fp(A, 1e-9, 7, 30, 3, seed=2)
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, dev(A), 1e-9, 7, 30, 3, seed=2)
    assert not met and not gmet and gk == k == 30
    check_parity(A, (gp, gq, gL, gU), (p, q, L, U))


def test_fixed_rank_8192_fp64_full_parity(ctx):
    """The 8192 x 8192 fixed-rank workload (sigma_i = exp(-i/20) plus a
    1e-6 N(0,1)/sqrt(n) floor, k = 100, l = 110) in FP64 at v = 3."""
    w = synth.FIXED_RANK_8192
    Ad = w.build("cuda").double()
    Ad = synth.colmajor(Ad)
    A = Ad.cpu().numpy()
    ref = oracle.powerlu(A, w.k, w.l, 3, seed=0)
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, Ad, w.k, w.l, 3, seed=0, prec="fp64")
    check_parity(A, (gp, gq, gL, gU), ref)
    err = oracle.rel_lu_error(A, ref[0], ref[1], ref[2], ref[3])
    opt = oracle.eckart_young_error(w.sigma_values(), w.k)
    assert opt * (1 - 1e-9) <= err < 2.0 * opt


def test_powerlu_tf32_error_within_1p1_of_fp64(ctx):
    """Mixed precision: TF32 tensor-core passes, FP64 everything else."""
    sig = synth.sigma_profile("pow15", 4096)
    A = synth.svd_matrix_np(4096, 4096, sig, seed=2)
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    errs = {}
    for prec, Ad in (("fp64", dev(A64h)), ("tf32", dev(A32, torch.float32))):
        gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, Ad, 64, 74, 3, seed=0, prec=prec)
        errs[prec] = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
        assert rep["passes"] == 3
    assert errs["tf32"] <= 1.1 * errs["fp64"], errs


@pytest.mark.parametrize("v", [2, 4])
@pytest.mark.parametrize("prec,limit", [("tf32", 1.1), ("bf16", 1.5)])
def test_powerlu_mixed_even_pass_counts(ctx, v, prec, limit):
    """Even v (Alg. gpowerlu starts from A^T Omega, Omega m x l): v passes in
    the mixed modes, error bounded against the FP64 path at the same v."""
    sig = synth.sigma_profile("pow15", 2048)
    A = synth.svd_matrix_np(2048, 1536, sig[:1536], seed=8)
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A64h), 48, 58, v, seed=3, prec="fp64")
    assert rep["passes"] == v
    e64 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A32, torch.float32), 48, 58, v, seed=3, prec=prec)
    assert rep["passes"] == v
    e = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert e <= limit * e64, (e, e64)


@pytest.mark.parametrize("prec,limit", [("bf16", 1.5), ("fp8", 6.0)])
def test_powerlu_quantized_passes_run_and_report_error(ctx, prec, limit):
    """BF16 / FP8-E4M3 power passes over a quantized copy of A, final pass on
    the FP32 A: v passes, valid factors, error bounded against FP64."""
    sig = synth.sigma_profile("pow15", 2048)
    A = synth.svd_matrix_np(2048, 2048, sig, seed=3)
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A64h), 64, 74, 3, seed=0, prec="fp64")
    e64 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    gp, gq, gL, gU, rep = plu.plu_powerlu(ctx, dev(A32, torch.float32), 64, 74, 3, seed=0, prec=prec)
    assert rep["passes"] == 3
    p, q = gp.cpu().numpy(), gq.cpu().numpy()
    assert sorted(p.tolist()) == list(range(2048)) and sorted(q.tolist()) == list(range(2048))
    e = oracle.rel_lu_error(A64h, p, q, host(gL), host(gU))
    assert e <= limit * e64, (e, e64)


@pytest.mark.parametrize("m,n,k", [(1000, 800, 12), (3000, 2500, 40)])
def test_singlepass_fp64_parity(ctx, m, n, k):
    """Alg. singlepasslu on the same Omega: identical p, q; L, U to 1e-9
    (G^{dagger T} goes through CholeskyQR2 of G instead of (G^T G)^{-1})."""
    sig = synth.sigma_profile("type2", min(m, n))
    A = synth.svd_matrix_np(m, n, sig, seed=m)
    ref = oracle.singlepass(A, k, seed=5)
    gp, gq, gL, gU, rep = plu.plu_singlepass(ctx, dev(A), k, seed=5, prec="fp64")
    assert rep["passes"] == 1
    check_parity(A, (gp, gq, gL, gU), ref, tol=1e-9)


def test_singlepass_streams_column_panels_and_tf32(ctx):
    """Wide enough that the column sweep takes several L2-sized panels; TF32
    error within 1.25x of the FP64 single pass (the single pass has no
    re-orthogonalising step, so TF32 rounding enters G and H directly)."""
    sig = synth.sigma_profile("type1", 3000)
    A = synth.svd_matrix_np(6000, 3000, sig, seed=7)      # 6000 x 8 B x 1024 cols = 49 MB
    A32 = A.astype(np.float32)
    A64h = A32.astype(np.float64)
    ref = oracle.singlepass(A64h, 30, seed=1)
    gp, gq, gL, gU, _ = plu.plu_singlepass(ctx, dev(A64h), 30, seed=1, prec="fp64")
    check_parity(A64h, (gp, gq, gL, gU), ref, tol=1e-9)
    e64 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    gp, gq, gL, gU, _ = plu.plu_singlepass(ctx, dev(A32, torch.float32), 30, seed=1, prec="tf32")
    e32 = oracle.rel_lu_error(A64h, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    assert e32 <= 1.25 * e64, (e32, e64)   # no re-orthogonalisation: TF32 enters G and H directly


def _batch_cases():
    rng = np.random.default_rng(3)
    cases = []
    for i in range(14):
        m = int(rng.integers(150, 900))
        n = int(rng.integers(100, m + 1))
        k = int(rng.integers(4, 20))
        algo = 1 if i % 5 == 4 else 0
        cases.append(dict(m=m, n=n, k=k, l=k + 6, v=2 + (i % 3), algo=algo, seed=100 + i))
    return cases


def test_batched_fp64_matches_oracle_per_problem(ctx):
    """One graph launch over a mixed batch (PowerLU v = 2..4 and single pass,
    uneven shapes): every problem matches the oracle -- identical pivots,
    factors to 1e-9."""
    cases = _batch_cases()
    mats = []
    probs = []
    for c in cases:
        sig = synth.sigma_profile("expk", min(c["m"], c["n"]), k=c["k"])
        A = synth.svd_matrix_np(c["m"], c["n"], sig, seed=c["seed"])
        mats.append(A)
        probs.append(dict(A=dev(A), k=c["k"], l=c["l"], v=c["v"], algo=c["algo"], seed=c["seed"]))
    outs, rep = plu.plu_batched(ctx, probs, prec="fp64")
    assert rep["launches"] > 0
    for c, A, (gp, gq, gL, gU) in zip(cases, mats, outs):
        if c["algo"] == 1:
            ref = oracle.singlepass(A, c["k"], seed=c["seed"])
        else:
            ref = oracle.powerlu(A, c["k"], c["l"], c["v"], seed=c["seed"])
        check_parity(A, (gp, gq, gL, gU), ref, tol=1e-9)


@pytest.mark.parametrize("bm,bn", [(64, 32), (64, 64), (128, 32)])
def test_batched_each_gemm_tile_shape_matches_oracle(ctx, bm, bn):
    """Every grouped-GEMM tile shape the autotuner can pick, forced for the
    whole batch: identical pivots and factors to 1e-9 against the oracle."""
    cases = _batch_cases()[:7]
    mats, probs = [], []
    for c in cases:
        sig = synth.sigma_profile("expk", min(c["m"], c["n"]), k=c["k"])
        A = synth.svd_matrix_np(c["m"], c["n"], sig, seed=c["seed"])
        mats.append(A)
        probs.append(dict(A=dev(A), k=c["k"], l=c["l"], v=c["v"], algo=c["algo"], seed=c["seed"]))
    plu.plu_set_batched_tile(ctx, bm, bn)
    try:
        outs, _ = plu.plu_batched(ctx, probs, prec="fp64")
        assert set(plu.plu_batched_tiles(ctx)) == {(bm, bn)}
    finally:
        plu.plu_set_batched_tile(ctx, 0, 0)
    for c, A, (gp, gq, gL, gU) in zip(cases, mats, outs):
        if c["algo"] == 1:
            ref = oracle.singlepass(A, c["k"], seed=c["seed"])
        else:
            ref = oracle.powerlu(A, c["k"], c["l"], c["v"], seed=c["seed"])
        check_parity(A, (gp, gq, gL, gU), ref, tol=1e-9)


def test_batched_autotuner_choice_is_cached_and_valid(ctx):
    """The first call of a batch signature times the tile shapes; a second
    call reuses the same choice; every chosen shape is one the library has;
    a shape it does not have is refused."""
    cases = _batch_cases()[7:]
    probs = []
    for c in cases:
        A = synth.svd_matrix_np(c["m"], c["n"], synth.sigma_profile("type2", min(c["m"], c["n"])),
                                seed=c["seed"])
        probs.append(dict(A=dev(A.astype(np.float32), torch.float32), k=c["k"], l=c["l"], v=c["v"],
                          algo=c["algo"], seed=c["seed"]))
    plu.plu_batched(ctx, probs, prec="fp32")
    first = plu.plu_batched_tiles(ctx)
    plu.plu_batched(ctx, probs, prec="fp32")
    assert plu.plu_batched_tiles(ctx) == first
    assert len(first) > 0 and set(first) <= {(64, 32), (64, 64), (128, 32)}
    with pytest.raises(plu.PLUError):
        plu.plu_set_batched_tile(ctx, 48, 48)


def _fp64_batch(cases):
    mats, probs = [], []
    for c in cases:
        sig = synth.sigma_profile("expk", min(c["m"], c["n"]), k=c["k"])
        A = synth.svd_matrix_np(c["m"], c["n"], sig, seed=c["seed"])
        mats.append(A)
        probs.append(dict(A=dev(A), k=c["k"], l=c["l"], v=c["v"], algo=c["algo"], seed=c["seed"]))
    return mats, probs


def test_batched_tune_file_persists_and_split_k_matches_oracle(ctx, tmp_path):
    """The autotuner's choices go to the tuning file; a new context reads them
    back without timing (no line added, same shapes and split-K).  A file
    line that asks every launch for 64 x 32 tiles with K chunks of 256 (the
    split-K reduction in FP64) gives identical pivots and factors to 1e-9
    against the oracle."""
    cases = _batch_cases()[2:]                  # a batch signature no other test uses
    mats, probs = _fp64_batch(cases)
    path = tmp_path / "tune.txt"
    plu.plu_set_batched_tune_file(ctx, str(path))
    try:
        plu.plu_batched(ctx, probs, prec="fp64")
        tiles, splits = plu.plu_batched_tiles(ctx), plu.plu_batched_splitk(ctx)
    finally:
        plu.plu_set_batched_tune_file(ctx, None)
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    head = lines[0].split()
    assert head[:2] == ["plu-batched-tune", "1"] and int(head[3]) == len(tiles) == len(splits)
    assert set(splits) <= {0, 1024, 256}
    c2 = plu.Context(0)
    try:
        plu.plu_set_batched_tune_file(c2, str(path))
        plu.plu_batched(c2, probs, prec="fp64")
        assert plu.plu_batched_tiles(c2) == tiles and plu.plu_batched_splitk(c2) == splits
        assert path.read_text().splitlines() == lines
    finally:
        torch.cuda.synchronize()
        c2.close()
    # every launch: 64 x 32 tiles, K chunks of 256 (choice 0 + 3 * 2)
    forced = " ".join(head[:4] + ["6"] * int(head[3]))
    path.write_text(lines[0] + "\n" + forced + "\n")
    c3 = plu.Context(0)
    try:
        plu.plu_set_batched_tune_file(c3, str(path))
        outs, _ = plu.plu_batched(c3, probs, prec="fp64")
        assert set(plu.plu_batched_splitk(c3)) == {256}
    finally:
        torch.cuda.synchronize()
        c3.close()
    for c, A, (gp, gq, gL, gU) in zip(cases, mats, outs):
        if c["algo"] == 1:
            ref = oracle.singlepass(A, c["k"], seed=c["seed"])
        else:
            ref = oracle.powerlu(A, c["k"], c["l"], c["v"], seed=c["seed"])
        check_parity(A, (gp, gq, gL, gU), ref, tol=1e-9)


def test_batched_large_panels_on_several_ctas_match_oracle(ctx):
    """Panels with more than 1.5e6 FMAs of elimination are factored by groups
    of CTAs that exchange column-step candidates (4096 x 74: 8 CTAs; the
    single-pass and tail LUs of 3000 x 64 and 2500 x 64 too), beside small
    problems factored by one CTA: identical pivots and factors to 1e-9."""
    cases = [dict(m=4096, n=1500, k=64, l=74, v=3, algo=0, seed=41),
             dict(m=3000, n=2500, k=64, l=64, v=1, algo=1, seed=42),
             dict(m=700, n=500, k=12, l=18, v=2, algo=0, seed=43),
             dict(m=2600, n=2600, k=40, l=50, v=4, algo=0, seed=44)]
    mats, probs = _fp64_batch(cases)
    outs, _ = plu.plu_batched(ctx, probs, prec="fp64")
    for c, A, (gp, gq, gL, gU) in zip(cases, mats, outs):
        if c["algo"] == 1:
            ref = oracle.singlepass(A, c["k"], seed=c["seed"])
        else:
            ref = oracle.powerlu(A, c["k"], c["l"], c["v"], seed=c["seed"])
        check_parity(A, (gp, gq, gL, gU), ref, tol=1e-9)


def test_batched_tune_file_must_be_writable(ctx, tmp_path):
    with pytest.raises(plu.PLUError):
        plu.plu_set_batched_tune_file(ctx, str(tmp_path / "no" / "such" / "dir" / "t.txt"))


def test_batched_fp32_error_close_to_fp64(ctx):
    cases = _batch_cases()[:8]
    probs32, probs64, mats = [], [], []
    for c in cases:
        sig = synth.sigma_profile("expk", min(c["m"], c["n"]), k=c["k"])
        A = synth.svd_matrix_np(c["m"], c["n"], sig, seed=c["seed"]).astype(np.float32)
        A64 = A.astype(np.float64)
        mats.append(A64)
        probs32.append(dict(A=dev(A, torch.float32), k=c["k"], l=c["l"], v=c["v"], algo=c["algo"],
                            seed=c["seed"]))
        probs64.append(dict(A=dev(A64), k=c["k"], l=c["l"], v=c["v"], algo=c["algo"],
                            seed=c["seed"]))
    o32, _ = plu.plu_batched(ctx, probs32, prec="fp32")
    o64, _ = plu.plu_batched(ctx, probs64, prec="fp64")
    for A, a, b in zip(mats, o32, o64):
        e32 = oracle.rel_lu_error(A, a[0].cpu().numpy(), a[1].cpu().numpy(), host(a[2]), host(a[3]))
        e64 = oracle.rel_lu_error(A, b[0].cpu().numpy(), b[1].cpu().numpy(), host(b[2]), host(b[3]))
        assert e32 <= 1.1 * e64 + 1e-6, (e32, e64)


def test_fixed_precision_20000x10000_full_size(ctx):
    """The fixed-precision workload at full size: 20000 x 10000 FP32 A,
    sigma_i = 1/i with a 100x gap at i = 400, b = 32, eps = 1e-3, l = 512,
    v = 4.  FP64 path: same rank, pivots and factors as the oracle; TF32 path:
    same rank, error within 1.1x of FP64 and below eps."""
    w = synth.FIXED_PREC_20000x10000
    A32 = w.build("cuda")                                   # FP32, column-major
    A64 = synth.colmajor(A32.double())
    Ah = A64.cpu().numpy()
    k, p, q, L, U, E, met = oracle.powerlu_fp(Ah, w.eps, w.b, w.l, w.v, seed=0)
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, A64, w.eps, w.b, w.l, w.v, seed=0,
                                                       prec="fp64")
    assert met and gmet and gk == k
    check_parity(Ah, (gp, gq, gL, gU), (p, q, L, U), tol=1e-9)
    e64 = oracle.rel_lu_error(Ah, gp.cpu().numpy(), gq.cpu().numpy(), host(gL), host(gU))
    tk, tp, tq, tL, tU, tmet, trep = plu.plu_powerlu_fp(ctx, A32, w.eps, w.b, w.l, w.v, seed=0,
                                                        prec="tf32")
    assert tmet and tk == k
    e32 = oracle.rel_lu_error(Ah, tp.cpu().numpy(), tq.cpu().numpy(), host(tL), host(tU))
    assert e64 <= w.eps and e32 <= 1.1 * e64, (e32, e64)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "fp8", "tf32x3"])
@pytest.mark.parametrize("v", [3, 4])
def test_powerlu_fp_norm_from_first_read(ctx, prec, v):
    """Alg. adaptivewithoutupdating step 1 fused into the first read of A:
    ||A||_F^2 summed by the first pass (A Omega for odd v, A^T Omega for even
    v: both tensor-core orientations, the split passes' splitter and
    transposer warps, the SIMT passes) or by the quantisation
    (BF16, FP8) equals the sum of the squares of the stored entries, and A is
    read exactly v times."""
    m, n = 3001, 2003                      # ragged tiles in both orientations
    A32 = synth.svd_matrix_np(m, n, synth.sigma_profile("type2", n), seed=4).astype(np.float32)
    A32[7, 5] = 3.0e3                      # a large entry among small ones
    gk, gp, gq, gL, gU, gmet, rep = plu.plu_powerlu_fp(ctx, dev(A32, torch.float32), 1e-3, 8, 48,
                                                       v, seed=1, prec=prec)
    nA2 = float(np.sum(A32.astype(np.float64) ** 2))
    assert abs(rep["normA2"] - nA2) <= 1e-12 * nA2
    assert rep["passes"] == v
