"""Pins of the oracle's Philox4x32-10 generator and Gaussian transform."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox4x32_10, ln_pos, sincos_turn, gaussian_matrix
from oracle.gaussian import gaussian_pairs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
    assert [int(x) for x in got] == out


def test_philox_counter_independence():
    # different counters of one key give unrelated words; same counter same words
    ctr = np.zeros((4, 4), dtype=np.uint32)
    ctr[:, 0] = [0, 1, 2, 0]
    w = philox4x32_10(ctr, (7, 9))
    assert (w[0] == w[3]).all()
    assert len({tuple(r) for r in w[:3]}) == 3


def _ulp32_err(got, ref):
    return np.abs(got.astype(np.float64) - ref) / np.spacing(np.abs(ref).astype(np.float32))


def test_ln_accuracy():
    """The float32 logarithm of the generator against numpy's float64 log, on
    the generator's inputs u = j 2^-24, j = 1 .. 2^24, and the branch edges."""
    rng = np.random.default_rng(1)
    j = np.concatenate([rng.integers(1, 2 ** 24 + 1, 400000),
                        [1, 2, 3, 2 ** 23, 2 ** 23 + 1, 2 ** 24 - 1, 2 ** 24, 11863283, 11863284]])
    u = (j.astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    got = ln_pos(u)
    assert got.dtype == np.float32
    ref = np.log(u.astype(np.float64))
    nz = ref != 0
    assert np.max(_ulp32_err(got[nz], ref[nz])) <= 4.0
    assert got[u == 1.0].tolist() == [0.0] * int(np.sum(u == 1.0))


def test_sincos_accuracy():
    """sin / cos of 2 pi (x >> 8) / 2^24 in float32 against numpy's float64
    functions (through the quarter-turn identity, so np.sin/np.cos see only
    |angle| <= pi/4), to a few float32 ulps."""
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.integers(0, 2 ** 32, 200000, dtype=np.uint64),
                        np.array([0, 255, 256, 2 ** 29, 2 ** 29 - 256, 2 ** 30, 2 ** 31,
                                  3 * 2 ** 30, 2 ** 32 - 1], dtype=np.uint64)])
    s, c = sincos_turn(x.astype(np.uint32))
    assert s.dtype == np.float32 and c.dtype == np.float32
    a = (x >> 8).astype(np.int64)
    q = a >> 22
    rem = a & 0x3FFFFF
    up = rem >= 2 ** 21
    q = np.where(up, (q + 1) & 3, q)
    d = np.where(up, rem - 2 ** 22, rem).astype(np.float64)
    phi = d * (np.pi / 2 ** 23)
    rs = np.select([q == 0, q == 1, q == 2], [np.sin(phi), np.cos(phi), -np.sin(phi)], -np.cos(phi))
    rc = np.select([q == 0, q == 1, q == 2], [np.cos(phi), -np.sin(phi), -np.cos(phi)], np.sin(phi))
    assert np.max(np.abs(s - rs)) <= 2.5e-7
    assert np.max(np.abs(c - rc)) <= 2.5e-7
    theta = 2 * np.pi * (a.astype(np.float64) / 2.0 ** 24)
    assert np.max(np.abs(s - np.sin(theta))) < 3e-7
    assert np.max(np.abs(c - np.cos(theta))) < 3e-7
    s64, c64 = s.astype(np.float64), c.astype(np.float64)
    assert np.max(np.abs(s64 * s64 + c64 * c64 - 1.0)) < 5e-7


def test_gaussian_distribution():
    z = gaussian_matrix(1 << 10, 1 << 10, seed=12345, stream_id=1).ravel()
    assert abs(np.mean(z)) < 5e-3
    assert abs(np.var(z) - 1.0) < 5e-3
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # pairs are independent normals: even/odd entries uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5e-3


def test_gaussian_layout_and_streams():
    R, C = 7, 5
    M = gaussian_matrix(R, C, seed=3, stream_id=2)
    assert M.shape == (R, C) and M.flags.f_contiguous
    ze, zo = gaussian_pairs(0, (R * C + 1) // 2, 3, 2)
    flat = np.empty(2 * len(ze))
    flat[0::2] = ze
    flat[1::2] = zo
    for j in range(C):
        for i in range(R):
            assert M[i, j] == flat[i + j * R]
    assert not np.array_equal(M, gaussian_matrix(R, C, seed=3, stream_id=1))
    assert not np.array_equal(M, gaussian_matrix(R, C, seed=4, stream_id=2))
    assert np.array_equal(M, gaussian_matrix(R, C, seed=3, stream_id=2))
    # large seeds use both key words
    assert not np.array_equal(gaussian_matrix(R, C, seed=1 << 32, stream_id=2),
                              gaussian_matrix(R, C, seed=0, stream_id=2))
