"""Philox4x32-10 counter-based generator (oracle side).

Definition followed: Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Sec. 3.3 (Philox): a 4-word counter and a 2-word
key; each round multiplies words 0 and 2 by the constants M0, M1 (full 64-bit
products), swaps the halves and xors the high words with the other counter
words and the round key; the key is advanced by the Weyl constants W0, W1
between rounds; 10 rounds.

The paper draws every random test matrix as "a random Gaussian matrix"
(Algorithms rsvd, bpowerlu, gpowerlu, singlepasslu); it fixes no generator.
Reading used here: one Philox4x32-10 stream per (seed, stream id) with the
counter layout

    key     = (seed mod 2^32, seed div 2^32)
    counter = (q mod 2^32, q div 2^32, stream_id, 0)

where q is the index of a pair of matrix entries (see ``gaussian``).

Pinned by: the generator's published known-answer vectors
(tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

# Stream ids of the Gaussian test matrices.
STREAM_OMEGA_N = 1   # n x l  (odd v, Alg. gpowerlu; Alg. rlu; Alg. basicpoweriteration2)
STREAM_OMEGA_M = 2   # m x l  (even v, Alg. gpowerlu)
STREAM_OMEGA_SP = 3  # m x k  (Alg. singlepasslu)

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo(a_const, b):
    prod = a_const * b.astype(np.uint64)
    return (prod >> np.uint64(32)).astype(np.uint32), (prod & _MASK32).astype(np.uint32)


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to counters ``ctr`` (uint32, shape (N, 4)) under
    ``key`` (two uint32 words).  Returns uint32 (N, 4)."""
    c = np.asarray(ctr, dtype=np.uint32)
    c0, c1, c2, c3 = (c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy())
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        hi0, lo0 = _mulhilo(_M0, c0)
        hi1, lo1 = _mulhilo(_M1, c2)
        n0 = hi1 ^ c1 ^ np.uint32(k0)
        n2 = hi0 ^ c3 ^ np.uint32(k1)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
    return np.stack([c0, c1, c2, c3], axis=1)


def counters_for_pairs(q0, count, stream_id):
    """Counters of pair indices q0 .. q0+count-1 for one stream."""
    q = np.arange(q0, q0 + count, dtype=np.uint64)
    ctr = np.empty((count, 4), dtype=np.uint32)
    ctr[:, 0] = (q & _MASK32).astype(np.uint32)
    ctr[:, 1] = (q >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream_id)
    ctr[:, 3] = 0
    return ctr


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)
