"""Gaussian test matrices Omega (oracle side).

The paper draws "a random Gaussian matrix" of size n x l (Alg. bpowerlu
step 1, Alg. gpowerlu odd v), m x l (Alg. gpowerlu even v) or m x k
(Alg. singlepasslu step 1).  Reading used (the paper fixes no generator):
i.i.d. N(0, 1) entries by the Box-Muller transform (Box & Muller, 1958) of
Philox4x32-10 words, with the logarithm and the sine/cosine written out here
from their series so that the result is a fixed sequence of IEEE-754
double operations (+, -, *, /, sqrt; no fused multiply-add):

* entry (i, j) of an R x C matrix has column-major index t = i + j*R and
  belongs to the pair q = floor(t / 2); Philox(counter(q)) gives words
  x0, x1, x2, x3;
* u = ((x0 >> 5) * 2^26 + (x1 >> 6) + 1) * 2^-53, so u is in (0, 1];
* r = sqrt(-2 ln u), theta = 2 pi x2 / 2^32;
* entry = r cos(theta) if t is even, r sin(theta) if t is odd.

ln u: u = f 2^e with f in [sqrt(1/2), sqrt(2)); ln u = e ln 2 + 2 atanh(s),
s = (f - 1)/(f + 1), atanh(s) = s * sum_k s^(2k) / (2k + 1) for k <= 12.
sin / cos: the quarter turn is taken from the top two bits of x2, the rest
is centred to |phi| <= pi/4 and the Taylor series of sin (to phi^19) and
cos (to phi^20) are evaluated in nested form, 1 - (phi^2 * (1/d)) * t, with
the reciprocals 1/d of the denominators d = (2i)(2i+1) and (2i-1)(2i) as
correctly rounded constants (a multiplication per term instead of a
division; the generator is ours to fix, the paper leaves it open).

Pinned by: accuracy against numpy's log/sin/cos (a few ulp), and the
distribution of the output against the normal CDF (tests/test_oracle_rng.py).
"""
import numpy as np

from .philox import philox4x32_10, counters_for_pairs, seed_key

_SQRT_HALF = float(np.sqrt(0.5))
_LN2 = 0.69314718055994530942
_PI_OVER_2_31 = np.pi * 2.0 ** -31
_SIN_DEN = (342.0, 272.0, 210.0, 156.0, 110.0, 72.0, 42.0, 20.0, 6.0)
_COS_DEN = (380.0, 306.0, 240.0, 182.0, 132.0, 90.0, 56.0, 30.0, 12.0, 2.0)
_SIN_INV = tuple(1.0 / d for d in _SIN_DEN)        # correctly rounded reciprocals
_COS_INV = tuple(1.0 / d for d in _COS_DEN)
_ATANH_K = 12


def ln_pos(u):
    """Natural logarithm of positive normal doubles (array), fixed op order."""
    u = np.asarray(u, dtype=np.float64)
    f, e = np.frexp(u)                      # u = f * 2^e, f in [0.5, 1)
    small = f < _SQRT_HALF
    f = np.where(small, f * 2.0, f)
    e = np.where(small, e - 1, e).astype(np.float64)
    s = (f - 1.0) / (f + 1.0)
    w = s * s
    t = np.full_like(s, 1.0 / (2 * _ATANH_K + 1))
    for k in range(_ATANH_K - 1, -1, -1):
        t = t * w + 1.0 / (2 * k + 1)
    return e * _LN2 + (2.0 * s) * t


def sincos_turn(x):
    """(sin, cos) of 2*pi*x/2^32 for uint32 x (array), fixed op order."""
    x = np.asarray(x, dtype=np.uint32).astype(np.int64)
    quad = x >> 30
    rem = x & 0x3FFFFFFF
    up = rem >= (1 << 29)
    d = np.where(up, rem - (1 << 30), rem)
    quad = np.where(up, (quad + 1) & 3, quad)
    phi = d.astype(np.float64) * _PI_OVER_2_31
    x2 = phi * phi
    ts = np.ones_like(phi)
    for inv in _SIN_INV:
        ts = 1.0 - (x2 * inv) * ts
    s = phi * ts
    tc = np.ones_like(phi)
    for inv in _COS_INV:
        tc = 1.0 - (x2 * inv) * tc
    c = tc
    sin_out = np.select([quad == 0, quad == 1, quad == 2], [s, c, -s], -c)
    cos_out = np.select([quad == 0, quad == 1, quad == 2], [c, -s, -c], s)
    return sin_out, cos_out


def gaussian_pairs(q0, count, seed, stream_id):
    """Both Box-Muller outputs (z_even, z_odd) of pairs q0 .. q0+count-1."""
    words = philox4x32_10(counters_for_pairs(q0, count, stream_id), seed_key(seed))
    x0 = words[:, 0].astype(np.uint64)
    x1 = words[:, 1].astype(np.uint64)
    k = (x0 >> np.uint64(5)) * np.uint64(1 << 26) + (x1 >> np.uint64(6)) + np.uint64(1)
    u = k.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * ln_pos(u))
    s, c = sincos_turn(words[:, 2])
    return r * c, r * s


def gaussian_matrix(rows, cols, seed, stream_id):
    """R x C Gaussian matrix (Fortran-ordered float64) of one (seed, stream)."""
    total = rows * cols
    if total == 0:
        return np.zeros((rows, cols), dtype=np.float64, order="F")
    npairs = (total + 1) // 2
    out = np.empty(2 * npairs, dtype=np.float64)
    chunk = 1 << 22
    for q0 in range(0, npairs, chunk):
        cnt = min(chunk, npairs - q0)
        ze, zo = gaussian_pairs(q0, cnt, seed, stream_id)
        out[2 * q0:2 * (q0 + cnt):2] = ze
        out[2 * q0 + 1:2 * (q0 + cnt):2] = zo
    return np.asfortranarray(out[:total].reshape(cols, rows).T)
