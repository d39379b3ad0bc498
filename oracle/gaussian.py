"""Gaussian test matrices Omega (oracle side).

The paper draws "a random Gaussian matrix" of size n x l (Alg. bpowerlu
step 1, Alg. gpowerlu odd v), m x l (Alg. gpowerlu even v) or m x k
(Alg. singlepasslu step 1).  Reading used (the paper fixes no generator,
only the distribution): i.i.d. N(0, 1) entries by the Box-Muller transform
(Box & Muller, 1958) of Philox4x32-10 words, evaluated in IEEE-754 single
precision as a fixed sequence of correctly rounded operations (+, -, *, /,
sqrt; no fused multiply-add), with the logarithm and the sine/cosine written
out here from their series.  The entries are exact in float64.

* entry (i, j) of an R x C matrix has column-major index t = i + j*R and
  belongs to the pair q = floor(t / 2); Philox(counter(q)) gives words
  x0, x1, x2, x3;
* u = ((x0 >> 8) + 1) * 2^-24, so u is in (0, 1] and exact in float32;
* r = sqrt(-2 ln u), theta = 2 pi (x2 >> 8) / 2^24;
* entry = r cos(theta) if t is even, r sin(theta) if t is odd.

ln u: u = f 2^e with f in [sqrt(1/2), sqrt(2)); ln u = e ln 2 + 2 atanh(s),
s = (f - 1)/(f + 1), atanh(s) = s * sum_k s^(2k) / (2k + 1) for k <= 6
(|s| <= 0.172, so the first term left out is below 2^-30 of the sum).
sin / cos: the quarter turn is taken from the top two of the 24 angle bits,
the rest is centred to |phi| <= pi/4, and the Taylor series of sin (to
phi^11) and cos (to phi^12) are evaluated in nested form, 1 - (phi^2 *
(1/d)) * t, with the reciprocals 1/d of the denominators d = (2i)(2i+1) and
(2i-1)(2i) as float32 divisions (a multiplication per term).  ln 2 and
pi 2^-23 are the float32 values given by their bit patterns.

Pinned by: accuracy against numpy's float64 log/sin/cos (float32 level), and
the distribution of the output against the normal CDF
(tests/test_oracle_rng.py).
"""
import numpy as np

from .philox import philox4x32_10, counters_for_pairs, seed_key

F32 = np.float32


def _f32_bits(b):
    return np.array([b], dtype=np.uint32).view(np.float32)[0]


_SQRT_HALF = _f32_bits(0x3F3504F3)            # 0.70710677, float32 nearest to sqrt(1/2)
_LN2 = _f32_bits(0x3F317218)                  # float32 nearest to ln 2
_PI_2M23 = _f32_bits(0x34C90FDB)              # float32 pi times 2^-23 (exact scaling)
_ONE = F32(1.0)
_TWO = F32(2.0)
_ATANH_K = 6
_INV_ODD = tuple(_ONE / F32(2 * k + 1) for k in range(_ATANH_K + 1))
_SIN_INV = tuple(_ONE / F32(d) for d in (110.0, 72.0, 42.0, 20.0, 6.0))
_COS_INV = tuple(_ONE / F32(d) for d in (132.0, 90.0, 56.0, 30.0, 12.0, 2.0))


def ln_pos(u):
    """Natural logarithm of positive normal float32 values (array), fixed
    float32 operation order."""
    u = np.asarray(u, dtype=np.float32)
    f, e = np.frexp(u)                      # u = f * 2^e, f in [0.5, 1)
    small = f < _SQRT_HALF
    f = np.where(small, f * _TWO, f).astype(np.float32)
    e = np.where(small, e - 1, e).astype(np.float32)
    s = (f - _ONE) / (f + _ONE)
    w = s * s
    t = np.full_like(s, _INV_ODD[_ATANH_K])
    for k in range(_ATANH_K - 1, -1, -1):
        t = t * w + _INV_ODD[k]
    return e * _LN2 + (_TWO * s) * t


def sincos_turn(x):
    """(sin, cos) of 2*pi*(x >> 8)/2^24 for uint32 x (array), fixed float32
    operation order."""
    a = (np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(np.int64)
    quad = a >> 22
    rem = a & 0x3FFFFF
    up = rem >= (1 << 21)
    d = np.where(up, rem - (1 << 22), rem)
    quad = np.where(up, (quad + 1) & 3, quad)
    phi = d.astype(np.float32) * _PI_2M23      # |d| <= 2^21: exact conversion
    x2 = phi * phi
    ts = np.ones_like(phi)
    for inv in _SIN_INV:
        ts = _ONE - (x2 * inv) * ts
    s = phi * ts
    tc = np.ones_like(phi)
    for inv in _COS_INV:
        tc = _ONE - (x2 * inv) * tc
    c = tc
    sin_out = np.select([quad == 0, quad == 1, quad == 2], [s, c, -s], -c)
    cos_out = np.select([quad == 0, quad == 1, quad == 2], [c, -s, -c], s)
    return sin_out.astype(np.float32), cos_out.astype(np.float32)


def gaussian_pairs(q0, count, seed, stream_id):
    """Both Box-Muller outputs (z_even, z_odd) of pairs q0 .. q0+count-1,
    as float64 (exact copies of the float32 results)."""
    words = philox4x32_10(counters_for_pairs(q0, count, stream_id), seed_key(seed))
    x0 = words[:, 0].astype(np.uint32)
    u = ((x0 >> np.uint32(8)) + np.uint32(1)).astype(np.float32) * _f32_bits(0x33800000)  # 2^-24
    r = np.sqrt(-_TWO * ln_pos(u))
    s, c = sincos_turn(words[:, 2])
    return (r * c).astype(np.float64), (r * s).astype(np.float64)


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
