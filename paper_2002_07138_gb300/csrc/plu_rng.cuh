// Device-side Philox4x32-10 and Box-Muller helpers shared by the Gaussian
// kernels (plu_rng.cu, plu_batch.cu).  See plu_rng.cu for the definition.
#pragma once
#include <cstdint>

namespace plu {
namespace rng {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

// ln(u) for u in (0, 1]: u = f 2^e, f in [sqrt(1/2), sqrt(2)),
// ln u = e ln2 + 2 s sum_{k=0}^{12} s^{2k}/(2k+1), s = (f-1)/(f+1).
__device__ __forceinline__ double ln_unit(double u) {
    const long long bits = __double_as_longlong(u);
    int e = int((bits >> 52) & 0x7FF) - 1022;                   // u normal here
    double f = __longlong_as_double((bits & 0x800FFFFFFFFFFFFFLL) | (1022LL << 52));
    const double sqrt_half = 0.70710678118654752440;            // nearest double
    if (f < sqrt_half) {
        f = __dmul_rn(f, 2.0);
        e -= 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double w = __dmul_rn(s, s);
    // 1/(2k+1), k = 0..12, as correctly rounded constants (the same values the
    // division would give)
    constexpr double inv_odd[13] = {1.0 / 1.0,  1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0,
                                    1.0 / 11.0, 1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0,
                                    1.0 / 21.0, 1.0 / 23.0, 1.0 / 25.0};
    double t = inv_odd[12];
#pragma unroll
    for (int k = 11; k >= 0; --k) t = __dadd_rn(__dmul_rn(t, w), inv_odd[k]);
    const double ln2 = 0.69314718055994530942;
    return __dadd_rn(__dmul_rn(double(e), ln2), __dmul_rn(__dmul_rn(2.0, s), t));
}

// (sin, cos) of 2 pi x / 2^32.
__device__ __forceinline__ void sincos_turn(uint32_t x, double& so, double& co) {
    int quad = int(x >> 30);
    const int rem = int(x & 0x3FFFFFFFu);
    int d = rem;
    if (rem >= (1 << 29)) {
        d = rem - (1 << 30);
        quad = (quad + 1) & 3;
    }
    const double pi_over_2_31 = 3.141592653589793116 * (1.0 / 2147483648.0);
    const double phi = __dmul_rn(double(d), pi_over_2_31);
    const double x2 = __dmul_rn(phi, phi);
    // nested Taylor series; 1/d of the denominators d = (2i)(2i+1), (2i-1)(2i)
    // as correctly rounded constants (compile-time IEEE divisions)
    constexpr double sinv[9] = {1.0 / 342.0, 1.0 / 272.0, 1.0 / 210.0, 1.0 / 156.0, 1.0 / 110.0,
                                1.0 / 72.0,  1.0 / 42.0,  1.0 / 20.0,  1.0 / 6.0};
    constexpr double cinv[10] = {1.0 / 380.0, 1.0 / 306.0, 1.0 / 240.0, 1.0 / 182.0, 1.0 / 132.0,
                                 1.0 / 90.0,  1.0 / 56.0,  1.0 / 30.0,  1.0 / 12.0,  1.0 / 2.0};
    double ts = 1.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) ts = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, sinv[i]), ts));
    const double s = __dmul_rn(phi, ts);
    double tc = 1.0;
#pragma unroll
    for (int i = 0; i < 10; ++i) tc = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, cinv[i]), tc));
    const double c = tc;
    switch (quad) {
        case 0: so = s; co = c; break;
        case 1: so = c; co = -s; break;
        case 2: so = -s; co = -c; break;
        default: so = -c; co = s; break;
    }
}

// Both Box-Muller outputs of pair q of stream (seed, stream_id).
__device__ __forceinline__ void gaussian_pair(uint64_t q, uint32_t k0, uint32_t k1,
                                              uint32_t stream_id, double& z_even, double& z_odd) {
    uint32_t c0 = uint32_t(q), c1 = uint32_t(q >> 32), c2 = stream_id, c3 = 0;
    philox4x32_10(c0, c1, c2, c3, k0, k1);
    const uint64_t kint = (uint64_t(c0 >> 5) << 26) + uint64_t(c1 >> 6) + 1ull;
    const double u = __dmul_rn(double(kint), 1.0 / 9007199254740992.0);   // 2^-53
    const double r = __dsqrt_rn(__dmul_rn(-2.0, ln_unit(u)));
    double sn, cs;
    sincos_turn(c2, sn, cs);
    z_even = __dmul_rn(r, cs);
    z_odd = __dmul_rn(r, sn);
}

}  // namespace rng
}  // namespace plu
