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

// ln(u) for float32 u in (0, 1]: u = f 2^e, f in [sqrt(1/2), sqrt(2)),
// ln u = e ln2 + 2 s sum_{k=0}^{6} s^{2k}/(2k+1), s = (f-1)/(f+1); every step
// a correctly rounded float32 operation.
__device__ __forceinline__ float ln_unit(float u) {
    const int bits = __float_as_int(u);
    int e = ((bits >> 23) & 0xFF) - 126;                         // u normal here
    float f = __int_as_float((bits & 0x807FFFFF) | (126 << 23));  // f in [0.5, 1)
    if (f < __int_as_float(0x3F3504F3)) {                         // float32 sqrt(1/2)
        f = __fmul_rn(f, 2.0f);
        e -= 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float w = __fmul_rn(s, s);
    // 1/(2k+1), k = 0..6, as float32 divisions
    constexpr float inv_odd[7] = {1.0f / 1.0f, 1.0f / 3.0f,  1.0f / 5.0f, 1.0f / 7.0f,
                                  1.0f / 9.0f, 1.0f / 11.0f, 1.0f / 13.0f};
    float t = inv_odd[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) t = __fadd_rn(__fmul_rn(t, w), inv_odd[k]);
    const float ln2 = __int_as_float(0x3F317218);                 // float32 ln 2
    return __fadd_rn(__fmul_rn(__int2float_rn(e), ln2), __fmul_rn(__fmul_rn(2.0f, s), t));
}

// (sin, cos) of 2 pi (x >> 8) / 2^24 in float32.
__device__ __forceinline__ void sincos_turn(uint32_t x, float& so, float& co) {
    const int a = int(x >> 8);
    int quad = a >> 22;
    const int rem = a & 0x3FFFFF;
    int d = rem;
    if (rem >= (1 << 21)) {
        d = rem - (1 << 22);
        quad = (quad + 1) & 3;
    }
    // |d| <= 2^21 converts exactly; float32 pi times 2^-23
    const float phi = __fmul_rn(__int2float_rn(d), __int_as_float(0x34C90FDB));
    const float x2 = __fmul_rn(phi, phi);
    // nested Taylor series; 1/d of the denominators d = (2i)(2i+1), (2i-1)(2i)
    // as float32 divisions
    constexpr float sinv[5] = {1.0f / 110.0f, 1.0f / 72.0f, 1.0f / 42.0f, 1.0f / 20.0f,
                               1.0f / 6.0f};
    constexpr float cinv[6] = {1.0f / 132.0f, 1.0f / 90.0f, 1.0f / 56.0f, 1.0f / 30.0f,
                               1.0f / 12.0f,  1.0f / 2.0f};
    float ts = 1.0f;
#pragma unroll
    for (int i = 0; i < 5; ++i) ts = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(x2, sinv[i]), ts));
    const float s = __fmul_rn(phi, ts);
    float tc = 1.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) tc = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(x2, cinv[i]), tc));
    const float c = tc;
    switch (quad) {
        case 0: so = s; co = c; break;
        case 1: so = c; co = -s; break;
        case 2: so = -s; co = -c; break;
        default: so = -c; co = s; break;
    }
}

// Both Box-Muller outputs of pair q of stream (seed, stream_id), in float32.
__device__ __forceinline__ void gaussian_pair_f(uint64_t q, uint32_t k0, uint32_t k1,
                                                uint32_t stream_id, float& z_even, float& z_odd) {
    uint32_t c0 = uint32_t(q), c1 = uint32_t(q >> 32), c2 = stream_id, c3 = 0;
    philox4x32_10(c0, c1, c2, c3, k0, k1);
    // u = ((w0 >> 8) + 1) 2^-24 in (0, 1], exact
    const float u = __fmul_rn(__uint2float_rn((c0 >> 8) + 1u), __int_as_float(0x33800000));
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_unit(u)));
    float sn, cs;
    sincos_turn(c2, sn, cs);
    z_even = __fmul_rn(r, cs);
    z_odd = __fmul_rn(r, sn);
}

// The same pair returned exactly as doubles.
__device__ __forceinline__ void gaussian_pair(uint64_t q, uint32_t k0, uint32_t k1,
                                              uint32_t stream_id, double& z_even, double& z_odd) {
    float ze, zo;
    gaussian_pair_f(q, k0, k1, stream_id, ze, zo);
    z_even = double(ze);
    z_odd = double(zo);
}

}  // namespace rng
}  // namespace plu
