// a1: Gaussian test matrices Omega on the device.
//
// The paper draws "a random Gaussian matrix" (Alg. bpowerlu step 1,
// Alg. gpowerlu, Alg. singlepasslu step 1) without fixing a generator.  This
// kernel uses Philox4x32-10 (Salmon et al., SC'11: 10 rounds of two 32x32->64
// multiplications by 0xD2511F53 / 0xCD9E8D57 with a Weyl key schedule
// 0x9E3779B9 / 0xBB67AE85) and the Box-Muller transform.  Entry t = i + j*rows
// is output t mod 2 of pair t/2, counter (t/2 lo, t/2 hi, stream_id, 0),
// key (seed lo, seed hi), in IEEE single precision:
//   u = ((w0 >> 8) + 1) 2^-24 in (0, 1]
//   r = sqrt(-2 ln u), theta = 2 pi (w2 >> 8) / 2^24, entry = r cos / r sin.
// ln and sin/cos are evaluated from their series (atanh form of ln on
// [sqrt(1/2), sqrt(2)); Taylor sin/cos on |phi| <= pi/4 after taking the
// quarter turn from the top bits of the angle; the series terms multiply by
// the float32 reciprocals of their denominators) with explicitly rounded
// IEEE float32 operations (no contraction into FMA), so every value is a
// fixed sequence of correctly rounded +, -, *, /, sqrt, reproducible bit for
// bit, and exact in the FP64 output.
#include "plu_internal.h"

#include "plu_rng.cuh"

namespace plu {
namespace {

// One thread per entry (CTA row blockIdx.y strides over the columns): the
// entry's pair is generated and the entry's half kept, so no thread divides
// by the column length.
__global__ void k_gaussian(int64_t rows, int64_t cols, uint32_t k0, uint32_t k1,
                           uint32_t stream_id, double* __restrict__ out, int64_t ld) {
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y) {
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
             i += int64_t(gridDim.x) * blockDim.x) {
            const uint64_t t = uint64_t(j) * uint64_t(rows) + uint64_t(i);
            double ze, zo;
            rng::gaussian_pair(t >> 1, k0, k1, stream_id, ze, zo);
            out[i + j * ld] = (t & 1) ? zo : ze;
        }
    }
}

// Even column length: one thread per pair, both entries in the same column
// (entry t = i + j rows with i even starts pair t / 2), converted to FP64 on
// the integer pipe (exact).
__global__ void k_gaussian_pairs(int64_t rows, int64_t cols, uint32_t k0, uint32_t k1,
                                 uint32_t stream_id, double* __restrict__ out, int64_t ld) {
    const int64_t half = rows / 2;
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y) {
        for (int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; h < half;
             h += int64_t(gridDim.x) * blockDim.x) {
            const uint64_t q = uint64_t(j) * uint64_t(half) + uint64_t(h);
            float ze, zo;
            rng::gaussian_pair_f(q, k0, k1, stream_id, ze, zo);
            double* o = out + 2 * h + j * ld;
            o[0] = f32_to_f64(ze);
            o[1] = f32_to_f64(zo);
        }
    }
}

}  // namespace

cudaError_t launch_gaussian(int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                            double* out, int64_t ld, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    // about 32 CTAs of 256 threads per SM over (row chunks) x (columns)
    const bool pairs = rows % 2 == 0;
    int64_t gy = cols < 65535 ? cols : 65535;
    int64_t gx = ((pairs ? rows / 2 : rows) + 255) / 256;
    const int64_t want = int64_t(152) * 32;
    if (gx * gy > want) gx = (want + gy - 1) / gy;
    if (gx < 1) gx = 1;
    count_launch();
    if (pairs)
        k_gaussian_pairs<<<dim3(unsigned(gx), unsigned(gy)), 256, 0, s>>>(
            rows, cols, uint32_t(seed), uint32_t(seed >> 32), stream_id, out, ld);
    else
        k_gaussian<<<dim3(unsigned(gx), unsigned(gy)), 256, 0, s>>>(
            rows, cols, uint32_t(seed), uint32_t(seed >> 32), stream_id, out, ld);
    return cudaGetLastError();
}

}  // namespace plu
