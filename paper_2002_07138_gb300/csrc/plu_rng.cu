// a1: Gaussian test matrices Omega on the device.
//
// The paper draws "a random Gaussian matrix" (Alg. bpowerlu step 1,
// Alg. gpowerlu, Alg. singlepasslu step 1) without fixing a generator.  This
// kernel uses Philox4x32-10 (Salmon et al., SC'11: 10 rounds of two 32x32->64
// multiplications by 0xD2511F53 / 0xCD9E8D57 with a Weyl key schedule
// 0x9E3779B9 / 0xBB67AE85) and the Box-Muller transform.  Entry t = i + j*rows
// is output t mod 2 of pair t/2, counter (t/2 lo, t/2 hi, stream_id, 0),
// key (seed lo, seed hi):
//   u = ((w0 >> 5) 2^26 + (w1 >> 6) + 1) 2^-53 in (0, 1]
//   r = sqrt(-2 ln u), theta = 2 pi w2 / 2^32, entry = r cos / r sin.
// ln and sin/cos are evaluated from their series (atanh form of ln on
// [sqrt(1/2), sqrt(2)); Taylor sin/cos on |phi| <= pi/4 after taking the
// quarter turn from the top bits of w2; the series terms multiply by the
// correctly rounded reciprocals of their denominators) with explicitly
// rounded IEEE operations (no contraction into FMA), so every value is a
// fixed sequence of correctly rounded +, -, *, /, sqrt and is reproducible
// bit for bit.
#include "plu_internal.h"

#include "plu_rng.cuh"

namespace plu {
namespace {

__global__ void k_gaussian(int64_t rows, int64_t total, uint64_t npairs, uint32_t k0,
                           uint32_t k1, uint32_t stream_id, double* __restrict__ out,
                           int64_t ld) {
    for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < npairs;
         q += uint64_t(gridDim.x) * blockDim.x) {
        double ze, zo;
        rng::gaussian_pair(q, k0, k1, stream_id, ze, zo);
        const int64_t t0 = int64_t(2 * q);
        const int64_t i0 = t0 % rows, j0 = t0 / rows;
        out[i0 + j0 * ld] = ze;
        const int64_t t1 = t0 + 1;
        if (t1 < total) {
            const int64_t i1 = t1 % rows, j1 = t1 / rows;
            out[i1 + j1 * ld] = zo;
        }
    }
}

}  // namespace

cudaError_t launch_gaussian(int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                            double* out, int64_t ld, cudaStream_t s) {
    const int64_t total = rows * cols;
    if (total <= 0) return cudaSuccess;
    const uint64_t npairs = uint64_t(total + 1) / 2;
    const int threads = 256;
    uint64_t blocks = (npairs + threads - 1) / threads;
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    count_launch();
    k_gaussian<<<unsigned(blocks), threads, 0, s>>>(rows, total, npairs, uint32_t(seed),
                                                   uint32_t(seed >> 32), stream_id, out, ld);
    return cudaGetLastError();
}

}  // namespace plu
