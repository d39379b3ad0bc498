// SIMT skinny GEMMs: the passes over A in FP64 (PLU_FP64) and FP32
// (PLU_FP32) arithmetic, and the small FP64 products between passes.
//
// A pass of Alg. gpowerlu / Alg. bpowerlu is Y = A X (m x n by n x l) or
// Y = A^T X (n x m by m x l) with column-major A.  On GB300 FP64 FMA runs at
// about 1/64 of the FP32 rate (~1 TFLOP/s), so the FP64 products are bound by
// the FP64 pipe, not by HBM: a 64x64x16 register-tiled kernel (4x4 outputs per
// thread, operands staged through padded shared memory) saturates it.  Each
// warp owns an 8-column strip of the tile, so the triangular products skip
// the FMAs of known-zero terms warp by warp (16 x 8 granularity), not only
// whole tiles: with the FP64 pipe as the bound, skipped FMAs are saved time.  When
// the output has too few 64x64 tiles to fill 152 SMs the reduction dimension
// is split; each split writes its partial tile and a second kernel sums the
// splits in a fixed order, so results do not depend on scheduling.
#include "plu_internal.h"

#include <climits>

namespace plu {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T> __device__ __forceinline__ T to_acc(float x) { return T(x); }

// An operand value in the arithmetic type TC: FP64 to FP32 on the integer pipe
template <typename TC, typename TS> __device__ __forceinline__ TC to_tc(TS v) {
    if constexpr (sizeof(TC) == 4 && sizeof(TS) == 8) return f64_to_f32_rn(double(v));
    else return TC(v);
}

// C partial (split z) = op(A)[M x Kz] * op(B)[Kz x N].
//   op(A)(i, k) = TRANSA ? A[k + i*lda] : A[i + k*lda]
//   op(B)(k, j) = TRANSB ? B[j + k*ldb] : B[k + j*ldb]
template <typename TA, typename TB, typename TC, bool TRANSA, bool TRANSB>
__global__ void __launch_bounds__(NT)
k_gemm_simt(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A, int64_t lda,
            const TB* __restrict__ B, int64_t ldb, TC* __restrict__ P, int64_t kchunk, int tri,
            const int* __restrict__ skip, double* __restrict__ norm_parts) {
    if (skip && *skip) return;                      // work cancelled on the device
    // ||A||_F^2 from the entries this CTA loads (the CTAs of the first column
    // tile cover every entry of A once)
    const bool want_norm = norm_parts != nullptr && blockIdx.y == 0;
    SqSum32 nsq;
    double nsq64 = 0.0;
    __shared__ TC As[2][BK][BM + 1];
    __shared__ TC Bs[2][BK][BN + 1];
    const int t = threadIdx.x;
    // warp w computes columns 8w .. 8w+7 of the tile: lane -> rows
    // (lane % 16) + 16a and columns 8w + lane / 16 + 2b, a, b = 0..3
    const int warp = t >> 5, lane = t & 31;
    const int ty = lane & 15, tx = 8 * warp + (lane >> 4);
    const int64_t i0 = int64_t(blockIdx.x) * BM;
    const int64_t j0 = int64_t(blockIdx.y) * BN;
    const int64_t kbeg = int64_t(blockIdx.z) * kchunk;
    int64_t kend = min(K, kbeg + kchunk);
    // tri 1: only the upper triangle of C is wanted (tiles wholly below the
    // diagonal write zeros); tri 2: op(B) is upper triangular (rows k > j of
    // column j are zero, so the reduction stops at the tile's last column);
    // tri 3: op(B) is lower triangular (rows k < j are zero, so the reduction
    // starts at the tile's first column)
    if (tri == 1 && i0 >= j0 + BN) kend = kbeg;
    if (tri == 2 && kend > j0 + BN) kend = j0 + BN;
    int64_t kstart = kbeg;
    if (tri == 3 && kstart < j0) kstart = j0 / BK * BK;
    if (kstart > kend) kstart = kend;

    TC ra[4], rb[4];
    auto load_a = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int ii, kk;
            if (TRANSA) { kk = t % 16; ii = t / 16 + 16 * r; }
            else        { ii = t % 64; kk = t / 64 + 4 * r; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            TC v = TC(0);
            if (gi < M && gk < kend) {
                const TA a = TRANSA ? A[gk + gi * lda] : A[gi + gk * lda];
                if (want_norm) {
                    if constexpr (sizeof(TA) == 4) nsq.add(float(a));
                    else nsq64 = fma(double(a), double(a), nsq64);
                }
                v = to_tc<TC>(a);
            }
            ra[r] = v;
        }
    };
    auto load_b = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int jj, kk;
            if (TRANSB) { jj = t % 64; kk = t / 64 + 4 * r; }
            else        { kk = t % 16; jj = t / 16 + 16 * r; }
            const int64_t gj = j0 + jj, gk = k0 + kk;
            TC v = TC(0);
            if (gj < N && gk < kend) v = to_tc<TC>(TRANSB ? B[gj + gk * ldb] : B[gk + gj * ldb]);
            rb[r] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int ii, kk;
            if (TRANSA) { kk = t % 16; ii = t / 16 + 16 * r; }
            else        { ii = t % 64; kk = t / 64 + 4 * r; }
            As[buf][kk][ii] = ra[r];
            int jj, kb;
            if (TRANSB) { jj = t % 64; kb = t / 64 + 4 * r; }
            else        { kb = t % 16; jj = t / 16 + 16 * r; }
            Bs[buf][kb][jj] = rb[r];
        }
    };

    TC acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
    // the warp's useful reduction range [wlo, whi] (tri 2, 3) and row groups
    // (tri 1: group a holds rows i0+16a.., wanted while i <= the strip's last column)
    const int64_t wc0 = j0 + 8 * warp, wc1 = wc0 + 7;
    const int64_t wlo = tri == 3 ? wc0 : INT64_MIN;
    const int64_t whi = tri == 2 ? wc1 : INT64_MAX;
    bool rowgrp[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) rowgrp[a] = tri != 1 || i0 + 16 * a <= wc1;

    int buf = 0;
    if (kstart < kend) {
        load_a(kstart);
        load_b(kstart);
        store(0);
    }
    __syncthreads();
    for (int64_t k0 = kstart; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) {
            load_a(k0 + BK);
            load_b(k0 + BK);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            if (k0 + kk < wlo || k0 + kk > whi) continue;   // warp-uniform
            TC av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[buf][kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][kk][tx + 2 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (!rowgrp[a]) continue;                     // warp-uniform
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if (norm_parts) {                                  // uniform over the CTA
        const double tot = cta_sum(want_norm ? nsq.value() + nsq64 : 0.0);
        if (want_norm && threadIdx.x == 0)
            norm_parts[blockIdx.x + int64_t(gridDim.x) * blockIdx.z] = tot;
    }
    TC* Pz = P + int64_t(blockIdx.z) * M * N;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gi = i0 + ty + 16 * a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t gj = j0 + tx + 2 * b;
            if (gj < N) Pz[gi + gj * M] = acc[a][b];
        }
    }
}

// C(i, j) = sum_z P[z](i, j), z in increasing order, in FP64 (accum > 0: added
// to C, accum < 0: subtracted from C).
template <typename TC>
__global__ void k_reduce_splits(int64_t M, int64_t N, int splits, const TC* __restrict__ P,
                                double* __restrict__ C, int64_t ldc, int accum,
                                const int* __restrict__ skip) {
    if (skip && *skip) return;
    // grid rows stride over the columns j, threads over the rows i
    const int64_t total = M * N;
    for (int64_t j = blockIdx.y; j < N; j += gridDim.y) {
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < M;
             i += int64_t(gridDim.x) * blockDim.x) {
            const int64_t e = i + j * M;
            double sum;
            if constexpr (sizeof(TC) == 4) {
                // compensated FP32 sum: no FP64 conversion and addition per split
                Sum2f acc;
                for (int z = 0; z < splits; ++z) acc.add(P[int64_t(z) * total + e]);
                sum = acc.value();
            } else {
                sum = 0.0;
                for (int z = 0; z < splits; ++z) sum += double(P[int64_t(z) * total + e]);
            }
            double* c = C + i + j * ldc;
            *c = accum > 0 ? *c + sum : accum < 0 ? *c - sum : sum;
        }
    }
}

__global__ void k_f64_to_f32(int64_t rows, int64_t cols, const double* __restrict__ X,
                             int64_t ldx, float* __restrict__ Y) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        Y[e] = f64_to_f32_rn(X[i + j * ldx]);
    }
}

int choose_splits(int64_t M, int64_t N, int64_t K, int num_sms) {
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    // many CTAs per SM so that uneven tiles (triangular shortcuts) balance
    const int64_t target = 16LL * num_sms;
    int64_t splits = (target + tiles - 1) / tiles;
    const int64_t max_by_k = (K + 8 * BK - 1) / (8 * BK);     // >= 8 k-steps per split
    if (splits > max_by_k) splits = max_by_k;
    if (splits < 1) splits = 1;
    if (splits > 256) splits = 256;
    return int(splits);
}

int grid_1d(int64_t work, int num_sms) {
    int64_t b = (work + 255) / 256;
    const int64_t cap = int64_t(num_sms) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return int(b);
}

// The split count is the preferred one, lowered to what the partial-sum
// buffer (part_cap bytes) holds; a buffer without room for one split is an
// error, never an overrun.
template <typename TA, typename TB, typename TC, bool TA_T, bool TB_T>
cudaError_t run(int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
                int64_t ldb, double* C, int64_t ldc, void* partials, size_t part_cap,
                int num_sms, cudaStream_t s, int tri = 0, int accum = 0,
                const int* skip = nullptr, const NormOut* norm = nullptr) {
    int splits = choose_splits(M, N, K, num_sms);
    const size_t one = size_t(M) * size_t(N) * sizeof(TC);
    if (!partials || part_cap < one) return cudaErrorInvalidValue;
    if (size_t(splits) * one > part_cap) splits = int(part_cap / one);
    int64_t kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    dim3 grid(unsigned((M + BM - 1) / BM), unsigned((N + BN - 1) / BN), unsigned(splits));
    TC* P = static_cast<TC*>(partials);
    const int64_t nparts = int64_t(grid.x) * grid.z;
    if (norm && (!norm->parts || !norm->out || nparts > norm->cap)) return cudaErrorInvalidValue;
    count_launch();
    k_gemm_simt<TA, TB, TC, TA_T, TB_T><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, kchunk,
                                                           tri, skip,
                                                           norm ? norm->parts : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (norm && (e = launch_sum_partials(norm->parts, int(nparts), norm->out, s)) != cudaSuccess)
        return e;
    count_launch();
    // about 16 CTAs per SM over (row chunks) x (columns)
    int64_t gx = (M + 255) / 256, gy = N;
    const int64_t want = int64_t(num_sms) * 16;
    if (gy > 65535) gy = 65535;
    if (gx * gy > want) gx = (want + gy - 1) / gy;
    if (gx < 1) gx = 1;
    k_reduce_splits<TC><<<dim3(unsigned(gx), unsigned(gy)), 256, 0, s>>>(M, N, splits, P, C, ldc,
                                                                         accum, skip);
    return cudaGetLastError();
}

}  // namespace

size_t gemm_partials_bytes(int64_t M, int64_t N, int64_t K, int prec, int num_sms) {
    const int splits = choose_splits(M, N, K, num_sms);
    const size_t el = (prec == PLU_FP32) ? sizeof(float) : sizeof(double);
    return size_t(splits) * size_t(M) * size_t(N) * el;
}

size_t gemm_f64_partials_bytes(int64_t M, int64_t N, int64_t K, int num_sms) {
    return gemm_partials_bytes(M, N, K, PLU_FP64, num_sms);
}

cudaError_t launch_gemm_simt(int trans, int64_t M, int64_t N, int64_t K, const void* A,
                             int dtype, int64_t lda, const double* B, int64_t ldb,
                             double* C, int64_t ldc, int prec, void* partials,
                             size_t part_cap, float* b32_scratch, int num_sms, cudaStream_t s,
                             int accum, const NormOut* norm) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (prec == PLU_FP32) {
        count_launch();
        k_f64_to_f32<<<grid_1d(K * N, num_sms), 256, 0, s>>>(K, N, B, ldb, b32_scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (dtype == PLU_F32) {
            const float* Af = static_cast<const float*>(A);
            return trans ? run<float, float, float, true, false>(M, N, K, Af, lda, b32_scratch, K, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm)
                         : run<float, float, float, false, false>(M, N, K, Af, lda, b32_scratch, K, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm);
        }
        const double* Ad = static_cast<const double*>(A);
        return trans ? run<double, float, float, true, false>(M, N, K, Ad, lda, b32_scratch, K, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm)
                     : run<double, float, float, false, false>(M, N, K, Ad, lda, b32_scratch, K, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm);
    }
    if (dtype == PLU_F32) {
        const float* Af = static_cast<const float*>(A);
        return trans ? run<float, double, double, true, false>(M, N, K, Af, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm)
                     : run<float, double, double, false, false>(M, N, K, Af, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm);
    }
    const double* Ad = static_cast<const double*>(A);
    return trans ? run<double, double, double, true, false>(M, N, K, Ad, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm)
                 : run<double, double, double, false, false>(M, N, K, Ad, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s, 0, accum, nullptr, norm);
}

int gemm_norm_parts(int64_t M, int64_t N, int64_t K, int num_sms) {
    return int(((M + BM - 1) / BM) * choose_splits(M, N, K, num_sms));
}

cudaError_t launch_gemm_f64(int transA, int transB, int64_t M, int64_t N, int64_t K,
                            const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc, void* partials, size_t part_cap,
                            int num_sms, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (transA) {
        return transB ? run<double, double, double, true, true>(M, N, K, A, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s)
                      : run<double, double, double, true, false>(M, N, K, A, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s);
    }
    return transB ? run<double, double, double, false, true>(M, N, K, A, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s)
                  : run<double, double, double, false, false>(M, N, K, A, lda, B, ldb, C, ldc, partials, part_cap, num_sms, s);
}

cudaError_t launch_gemm_f64_tri(int transA, int tri, int64_t M, int64_t N, int64_t K,
                                const double* A, int64_t lda, const double* B, int64_t ldb,
                                double* C, int64_t ldc, void* partials, size_t part_cap,
                                int num_sms, cudaStream_t s, const int* skip) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    return transA ? run<double, double, double, true, false>(M, N, K, A, lda, B, ldb, C, ldc,
                                                             partials, part_cap, num_sms, s, tri,
                                                             0, skip)
                  : run<double, double, double, false, false>(M, N, K, A, lda, B, ldb, C, ldc,
                                                              partials, part_cap, num_sms, s, tri,
                                                              0, skip);
}

cudaError_t launch_gemm_f32_tri(int tri, int64_t M, int64_t N, int64_t K, const double* A,
                                int64_t lda, const double* B, int64_t ldb, double* C,
                                int64_t ldc, void* partials, size_t part_cap, int num_sms,
                                cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    return run<double, double, float, false, false>(M, N, K, A, lda, B, ldb, C, ldc, partials,
                                                    part_cap, num_sms, s, tri, 0);
}

}  // namespace plu
