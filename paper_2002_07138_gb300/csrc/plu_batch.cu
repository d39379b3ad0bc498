// Batched factorisation of many independent matrices of uneven size.
//
// Each problem is PowerLU (Alg. bpowerlu with Alg. gpowerlu, any v >= 2) or
// the single-pass LU (Alg. singlepasslu).  A problem is turned into a list of
// steps (Gaussian sketch, pass A X / A^T X, LU re-orthogonalisation, QR,
// final pass, LU tail); step t of every problem forms phase t.  A phase is
// executed as one grouped launch per kind of step: every kernel below reads
// a table of jobs (one per problem, or one per output tile) and a CTA looks
// up its job, so all problems of a phase run side by side across the GPU.
// The whole sequence of grouped launches is captured into one CUDA graph and
// launched once.
//
// Grouped kernels: the Gaussian sketch (Philox4x32-10 + Box-Muller, the same
// values as plu_gaussian); a SIMT GEMM over 64 x 32 output tiles (FP32 or
// FP64 arithmetic, no split of the reduction: the problems are small, so the
// tiles of all problems already fill the GPU); the partial-pivoting LU of a
// problem's panel in one CTA (same pivot order and virtual pivoting as the
// cooperative panel LU); the Cholesky factor and triangular inverse of
// CholeskyQR2 in one CTA per problem.
#include "plu_internal.h"
#include "plu_rng.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

namespace plu {
namespace {

// ------------------------------------------------------------ job tables
struct GaussJob {
    double* out;
    int64_t rows, ld;
    int cols;
    uint32_t k0, k1, stream;
};

struct GemmJob {
    const void* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
    int M, N, K;
    int transA, transB, a_f32, accum, tri;
    int tiles_m, tiles_n;
    int64_t tile0;
    const int* skip;     // nullable: when *skip, return (copy_on_skip: C = A instead)
    int copy_on_skip;
    int ksplit, kchunk;  // split-K: ksplit chunks of kchunk (a multiple of 16) of K
    double* part;        // ksplit > 1: chunk c's M x N partial at part + c M N (ld M)
};

// C = (accum ? C : 0) + the sum of a split-K job's partials, in chunk order;
// elements elem0 .. elem0 + M N - 1 of the grouped reduce.
struct RedJob {
    const double* part;
    double* C;
    int64_t ldc;
    int M, N, ksplit, accum;
    int64_t elem0;
    const int* skip;     // the GEMM job's skip flag (nothing to reduce when set)
};

struct LuJob {
    double* X;
    int64_t rows, ldx;
    int cols, mode;
    int32_t* perm;
    double* L;
    int64_t ldL;
    int l_trans;
    double* U;
    int64_t ldU;
    int u_trans;
    int32_t* info;
    int* pos;
    int* pivstep;
};

struct CholJob {
    double* W;
    double* Wsave;
    int n;
    int64_t rows;
    const int* skip;     // nullable: when *skip, return at once
    int* decide;         // nullable: set to 1 when R's diagonal spread is <= 1e5
};

struct TrinvJob {
    const double* R;
    double* Rinv;
    int n;
    const int* skip;
};

// --------------------------------------------------------- Gaussian
__global__ void k_b_gaussian(const GaussJob* __restrict__ jobs) {
    const GaussJob J = jobs[blockIdx.y];
    const int64_t total = J.rows * J.cols;
    const uint64_t npairs = uint64_t(total + 1) / 2;
    for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < npairs;
         q += uint64_t(gridDim.x) * blockDim.x) {
        double ze, zo;
        rng::gaussian_pair(q, J.k0, J.k1, J.stream, ze, zo);
        const int64_t t0 = int64_t(2 * q);
        J.out[t0 % J.rows + (t0 / J.rows) * J.ld] = ze;
        const int64_t t1 = t0 + 1;
        if (t1 < total) J.out[t1 % J.rows + (t1 / J.rows) * J.ld] = zo;
    }
}

// ------------------------------------------------------ grouped GEMM
// C = op(A) op(B) (+ C), op(A) M x K, op(B) K x N; one BMV x BNV tile per CTA
// of 256 threads, each thread (BMV/16) x (BNV/16) outputs.  The tile shape of
// every grouped launch is picked by timing (run_batch's autotuner) among
// kGemmVariants shapes.
constexpr int GBK = 16, GNT = 256;
constexpr int kGemmVariants = 3;
constexpr int kVarBM[kGemmVariants] = {64, 64, 128};
constexpr int kVarBN[kGemmVariants] = {32, 64, 32};
// Split-K choices: no split, K chunks of 1024, of 256.  A choice is
// variant + kGemmVariants * split index.  Only jobs with at most kSplitTiles
// output tiles and a longer K are split (the Gram matrices X^T X of the
// problems' CholeskyQR, whose few tiles otherwise each walk all of K), into
// at most kMaxSplit chunks.
constexpr int kSplitChoices = 3;
constexpr int kSplitK[kSplitChoices] = {0, 1024, 256};
constexpr int kGemmChoices = kGemmVariants * kSplitChoices;
constexpr int kSplitTiles = 8, kMaxSplit = 32;

// An FP64 operand value in the arithmetic type TC (FP32: on the integer pipe)
template <typename TC> __device__ __forceinline__ TC b_to_tc(double v) {
    if constexpr (sizeof(TC) == 4) return f64_to_f32_rn(v);
    else return v;
}

// n consecutive TC values from 16-byte (n * sizeof(TC) >= 16) or 8-byte
// aligned shared memory, as one or more vector loads
template <int N, typename TC> __device__ __forceinline__ void vload(const TC* p, TC* out) {
    if constexpr (sizeof(TC) == 4 && N == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else if constexpr (sizeof(TC) == 4 && N == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        out[0] = v.x; out[1] = v.y;
    } else if constexpr (sizeof(TC) == 8 && N == 2) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        out[0] = v.x; out[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = p[i];
    }
}

template <typename TC, int BMV, int BNV>
__global__ void __launch_bounds__(GNT)
k_b_gemm(const GemmJob* __restrict__ jobs, int njobs) {
    constexpr int TM = BMV / 16, TN = BNV / 16;
    // each thread owns TM consecutive rows and TN consecutive columns of the
    // tile; its operands come in vector loads of up to 16 bytes
    constexpr int VA = (TM * int(sizeof(TC))) >= 16 ? 16 / int(sizeof(TC)) : TM;
    constexpr int VB = (TN * int(sizeof(TC))) >= 16 ? 16 / int(sizeof(TC)) : TN;
    // rows padded to keep 16-byte alignment: each thread reads its TM (TN)
    // consecutive outputs' operands with vector loads
    constexpr int PAD = 16 / int(sizeof(TC));
    __shared__ __align__(16) TC As[2][GBK][BMV + PAD];
    __shared__ __align__(16) TC Bs[2][GBK][BNV + PAD];
    // job of this tile: last job with tile0 <= blockIdx.x; the job's tiles
    // run (row tile, column tile, K chunk), row tile fastest
    int lo = 0, hi = njobs - 1;
    const int64_t tile = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    const GemmJob J = jobs[lo];
    const int64_t local = tile - J.tile0;
    const int64_t mn_tiles = int64_t(J.tiles_m) * J.tiles_n;
    const int kc = int(local / mn_tiles);
    const int64_t i0 = (local % mn_tiles % J.tiles_m) * BMV;
    const int64_t j0 = (local % mn_tiles / J.tiles_m) * BNV;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    if (J.skip && *J.skip) {
        // a skipped second CholeskyQR round: its X R^-1 becomes the copy
        // C = A (A FP64, not transposed), the Gram does nothing
        if (J.copy_on_skip) {
            const double* Ad = static_cast<const double*>(J.A);
            for (int e = t; e < BMV * BNV; e += GNT) {
                const int64_t gi = i0 + e % BMV, gj = j0 + e / BMV;
                if (gi < J.M && gj < J.N) J.C[gi + gj * J.ldc] = Ad[gi + gj * J.lda];
            }
        }
        return;
    }
    int64_t kend = J.K;
    if (J.tri == 2 && kend > j0 + BNV) kend = j0 + BNV;
    const bool skip = (J.tri == 1 && i0 >= j0 + BNV);
    if (skip) kend = 0;
    const int64_t kbeg = int64_t(kc) * J.kchunk;
    if (J.ksplit > 1 && kend > kbeg + J.kchunk) kend = kbeg + J.kchunk;
    const float* Af = static_cast<const float*>(J.A);
    const double* Ad = static_cast<const double*>(J.A);
    // the next K step is loaded into registers while the current one is
    // multiplied out of shared memory (two buffers, one barrier per step)
    TC ra[TM], rb[TN];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            int ii, kk;
            if (J.transA) { kk = t % 16; ii = t / 16 + 16 * r; }
            else          { ii = t % BMV; kk = t / BMV + (GNT / BMV) * r; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            TC v = TC(0);
            if (gi < J.M && gk < kend) {
                const int64_t off = J.transA ? gk + gi * J.lda : gi + gk * J.lda;
                v = J.a_f32 ? TC(Af[off]) : b_to_tc<TC>(Ad[off]);
            }
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            int jj, kk;
            if (J.transB) { jj = t % BNV; kk = t / BNV + (GNT / BNV) * r; }
            else          { kk = t % 16; jj = t / 16 + 16 * r; }
            const int64_t gj = j0 + jj, gk = k0 + kk;
            TC v = TC(0);
            if (gj < J.N && gk < kend)
                v = b_to_tc<TC>(J.transB ? J.B[gj + gk * J.ldb] : J.B[gk + gj * J.ldb]);
            rb[r] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            int ii, kk;
            if (J.transA) { kk = t % 16; ii = t / 16 + 16 * r; }
            else          { ii = t % BMV; kk = t / BMV + (GNT / BMV) * r; }
            As[buf][kk][ii] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            int jj, kk;
            if (J.transB) { jj = t % BNV; kk = t / BNV + (GNT / BNV) * r; }
            else          { kk = t % 16; jj = t / 16 + 16 * r; }
            Bs[buf][kk][jj] = rb[r];
        }
    };
    TC acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = TC(0);
    if (kend > kbeg) {
        load(kbeg);
        store(0);
        __syncthreads();
        int buf = 0;
        for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
            const bool more = k0 + GBK < kend;
            if (more) load(k0 + GBK);
#pragma unroll
            for (int kk = 0; kk < GBK; ++kk) {
                TC av[TM], bv[TN];
#pragma unroll
                for (int a = 0; a < TM; a += VA)
                    vload<VA>(&As[buf][kk][ty * TM + a], av + a);
#pragma unroll
                for (int c = 0; c < TN; c += VB)
                    vload<VB>(&Bs[buf][kk][tx * TN + c], bv + c);
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                    for (int c = 0; c < TN; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
            }
            if (more) store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    double* pc = J.ksplit > 1 ? J.part + int64_t(kc) * J.M * J.N : nullptr;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int64_t gi = i0 + ty * TM + a;
        if (gi >= J.M) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int64_t gj = j0 + tx * TN + c;
            if (gj >= J.N) continue;
            if (pc) {
                pc[gi + gj * J.M] = double(acc[a][c]);
            } else {
                double* cp = J.C + gi + gj * J.ldc;
                *cp = J.accum ? *cp + double(acc[a][c]) : double(acc[a][c]);
            }
        }
    }
}

// The split-K jobs' reduction (RedJob), one element per thread.
__global__ void k_b_splitk_reduce(const RedJob* __restrict__ jobs, int njobs, int64_t total) {
    const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (e >= total) return;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].elem0 <= e) lo = mid;
        else hi = mid - 1;
    }
    const RedJob J = jobs[lo];
    if (J.skip && *J.skip) return;
    const int64_t x = e - J.elem0;
    const int64_t mn = int64_t(J.M) * J.N;
    double s = 0.0;
    for (int c = 0; c < J.ksplit; ++c) s += J.part[int64_t(c) * mn + x];
    double* cp = J.C + x % J.M + (x / J.M) * J.ldc;
    *cp = J.accum ? *cp + s : s;
}

// One grouped GEMM launch in tile shape `variant` over a job table whose tile
// fields were laid out for that shape.
cudaError_t launch_b_gemm(int variant, int tc32, const GemmJob* tab, int njobs, int64_t tiles,
                          cudaStream_t s) {
    if (tiles < 1) return cudaSuccess;
    switch (variant * 2 + (tc32 ? 1 : 0)) {
        case 0: k_b_gemm<double, 64, 32><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        case 1: k_b_gemm<float, 64, 32><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        case 2: k_b_gemm<double, 64, 64><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        case 3: k_b_gemm<float, 64, 64><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        case 4: k_b_gemm<double, 128, 32><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        case 5: k_b_gemm<float, 128, 32><<<unsigned(tiles), GNT, 0, s>>>(tab, njobs); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------- one-CTA partial-pivoting LU
constexpr int LNT = 512;
// multi-CTA LU: a panel with more than kMcWork FMAs of elimination gets
// ceil(work / kMcWork) CTAs (at most kMcMaxG, at least kMcMinRows rows each)
constexpr double kMcWork = 1.5e6;
constexpr int kMcMaxG = 16, kMcMinRows = 256;
constexpr int64_t kBatchSpin = 16LL << 20;   // spin limit of a group's column-step wait

struct BCand {
    double v;
    int pos;
    int row;
};

// v = |x|: bit patterns order as integers, NaNs lie above +inf's pattern
__device__ __forceinline__ bool b_better(const BCand& a, const BCand& b) {
    if (a.row < 0) return false;
    if (b.row < 0) return true;
    const long long ab = __double_as_longlong(a.v), bb = __double_as_longlong(b.v);
    const bool an = ab > 0x7FF0000000000000LL, bn = bb > 0x7FF0000000000000LL;
    if (an || bn) return an && bn ? a.pos < b.pos : bn;
    if (ab > bb) return true;
    if (ab < bb) return false;
    return a.pos < b.pos;
}

__device__ __forceinline__ BCand b_warp_best(BCand c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        BCand o;
        o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
        o.pos = __shfl_xor_sync(0xffffffffu, c.pos, off);
        o.row = __shfl_xor_sync(0xffffffffu, c.row, off);
        if (b_better(o, c)) c = o;
    }
    return c;
}

// The whole panel of one problem in one CTA: rows stay in place, each row's
// current position is tracked (LAPACK's interchange order decides ties), the
// pivot row is staged in shared memory, then the finalising writes of the
// cooperative version (P^T L in place, or perm, L, U) in the same kernel.
__global__ void __launch_bounds__(LNT)
k_b_panel_lu(const LuJob* __restrict__ jobs) {
    extern __shared__ double urow[];
    __shared__ BCand red[LNT / 32];
    __shared__ BCand piv;
    __shared__ int first_zero;
    const LuJob J = jobs[blockIdx.x];
    const int t = threadIdx.x;
    const int64_t rows = J.rows;
    const int cols = J.cols;
    const int steps = int(rows < int64_t(cols) ? rows : int64_t(cols));
    double* X = J.X;
    for (int64_t i = t; i < rows; i += LNT) {
        J.pos[i] = int(i);
        J.pivstep[i] = -1;
    }
    if (t == 0) first_zero = 0;
    __syncthreads();
    for (int j = 0; j < steps; ++j) {
        BCand best{-1.0, INT_MAX, -1};
        for (int64_t i = t; i < rows; i += LNT) {
            if (J.pivstep[i] >= 0) continue;
            const BCand c{fabs(X[i + int64_t(j) * J.ldx]), J.pos[i], int(i)};
            if (b_better(c, best)) best = c;
        }
        best = b_warp_best(best);
        if ((t & 31) == 0) red[t >> 5] = best;
        __syncthreads();
        if (t < 32) {
            BCand x = (t < LNT / 32) ? red[t] : BCand{-1.0, INT_MAX, -1};
            x = b_warp_best(x);
            if (t == 0) piv = x;
        }
        __syncthreads();
        const BCand pv = piv;
        for (int64_t i = t; i < rows; i += LNT) {
            if (i == pv.row) {
                J.pos[i] = j;
                J.pivstep[i] = j;
            } else if (J.pos[i] == j) {
                J.pos[i] = pv.pos;
            }
        }
        for (int c = j + t; c < cols; c += LNT) urow[c] = X[pv.row + int64_t(c) * J.ldx];
        if (t == 0 && pv.v == 0.0 && first_zero == 0) first_zero = j + 1;
        __syncthreads();
        const double ujj = urow[j];
        if (ujj != 0.0) {
            const double rinv = 1.0 / ujj;
            for (int64_t i = t; i < rows; i += LNT) {
                if (J.pivstep[i] >= 0) continue;
                double* xi = X + i;
                const double lij = lu_multiplier(xi[int64_t(j) * J.ldx], ujj, rinv);
                xi[int64_t(j) * J.ldx] = lij;
                for (int c = j + 1; c < cols; ++c) {
                    double* p = xi + int64_t(c) * J.ldx;
                    *p = fma(-lij, urow[c], *p);
                }
            }
        }
        __syncthreads();
    }
    if (t == 0 && J.info) *J.info = first_zero;
    const int r = steps;
    for (int64_t i = t; i < rows; i += LNT) {
        const int s = J.pivstep[i];
        if (J.mode == 0) {
            if (s >= 0) {
                X[i + int64_t(s) * J.ldx] = 1.0;
                for (int c = s + 1; c < cols; ++c) X[i + int64_t(c) * J.ldx] = 0.0;
            }
            continue;
        }
        const int64_t pp = J.pos[i];
        J.perm[pp] = int32_t(i);
        for (int c = 0; c < r; ++c) {
            double v;
            if (s >= 0 && c == s) v = 1.0;
            else if (s >= 0 && c > s) v = 0.0;
            else v = X[i + int64_t(c) * J.ldx];
            if (J.l_trans) J.L[c + pp * J.ldL] = v;
            else J.L[pp + int64_t(c) * J.ldL] = v;
        }
        if (s >= 0) {
            for (int c = 0; c < cols; ++c) {
                const double v = (c >= s) ? X[i + int64_t(c) * J.ldx] : 0.0;
                if (J.u_trans) J.U[c + int64_t(s) * J.ldU] = v;
                else J.U[s + int64_t(c) * J.ldU] = v;
            }
        }
    }
}

// ------------------------------- the LU of one problem over several CTAs
// The large problems' panels: G CTAs of a cooperative launch share one
// problem, each owning a contiguous run of its rows; a column step publishes
// each CTA's candidate in a slot (two sets, by step parity, so a fast CTA
// never overwrites slots a slow one still reads), counts arrivals on the
// problem's counter (release), and every CTA, once all G have arrived
// (acquire; bounded spin, PLU timeout status on expiry), reduces the G slots
// to the same pivot.  The pivot's row is read from L2 (its owner updated it
// before publishing).  Same pivot order, tie rule, multipliers and FMAs per
// entry as k_b_panel_lu, so the same factors.
struct McCta {
    int job;
    int rank, G;
    int64_t r0, r1;      // rows [r0, r1) of the problem
};

struct McSync {
    int64_t cnt_off;     // per job: byte offsets (from the table base) of the
    int64_t slots_off;   // arrival counter and of its 2 x G candidate slots
};

__global__ void __launch_bounds__(LNT)
k_b_panel_lu_mc(const LuJob* __restrict__ jobs, const McCta* __restrict__ ctas,
                const McSync* __restrict__ syncs, unsigned char* __restrict__ base,
                int* __restrict__ status, int64_t budget) {
    extern __shared__ double urow[];
    __shared__ BCand red[LNT / 32];
    __shared__ BCand piv;
    __shared__ int first_zero;
    __shared__ int ok;
    const McCta C = ctas[blockIdx.x];
    const LuJob J = jobs[C.job];
    unsigned* const cnt = reinterpret_cast<unsigned*>(base + syncs[C.job].cnt_off);
    BCand* const slots = reinterpret_cast<BCand*>(base + syncs[C.job].slots_off);
    const int t = threadIdx.x;
    const int cols = J.cols;
    const int steps = int(J.rows < int64_t(cols) ? J.rows : int64_t(cols));
    double* X = J.X;
    for (int64_t i = C.r0 + t; i < C.r1; i += LNT) {
        J.pos[i] = int(i);
        J.pivstep[i] = -1;
    }
    if (t == 0) {
        first_zero = 0;
        ok = 1;
    }
    __syncthreads();
    for (int j = 0; j < steps; ++j) {
        BCand best{-1.0, INT_MAX, -1};
        for (int64_t i = C.r0 + t; i < C.r1; i += LNT) {
            if (J.pivstep[i] >= 0) continue;
            const BCand c{fabs(X[i + int64_t(j) * J.ldx]), J.pos[i], int(i)};
            if (b_better(c, best)) best = c;
        }
        best = b_warp_best(best);
        if ((t & 31) == 0) red[t >> 5] = best;
        __syncthreads();
        if (t < 32) {
            BCand x = (t < LNT / 32) ? red[t] : BCand{-1.0, INT_MAX, -1};
            x = b_warp_best(x);
            if (t == 0) {
                BCand* slot = slots + (j & 1) * C.G + C.rank;
                slot->v = x.v;
                slot->pos = x.pos;
                slot->row = x.row;
                __threadfence();
                red_release_add_u32(cnt, 1u);
                const unsigned target = unsigned(j + 1) * unsigned(C.G);
                int64_t spins = 0;
                while (ld_acquire_u32(cnt) < target) {
                    if (ld_volatile_i32(status) != DEV_OK || ++spins > budget) {
                        atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        if (!ok) return;
        if (t < 32) {
            BCand x{-1.0, INT_MAX, -1};
            for (int g = t; g < C.G; g += 32) {
                const BCand* sl = slots + (j & 1) * C.G + g;
                const BCand c{__ldcg(&sl->v), __ldcg(&sl->pos), __ldcg(&sl->row)};
                if (b_better(c, x)) x = c;
            }
            x = b_warp_best(x);
            if (t == 0) piv = x;
        }
        __syncthreads();
        const BCand pv = piv;
        if (pv.row < 0) break;                        // no row left (cannot happen: rows >= steps)
        for (int64_t i = C.r0 + t; i < C.r1; i += LNT) {
            if (i == pv.row) {
                J.pos[i] = j;
                J.pivstep[i] = j;
            } else if (J.pos[i] == j) {
                J.pos[i] = pv.pos;
            }
        }
        for (int c = j + t; c < cols; c += LNT) urow[c] = __ldcg(&X[pv.row + int64_t(c) * J.ldx]);
        if (t == 0 && pv.v == 0.0 && first_zero == 0) first_zero = j + 1;
        __syncthreads();
        const double ujj = urow[j];
        if (ujj != 0.0) {
            const double rinv = 1.0 / ujj;
            for (int64_t i = C.r0 + t; i < C.r1; i += LNT) {
                if (J.pivstep[i] >= 0) continue;
                double* xi = X + i;
                const double lij = lu_multiplier(xi[int64_t(j) * J.ldx], ujj, rinv);
                xi[int64_t(j) * J.ldx] = lij;
                for (int c = j + 1; c < cols; ++c) {
                    double* p = xi + int64_t(c) * J.ldx;
                    *p = fma(-lij, urow[c], *p);
                }
            }
        }
        __syncthreads();
    }
    if (t == 0 && J.info && C.rank == 0) *J.info = first_zero;
    const int r = steps;
    for (int64_t i = C.r0 + t; i < C.r1; i += LNT) {
        const int s = J.pivstep[i];
        if (J.mode == 0) {
            if (s >= 0) {
                X[i + int64_t(s) * J.ldx] = 1.0;
                for (int c = s + 1; c < cols; ++c) X[i + int64_t(c) * J.ldx] = 0.0;
            }
            continue;
        }
        const int64_t pp = J.pos[i];
        J.perm[pp] = int32_t(i);
        for (int c = 0; c < r; ++c) {
            double v;
            if (s >= 0 && c == s) v = 1.0;
            else if (s >= 0 && c > s) v = 0.0;
            else v = X[i + int64_t(c) * J.ldx];
            if (J.l_trans) J.L[c + pp * J.ldL] = v;
            else J.L[pp + int64_t(c) * J.ldL] = v;
        }
        if (s >= 0) {
            for (int c = 0; c < cols; ++c) {
                const double v = (c >= s) ? X[i + int64_t(c) * J.ldx] : 0.0;
                if (J.u_trans) J.U[c + int64_t(s) * J.ldU] = v;
                else J.U[s + int64_t(c) * J.ldU] = v;
            }
        }
    }
}

// ---------------------------------------- one-CTA Cholesky W = R^T R
// Upper triangle read, R written over it, lower part zeroed; a non-positive
// pivot restarts from the saved Gram matrix with the shifted-CholeskyQR shift
// 11 (rows n + n(n+1)) u tr(W).
constexpr int CNT = 512;

__global__ void __launch_bounds__(CNT)
k_b_cholesky(const CholJob* __restrict__ jobs, int* __restrict__ status) {
    __shared__ int broke;
    __shared__ double rjj;
    const CholJob J = jobs[blockIdx.x];
    if (J.skip && *J.skip) return;
    const int n = J.n;
    double* W = J.W;
    const int t = threadIdx.x;
    for (int64_t e = t; e < int64_t(n) * n; e += CNT) J.Wsave[e] = W[e];
    __syncthreads();
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            double tr = 0.0;
            for (int i = 0; i < n; ++i) tr += J.Wsave[i + int64_t(i) * n];
            const double shift =
                11.0 * (double(J.rows) * n + double(n) * (n + 1)) * 1.1102230246251565e-16 * tr;
            for (int64_t e = t; e < int64_t(n) * n; e += CNT) {
                const int a = int(e % n), c = int(e / n);
                W[e] = J.Wsave[e] + (a == c ? shift : 0.0);
            }
            __syncthreads();
        }
        if (t == 0) broke = 0;
        __syncthreads();
        // LDL^T order: one reciprocal 1/d_j per pivot on the critical path
        // (thread 0), the rank-1 update with the unscaled row j, and the
        // square roots and row scalings afterwards, in parallel
        for (int j = 0; j < n; ++j) {
            if (t == 0) {
                const double d = W[j + int64_t(j) * n];
                if (!(d > 0.0)) broke = 1;
                rjj = (d > 0.0) ? 1.0 / d : 0.0;
            }
            __syncthreads();
            if (broke) break;
            const double z = rjj;
            const int m = n - j - 1;
            for (int64_t e = t; e < int64_t(m) * m; e += CNT) {
                const int a = j + 1 + int(e % m), c = j + 1 + int(e / m);
                if (a <= c)
                    W[a + int64_t(c) * n] =
                        fma(-W[j + int64_t(a) * n] * z, W[j + int64_t(c) * n], W[a + int64_t(c) * n]);
            }
            __syncthreads();
        }
        if (!broke) {
            // R(j, c) = W(j, c) / sqrt(d_j) for c >= j (R(j, j) = sqrt(d_j));
            // 1/sqrt(d_j) goes to Wsave (no longer needed once the
            // factorisation has succeeded) before any W entry changes
            for (int a = t; a < n; a += CNT) J.Wsave[a] = rsqrt(W[a + int64_t(a) * n]);
            __syncthreads();
            for (int64_t e = t; e < int64_t(n) * n; e += CNT) {
                const int a = int(e % n), c = int(e / n);
                if (a <= c) W[e] *= J.Wsave[a];
            }
            __syncthreads();
        }
        if (!broke) break;
        if (attempt == 1 && t == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
    }
    __syncthreads();
    for (int64_t e = t; e < int64_t(n) * n; e += CNT) {
        const int a = int(e % n), c = int(e / n);
        if (a > c) W[e] = 0.0;
    }
    if (J.decide && t < 32) {
        // the second CholeskyQR round is needed when max|r_ii| / min|r_ii|
        // exceeds 1e5 (one round leaves an orthogonality loss ~spread^2 u)
        double dmax = 0.0, dmin = 1.7976931348623157e308;
        for (int i = t; i < n; i += 32) {
            const double d = fabs(W[i + int64_t(i) * n]);
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
            dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
        }
        if (t == 0) *J.decide = (dmin > 0.0 && dmax <= 1e5 * dmin) ? 1 : 0;
    }
}

// Rinv(:, j) = R^{-1} e_j, CTA (j, job).  The reciprocals of the diagonal
// are taken up front in parallel: a dependent FP64 division costs ~430
// cycles of the narrow FP64 pipe, a multiply ~65.
__global__ void k_b_trinv(const TrinvJob* __restrict__ jobs) {
    extern __shared__ double x[];                 // x[n], then rd[n]
    const TrinvJob J = jobs[blockIdx.y];
    const int j = blockIdx.x;
    if (j >= J.n || (J.skip && *J.skip)) return;
    const int n = J.n;
    double* rd = x + n;
    const int t = threadIdx.x;
    for (int i = t; i < n; i += blockDim.x) {
        x[i] = (i == j) ? 1.0 : 0.0;
        if (i <= j) rd[i] = 1.0 / J.R[i + int64_t(i) * n];
    }
    __syncthreads();
    for (int i = j; i >= 0; --i) {
        if (t == 0) x[i] *= rd[i];
        __syncthreads();
        const double xi = x[i];
        for (int k = t; k < i; k += blockDim.x) x[k] -= xi * J.R[k + int64_t(i) * n];
        __syncthreads();
    }
    for (int i = t; i < n; i += blockDim.x) J.Rinv[i + int64_t(j) * n] = x[i];
}

// ------------------------------------------------------- host planning
enum OpKind { OP_GAUSS, OP_PASS, OP_LU, OP_QR, OP_TAIL, OP_SPTAIL };

struct Op {
    int kind;
    // OP_GAUSS
    double* g_out; int64_t g_rows; int g_cols; uint32_t g_stream;
    // OP_PASS: Y = op(A) X
    int trans; const double* X; int64_t ldx; double* Y; int64_t ldy; int cols;
    // OP_LU / OP_QR on V (rows x l)
    double* P; int64_t prow;
};

struct ProbWs {
    double *V, *Z, *X2, *L1, *U1T, *BT, *U2T, *W, *Wsave, *Rinv, *Rinv1, *T;
    int *pos, *piv;
    int32_t* info;
    int* qskip;          // the second CholeskyQR round is skipped (FP32 passes)
};

struct LaunchRec {
    int kind;          // 0 gauss, 1 gemm, 2 lu, 3 chol, 4 trinv
    size_t off;        // byte offset of the job table
    int njobs;
    int64_t tiles;     // gemm: total tiles
    int maxn;          // trinv / lu smem
    int tc32;          // gemm arithmetic FP32
    int gidx = -1;     // gemm: index of its job list in Builder::gjobs
    int variant = 0;   // gemm: tile shape and split-K choice (lay_tiles)
    size_t red_off = 0;  // gemm: split-K reduction table
    int red_jobs = 0;
    int64_t red_elems = 0;
    size_t cta_off = 0, sync_off = 0, zero_off = 0, zero_bytes = 0;   // multi-CTA LU
    int nctas = 0;
};

// The tile and split-K fields of a grouped GEMM's jobs for `choice`; returns
// the total number of tiles.  Split jobs take their partials from `part`
// (consecutive, *part_elems doubles in all; part may be null when only the
// size is wanted).  The split jobs' reduction table goes to *red.
int64_t lay_tiles(std::vector<GemmJob>& jobs, int choice, double* part, int64_t* part_elems,
                  std::vector<RedJob>* red) {
    const int variant = choice % kGemmVariants;
    const int kc = kSplitK[choice / kGemmVariants];
    const int bm = kVarBM[variant], bn = kVarBN[variant];
    int64_t tiles = 0, pe = 0, elems = 0;
    if (red) red->clear();
    for (auto& j : jobs) {
        j.tiles_m = (j.M + bm - 1) / bm;
        j.tiles_n = (j.N + bn - 1) / bn;
        j.ksplit = 1;
        j.kchunk = 0;
        j.part = nullptr;
        if (kc > 0 && !j.copy_on_skip && j.tiles_m * j.tiles_n <= kSplitTiles && j.K > kc) {
            int ks = (j.K + kc - 1) / kc;
            if (ks > kMaxSplit) ks = kMaxSplit;
            j.kchunk = ((j.K + ks - 1) / ks + GBK - 1) / GBK * GBK;
            j.ksplit = (j.K + j.kchunk - 1) / j.kchunk;
            if (j.ksplit > 1) {
                j.part = part ? part + pe : nullptr;
                if (red) {
                    RedJob r{};
                    r.part = j.part;
                    r.C = j.C;
                    r.ldc = j.ldc;
                    r.M = j.M;
                    r.N = j.N;
                    r.ksplit = j.ksplit;
                    r.accum = j.accum;
                    r.elem0 = elems;
                    r.skip = j.skip;
                    red->push_back(r);
                }
                pe += int64_t(j.ksplit) * j.M * j.N;
                elems += int64_t(j.M) * j.N;
            } else {
                j.ksplit = 1;
                j.kchunk = 0;
            }
        }
        j.tile0 = tiles;
        tiles += int64_t(j.tiles_m) * j.tiles_n * j.ksplit;
    }
    if (part_elems) *part_elems = pe;
    return tiles;
}

struct Builder {
    std::vector<unsigned char> blob;
    std::vector<LaunchRec> recs;
    template <typename T>
    size_t put(const std::vector<T>& v) {
        size_t off = (blob.size() + 255) & ~size_t(255);
        blob.resize(off + v.size() * sizeof(T));
        memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
    // grouped GEMMs: the job lists are kept aside until their tile shapes are
    // chosen (place_gemms)
    std::vector<std::vector<GemmJob>> gjobs;
    void gemm(std::vector<GemmJob>& jobs, int tc32) {
        if (jobs.empty()) return;
        LaunchRec r{1, 0, int(jobs.size()), 0, 0, tc32};
        r.gidx = int(gjobs.size());
        gjobs.push_back(jobs);
        recs.push_back(r);
        jobs.clear();
    }
    // every grouped GEMM's table, laid out for its chosen shape, into the blob
    // and the split jobs' reduction tables; the launches run one after the
    // other, so all take their partials from the same `part` region.
    // Returns the doubles of partials the largest launch needs.
    int64_t place_gemms(const std::vector<int>& choice, double* part) {
        int64_t most = 0;
        for (auto& r : recs) {
            if (r.kind != 1) continue;
            r.variant = choice[r.gidx];
            int64_t pe = 0;
            std::vector<RedJob> red;
            r.tiles = lay_tiles(gjobs[r.gidx], r.variant, part, &pe, &red);
            r.off = put(gjobs[r.gidx]);
            r.red_jobs = int(red.size());
            r.red_elems = red.empty() ? 0 : red.back().elem0 + int64_t(red.back().M) * red.back().N;
            if (!red.empty()) r.red_off = put(red);
            if (pe > most) most = pe;
        }
        return most;
    }
    // co-resident CTAs of the multi-CTA LU (0: none)
    int mc_cap = 0;
    // A phase's LUs: the large panels (more than kMcWork FP64 FMAs of
    // elimination) on G CTAs each (a cooperative launch, first), the rest one
    // CTA each.
    void lu(std::vector<LuJob>& jobs) {
        if (jobs.empty()) return;
        std::vector<LuJob> one, many;
        std::vector<int> G;
        for (auto& j : jobs) {
            const double work = double(j.rows) * j.cols * j.cols / 2.0;
            int g = int(std::min<double>(std::ceil(work / kMcWork), double(kMcMaxG)));
            const int64_t rg = j.rows / kMcMinRows;
            if (g > rg) g = int(rg);
            if (mc_cap >= 2 && g >= 2) {
                many.push_back(j);
                G.push_back(g);
            } else {
                one.push_back(j);
            }
        }
        // fit the co-resident capacity: shrink the groups, then drop the smallest
        auto total = [&]() { int s = 0; for (int g : G) s += g; return s; };
        while (!many.empty() && total() > mc_cap) {
            int big = 0;
            for (size_t i = 1; i < G.size(); ++i) if (G[i] > G[big]) big = int(i);
            if (G[big] > 2) {
                --G[big];
            } else {
                one.push_back(many.back());
                many.pop_back();
                G.pop_back();
            }
        }
        if (!many.empty()) {
            std::vector<McCta> ctas;
            std::vector<McSync> syncs;
            int maxc = 1;
            size_t zbytes = 0;
            std::vector<int64_t> cnt_rel, slot_rel;
            for (size_t q = 0; q < many.size(); ++q) {
                maxc = std::max(maxc, many[q].cols);
                cnt_rel.push_back(int64_t(zbytes));
                zbytes += 16;
                slot_rel.push_back(int64_t(zbytes));
                zbytes += size_t(2) * G[q] * sizeof(BCand);
                const int64_t rows = many[q].rows;
                for (int r = 0; r < G[q]; ++r)
                    ctas.push_back(McCta{int(q), r, G[q], rows * r / G[q], rows * (r + 1) / G[q]});
            }
            std::vector<unsigned char> zeros((zbytes + 255) & ~size_t(255), 0);
            LaunchRec rec{5, put(many), int(many.size()), 0, maxc, 0};
            rec.cta_off = put(ctas);
            rec.nctas = int(ctas.size());
            rec.zero_off = put(zeros);
            rec.zero_bytes = zeros.size();
            for (size_t q = 0; q < many.size(); ++q)
                syncs.push_back(McSync{int64_t(rec.zero_off) + cnt_rel[q],
                                       int64_t(rec.zero_off) + slot_rel[q]});
            rec.sync_off = put(syncs);
            recs.push_back(rec);
        }
        if (!one.empty()) {
            int maxc = 1;
            for (auto& j : one) maxc = std::max(maxc, j.cols);
            recs.push_back(LaunchRec{2, put(one), int(one.size()), 0, maxc, 0});
        }
        jobs.clear();
    }
    void gauss(std::vector<GaussJob>& jobs) {
        if (jobs.empty()) return;
        recs.push_back(LaunchRec{0, put(jobs), int(jobs.size()), 0, 0, 0});
        jobs.clear();
    }
    void chol(std::vector<CholJob>& jobs) {
        if (jobs.empty()) return;
        recs.push_back(LaunchRec{3, put(jobs), int(jobs.size()), 0, 0, 0});
        jobs.clear();
    }
    void trinv(std::vector<TrinvJob>& jobs) {
        if (jobs.empty()) return;
        int maxn = 1;
        for (auto& j : jobs) maxn = std::max(maxn, j.n);
        recs.push_back(LaunchRec{4, put(jobs), int(jobs.size()), 0, maxn, 0});
        jobs.clear();
    }
};

GemmJob mk_gemm(const void* A, int64_t lda, int a_f32, int transA, const double* B, int64_t ldb,
                int transB, double* C, int64_t ldc, int M, int N, int K, int accum = 0,
                int tri = 0) {
    GemmJob g{};
    g.A = A; g.lda = lda; g.a_f32 = a_f32; g.transA = transA;
    g.B = B; g.ldb = ldb; g.transB = transB;
    g.C = C; g.ldc = ldc; g.M = M; g.N = N; g.K = K; g.accum = accum; g.tri = tri;
    return g;
}

LuJob mk_lu(double* X, int64_t rows, int cols, int mode, int32_t* perm, double* L, int64_t ldL,
            int l_trans, double* U, int64_t ldU, int u_trans, int32_t* info, int* pos, int* piv) {
    LuJob j{};
    j.X = X; j.rows = rows; j.ldx = rows; j.cols = cols; j.mode = mode;
    j.perm = perm; j.L = L; j.ldL = ldL; j.l_trans = l_trans;
    j.U = U; j.ldU = ldU; j.u_trans = u_trans; j.info = info; j.pos = pos; j.pivstep = piv;
    return j;
}

}  // namespace

size_t batch_workspace_bytes(const plu_batch_problem* P, int count) {
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t m = P[i].m, n = P[i].n, mx = m > n ? m : n;
        const int64_t l = P[i].algo == 1 ? P[i].k : P[i].l, k = P[i].k;
        size_t d = size_t(n * l + m * l + mx * l + m * k + k * k + n * k + k * k + 5 * l * l + k * k);
        total += ((d * sizeof(double) + 255) & ~size_t(255)) +
                 ((size_t(2 * mx + 4) * sizeof(int) + 255) & ~size_t(255));
    }
    return total + 256;
}

// Build the job tables of every phase.  Returns the launch records and the
// job blob (device offsets relative to the table buffer).
static void plan_batch(const plu_batch_problem* P, int count, int prec, char* ws, Builder& B) {
    const int tc32 = prec == PLU_FP32 ? 1 : 0;
    std::vector<ProbWs> W(count);
    char* cur = ws;
    for (int i = 0; i < count; ++i) {
        const int64_t m = P[i].m, n = P[i].n, mx = m > n ? m : n;
        const int64_t l = P[i].algo == 1 ? P[i].k : P[i].l, k = P[i].k;
        double* d = reinterpret_cast<double*>(cur);
        ProbWs& w = W[i];
        w.V = d; d += n * l;
        w.Z = d; d += m * l;
        w.X2 = d; d += mx * l;
        w.L1 = d; d += m * k;
        w.U1T = d; d += k * k;
        w.BT = d; d += n * k;
        w.U2T = d; d += k * k;
        w.W = d; d += l * l;
        w.Wsave = d; d += l * l;
        w.Rinv = d; d += l * l;
        w.Rinv1 = d; d += l * l;
        w.T = d; d += l * l;
        d += k * k;
        cur += (size_t(reinterpret_cast<char*>(d) - cur) + 255) & ~size_t(255);
        int* ip = reinterpret_cast<int*>(cur);
        w.pos = ip;
        w.piv = ip + mx;
        w.info = ip + 2 * mx;
        w.qskip = ip + 2 * mx + 2;
        cur += (size_t(2 * mx + 4) * sizeof(int) + 255) & ~size_t(255);
    }
    // per-problem op lists
    std::vector<std::vector<Op>> ops(count);
    for (int i = 0; i < count; ++i) {
        const plu_batch_problem& p = P[i];
        ProbWs& w = W[i];
        const int64_t m = p.m, n = p.n;
        std::vector<Op>& L = ops[i];
        auto gauss = [&](double* out, int64_t rows, int cols, uint32_t st) {
            Op o{}; o.kind = OP_GAUSS; o.g_out = out; o.g_rows = rows; o.g_cols = cols; o.g_stream = st;
            L.push_back(o);
        };
        auto pass = [&](int trans, const double* X, int64_t ldx, double* Y, int64_t ldy, int cols) {
            Op o{}; o.kind = OP_PASS; o.trans = trans; o.X = X; o.ldx = ldx; o.Y = Y; o.ldy = ldy;
            o.cols = cols;
            L.push_back(o);
        };
        auto lu = [&](double* X, int64_t rows) { Op o{}; o.kind = OP_LU; o.P = X; o.prow = rows; L.push_back(o); };
        auto qr = [&](double* X, int64_t rows) { Op o{}; o.kind = OP_QR; o.P = X; o.prow = rows; L.push_back(o); };
        if (p.algo == 1) {
            gauss(w.X2, m, p.k, 3);
            pass(1, w.X2, m, w.V, n, p.k);          // G = A^T Omega
            pass(0, w.V, n, w.Z, m, p.k);           // H = A G
            Op o{}; o.kind = OP_SPTAIL; L.push_back(o);
            continue;
        }
        const int v = p.v, pp = (v - 1) / 2;
        if (v % 2 == 0) {
            gauss(w.Z, m, p.l, 2);
            pass(1, w.Z, m, w.V, n, p.l);
            if (v > 2) lu(w.V, n);
            else qr(w.V, n);
        } else {
            gauss(w.V, n, p.l, 1);
        }
        for (int it = 1; it <= pp; ++it) {
            pass(0, w.V, n, w.Z, m, p.l);
            lu(w.Z, m);
            pass(1, w.Z, m, w.V, n, p.l);
            if (it == pp) qr(w.V, n);
            else lu(w.V, n);
        }
        pass(0, w.V, n, w.Z, m, p.k);               // Y = A V(:, 1:k)
        Op o{}; o.kind = OP_TAIL; L.push_back(o);
    }
    size_t nph = 0;
    for (auto& L : ops) nph = std::max(nph, L.size());
    // the tails line up at the last phase
    for (auto& L : ops) {
        while (L.size() < nph) L.insert(L.end() - 2, Op{-1});
    }
    std::vector<GaussJob> gj;
    std::vector<GemmJob> gm;
    std::vector<LuJob> lj;
    std::vector<CholJob> cj;
    std::vector<TrinvJob> tj;
    for (size_t ph = 0; ph < nph; ++ph) {
        // Gaussians and passes
        for (int i = 0; i < count; ++i) {
            const Op& o = ops[i][ph];
            const plu_batch_problem& p = P[i];
            if (o.kind == OP_GAUSS)
                gj.push_back(GaussJob{o.g_out, o.g_rows, o.g_rows, o.g_cols, uint32_t(p.seed),
                                      uint32_t(p.seed >> 32), o.g_stream});
            if (o.kind == OP_PASS) {
                const int M = int(o.trans ? p.n : p.m), K = int(o.trans ? p.m : p.n);
                gm.push_back(mk_gemm(p.A, p.ld, p.dtype == PLU_F32, o.trans, o.X, o.ldx, 0, o.Y,
                                     o.ldy, M, o.cols, K));
            }
        }
        B.gauss(gj);
        B.gemm(gm, tc32);
        // LU re-orthogonalisation
        for (int i = 0; i < count; ++i) {
            const Op& o = ops[i][ph];
            if (o.kind == OP_LU)
                lj.push_back(mk_lu(o.P, o.prow, P[i].l, 0, nullptr, nullptr, 0, 0, nullptr, 0, 0,
                                   nullptr, W[i].pos, W[i].piv));
        }
        B.lu(lj);
        // CholeskyQR2 (two rounds: X2 = X R1^-1, X = X2 R2^-1).  With FP32
        // passes the second round is skipped, per problem on the device, when
        // R1's diagonal spread is at most 1e5 (as the mixed modes of
        // plu_powerlu do): its Gram, Cholesky and inverse return at once and
        // its X R^-1 becomes the copy X = X2.  FP64 batches keep both rounds.
        bool anyqr = false;
        for (int i = 0; i < count; ++i) anyqr |= ops[i][ph].kind == OP_QR;
        if (anyqr) {
            for (int round = 0; round < 2; ++round) {
                for (int i = 0; i < count; ++i) {
                    const Op& o = ops[i][ph];
                    if (o.kind != OP_QR) continue;
                    const int l = P[i].l;
                    const double* src = round == 0 ? o.P : W[i].X2;
                    gm.push_back(mk_gemm(src, o.prow, 0, 1, src, o.prow, 0, W[i].W, l, l, l,
                                         int(o.prow), 0, 1));
                    if (round == 1 && tc32) gm.back().skip = W[i].qskip;
                }
                B.gemm(gm, 0);
                for (int i = 0; i < count; ++i)
                    if (ops[i][ph].kind == OP_QR)
                        cj.push_back(CholJob{W[i].W, W[i].Wsave, P[i].l, ops[i][ph].prow,
                                             round == 1 && tc32 ? W[i].qskip : nullptr,
                                             round == 0 && tc32 ? W[i].qskip : nullptr});
                B.chol(cj);
                for (int i = 0; i < count; ++i)
                    if (ops[i][ph].kind == OP_QR)
                        tj.push_back(TrinvJob{W[i].W, W[i].Rinv, P[i].l,
                                              round == 1 && tc32 ? W[i].qskip : nullptr});
                B.trinv(tj);
                for (int i = 0; i < count; ++i) {
                    const Op& o = ops[i][ph];
                    if (o.kind != OP_QR) continue;
                    const int l = P[i].l;
                    const double* src = round == 0 ? o.P : W[i].X2;
                    double* dst = round == 0 ? W[i].X2 : o.P;
                    gm.push_back(mk_gemm(src, o.prow, 0, 0, W[i].Rinv, l, 0, dst, o.prow,
                                         int(o.prow), l, l, 0, 2));
                    if (round == 1 && tc32) {
                        gm.back().skip = W[i].qskip;
                        gm.back().copy_on_skip = 1;
                    }
                }
                B.gemm(gm, 0);
            }
        }
        // tails (the last phase)
        bool anytail = false, anysp = false;
        for (int i = 0; i < count; ++i) {
            anytail |= ops[i][ph].kind == OP_TAIL;
            anysp |= ops[i][ph].kind == OP_SPTAIL;
        }
        if (anysp) {
            // single pass: G = Q R (CholeskyQR2 of G in V, keeping R^-1 = R1^-1 R2^-1),
            // G^{dagger T} = Q R^-T, then the tail on M = G^{dagger T} U1^T
            for (int round = 0; round < 2; ++round) {
                for (int i = 0; i < count; ++i) {
                    if (ops[i][ph].kind != OP_SPTAIL) continue;
                    const int k = P[i].k;
                    const int64_t n = P[i].n;
                    const double* src = round == 0 ? W[i].V : W[i].X2;
                    gm.push_back(mk_gemm(src, n, 0, 1, src, n, 0, W[i].W, k, k, k, int(n), 0, 1));
                }
                B.gemm(gm, 0);
                for (int i = 0; i < count; ++i)
                    if (ops[i][ph].kind == OP_SPTAIL)
                        cj.push_back(CholJob{W[i].W, W[i].Wsave, P[i].k, P[i].n, nullptr, nullptr});
                B.chol(cj);
                for (int i = 0; i < count; ++i)
                    if (ops[i][ph].kind == OP_SPTAIL)
                        tj.push_back(TrinvJob{W[i].W, round == 0 ? W[i].Rinv1 : W[i].Rinv, P[i].k,
                                              nullptr});
                B.trinv(tj);
                for (int i = 0; i < count; ++i) {
                    if (ops[i][ph].kind != OP_SPTAIL) continue;
                    const int k = P[i].k;
                    const int64_t n = P[i].n;
                    const double* src = round == 0 ? W[i].V : W[i].X2;
                    double* dst = round == 0 ? W[i].X2 : W[i].V;
                    const double* Ri = round == 0 ? W[i].Rinv1 : W[i].Rinv;
                    gm.push_back(mk_gemm(src, n, 0, 0, Ri, k, 0, dst, n, int(n), k, k, 0, 2));
                }
                B.gemm(gm, 0);
            }
            // T = R1^-1 R2^-1 (both upper triangular); BT = Q T^T
            for (int i = 0; i < count; ++i)
                if (ops[i][ph].kind == OP_SPTAIL) {
                    const int k = P[i].k;
                    gm.push_back(mk_gemm(W[i].Rinv1, k, 0, 0, W[i].Rinv, k, 0, W[i].T, k, k, k, k));
                }
            B.gemm(gm, 0);
            for (int i = 0; i < count; ++i)
                if (ops[i][ph].kind == OP_SPTAIL) {
                    const int k = P[i].k;
                    gm.push_back(mk_gemm(W[i].V, P[i].n, 0, 0, W[i].T, k, 1, W[i].BT, P[i].n,
                                         int(P[i].n), k, k));
                }
            B.gemm(gm, tc32);
        }
        if (anytail || anysp) {
            // [L1, U1, P] = lu(Y)   (Y = A V_k, or H for the single pass; in Z)
            for (int i = 0; i < count; ++i) {
                const int kd = ops[i][ph].kind;
                if (kd != OP_TAIL && kd != OP_SPTAIL) continue;
                const int k = P[i].k;
                lj.push_back(mk_lu(W[i].Z, P[i].m, k, 1, P[i].p, W[i].L1, P[i].m, 0, W[i].U1T, k, 1,
                                   W[i].info, W[i].pos, W[i].piv));
            }
            B.lu(lj);
            // B^T = V_k U1^T (PowerLU) or M = G^{dagger T} U1^T (single pass), into X2
            for (int i = 0; i < count; ++i) {
                const int kd = ops[i][ph].kind;
                if (kd != OP_TAIL && kd != OP_SPTAIL) continue;
                const int k = P[i].k;
                const double* left = kd == OP_TAIL ? W[i].V : W[i].BT;
                gm.push_back(mk_gemm(left, P[i].n, 0, 0, W[i].U1T, k, 0, W[i].X2, P[i].n,
                                     int(P[i].n), k, k));
            }
            // the m x k x k products of the tail take FP32 FMAs with FP32 passes
            // (the passes' rounding dominates); the LUs stay FP64
            B.gemm(gm, tc32);
            // [L2, U2, Q] = lu(B^T), U = L2^T
            for (int i = 0; i < count; ++i) {
                const int kd = ops[i][ph].kind;
                if (kd != OP_TAIL && kd != OP_SPTAIL) continue;
                const int k = P[i].k;
                lj.push_back(mk_lu(W[i].X2, P[i].n, k, 1, P[i].q, P[i].U, P[i].ldU, 1, W[i].U2T, k,
                                   1, W[i].info + 1, W[i].pos, W[i].piv));
            }
            B.lu(lj);
            // L = L1 U2^T
            for (int i = 0; i < count; ++i) {
                const int kd = ops[i][ph].kind;
                if (kd != OP_TAIL && kd != OP_SPTAIL) continue;
                const int k = P[i].k;
                gm.push_back(mk_gemm(W[i].L1, P[i].m, 0, 0, W[i].U2T, k, 0, P[i].L, P[i].ldL,
                                     int(P[i].m), k, k));
            }
            B.gemm(gm, tc32);
        }
    }
}

cudaError_t launch_batch_plan(const Builder& B, const char* dtab, int* dev_status, int num_sms,
                              cudaStream_t s) {
    (void)num_sms;
    for (const LaunchRec& r : B.recs) {
        const char* tab = dtab + r.off;
        cudaError_t e = cudaSuccess;
        count_launch();
        switch (r.kind) {
            case 0:
                k_b_gaussian<<<dim3(32, unsigned(r.njobs)), 256, 0, s>>>(
                    reinterpret_cast<const GaussJob*>(tab));
                break;
            case 1:
                e = launch_b_gemm(r.variant % kGemmVariants, r.tc32,
                                  reinterpret_cast<const GemmJob*>(tab), r.njobs, r.tiles, s);
                if (e != cudaSuccess) return e;
                if (r.red_jobs > 0) {
                    count_launch();
                    k_b_splitk_reduce<<<unsigned((r.red_elems + 255) / 256), 256, 0, s>>>(
                        reinterpret_cast<const RedJob*>(dtab + r.red_off), r.red_jobs,
                        r.red_elems);
                }
                break;
            case 2:
                k_b_panel_lu<<<unsigned(r.njobs), LNT, size_t(r.maxn) * sizeof(double), s>>>(
                    reinterpret_cast<const LuJob*>(tab));
                break;
            case 5: {
                // zero the groups' counters and slots, then one cooperative
                // launch (its CTAs wait on one another, so they must all be
                // resident)
                e = cudaMemsetAsync(const_cast<char*>(dtab) + r.zero_off, 0, r.zero_bytes, s);
                if (e != cudaSuccess) return e;
                const LuJob* jt = reinterpret_cast<const LuJob*>(tab);
                const McCta* ct = reinterpret_cast<const McCta*>(dtab + r.cta_off);
                const McSync* sy = reinterpret_cast<const McSync*>(dtab + r.sync_off);
                unsigned char* bp = reinterpret_cast<unsigned char*>(const_cast<char*>(dtab));
                int64_t budget = kBatchSpin;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(unsigned(r.nctas));
                cfg.blockDim = dim3(LNT);
                cfg.dynamicSmemBytes = size_t(r.maxn) * sizeof(double);
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, k_b_panel_lu_mc, jt, ct, sy, bp, dev_status, budget);
                if (e != cudaSuccess) return e;
                break;
            }
            case 3:
                k_b_cholesky<<<unsigned(r.njobs), CNT, 0, s>>>(reinterpret_cast<const CholJob*>(tab),
                                                              dev_status);
                break;
            case 4:
                k_b_trinv<<<dim3(unsigned(r.maxn), unsigned(r.njobs)), 128,
                            2 * size_t(r.maxn) * sizeof(double), s>>>(
                    reinterpret_cast<const TrinvJob*>(tab));
                break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The split-K partials live in a device buffer owned by the caller's
// context, grown here when a plan needs more (after the stream drains).
static cudaError_t grow_part(double** part, size_t* cap, int64_t elems, cudaStream_t s) {
    const size_t need = size_t(elems > 0 ? elems : 1) * sizeof(double);
    if (need <= *cap && *part) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*part) cudaFree(*part);
    *part = nullptr;
    *cap = 0;
    if ((e = cudaMalloc(reinterpret_cast<void**>(part), need)) != cudaSuccess) return e;
    *cap = need;
    return cudaSuccess;
}

// Plan, upload the job tables, capture the grouped launches in a CUDA graph
// and launch it.  `tables` must hold batch_tables_bytes() bytes.
// The autotuner: every grouped GEMM of the plan is timed alone (with its
// split-K reduction) for each tile shape and split-K choice on its real job
// list (CUDA events, the better of two runs after one warm-up; the operands
// may hold anything then, as the graph recomputes every phase in order
// afterwards), and the fastest choice is kept.
cudaError_t tune_gemms(Builder& B, char* tables, size_t tables_cap, cudaStream_t s,
                       std::vector<int>* tuned, double** part, size_t* part_cap) {
    const size_t base = (B.blob.size() + 255) & ~size_t(255);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cudaErrorUnknown;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cudaErrorUnknown;
    }
    tuned->assign(B.gjobs.size(), 0);
    cudaError_t e = cudaSuccess;
    for (const LaunchRec& r : B.recs) {
        if (r.kind != 1) continue;
        std::vector<GemmJob> jobs = B.gjobs[r.gidx];
        float best = 0.f;
        for (int v = 0; v < kGemmChoices && e == cudaSuccess; ++v) {
            int64_t pe = 0;
            lay_tiles(jobs, v, nullptr, &pe, nullptr);
            // a split choice that splits nothing repeats the unsplit one
            if (v >= kGemmVariants && pe == 0) continue;
            if ((e = grow_part(part, part_cap, pe, s)) != cudaSuccess) break;
            std::vector<RedJob> red;
            const int64_t tiles = lay_tiles(jobs, v, *part, &pe, &red);
            const size_t bytes = jobs.size() * sizeof(GemmJob);
            const size_t roff = (base + bytes + 255) & ~size_t(255);
            const size_t rbytes = red.size() * sizeof(RedJob);
            if (roff + rbytes > tables_cap) {
                e = cudaErrorInvalidValue;
                break;
            }
            GemmJob* tab = reinterpret_cast<GemmJob*>(tables + base);
            RedJob* rtab = reinterpret_cast<RedJob*>(tables + roff);
            if ((e = cudaMemcpyAsync(tab, jobs.data(), bytes, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess)
                break;
            if (rbytes && (e = cudaMemcpyAsync(rtab, red.data(), rbytes, cudaMemcpyHostToDevice,
                                               s)) != cudaSuccess)
                break;
            const int64_t relems =
                red.empty() ? 0 : red.back().elem0 + int64_t(red.back().M) * red.back().N;
            float t_v = 0.f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, s);
                e = launch_b_gemm(v % kGemmVariants, r.tc32, tab, int(jobs.size()), tiles, s);
                if (e == cudaSuccess && !red.empty()) {
                    k_b_splitk_reduce<<<unsigned((relems + 255) / 256), 256, 0, s>>>(
                        rtab, int(red.size()), relems);
                    e = cudaGetLastError();
                }
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1 || (rep == 2 && ms < t_v)) t_v = ms;
            }
            if (v == 0 || t_v < best) {
                best = t_v;
                (*tuned)[r.gidx] = v;
            }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t run_batch(const plu_batch_problem* P, int count, int prec, char* ws, char* tables,
                      size_t tables_cap, int* dev_status, int num_sms, cudaStream_t s,
                      cudaStream_t cs, int* nlaunch, float* ms_graph, std::vector<int>* tuned,
                      int forced, double** part, size_t* part_cap) {
    Builder B;
    {
        // the multi-CTA LU's CTAs must all be resident at once
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_b_panel_lu_mc, LNT,
                                                          size_t(1024) * sizeof(double)) !=
            cudaSuccess)
            nb = 0;
        B.mc_cap = nb * num_sms;
    }
    plan_batch(P, count, prec, ws, B);
    if (forced >= 0) {
        if (forced >= kGemmVariants) return cudaErrorInvalidValue;
        tuned->assign(B.gjobs.size(), forced);
    } else if (tuned->size() != B.gjobs.size()) {
        const cudaError_t te = tune_gemms(B, tables, tables_cap, s, tuned, part, part_cap);
        if (te != cudaSuccess) return te;
    }
    for (int c : *tuned)
        if (c < 0 || c >= kGemmChoices) return cudaErrorInvalidValue;
    {
        // the partial region the chosen split-K needs, then the placement
        Builder dry = B;
        const int64_t need = dry.place_gemms(*tuned, nullptr);
        const cudaError_t ge = grow_part(part, part_cap, need, s);
        if (ge != cudaSuccess) return ge;
    }
    B.place_gemms(*tuned, *part);
    if (B.blob.size() > tables_cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(tables, B.blob.data(), B.blob.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long long before = g_launches;
    cudaError_t le = launch_batch_plan(B, tables, dev_status, num_sms, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le;
    }
    if (e != cudaSuccess) return e;
    *nlaunch = int(g_launches - before);
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return e;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    e = cudaGraphLaunch(exec, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_graph = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return e;
}

size_t batch_tables_bytes(int count) {
    // generous: every phase's tables for all problems, and room for the
    // autotuner's trial table
    return size_t(count) * 72 * sizeof(GemmJob) + (1 << 20);
}

int batch_gemm_tile(int choice, int* bm, int* bn) {
    if (choice < 0 || choice >= kGemmChoices) return 0;
    *bm = kVarBM[choice % kGemmVariants];
    *bn = kVarBN[choice % kGemmVariants];
    return 1;
}

int batch_gemm_splitk(int choice) {
    if (choice < 0 || choice >= kGemmChoices) return -1;
    return kSplitK[choice / kGemmVariants];
}

int batch_gemm_choices() { return kGemmChoices; }

}  // namespace plu
