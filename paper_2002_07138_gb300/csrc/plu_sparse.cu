// Passes over a sparse A (the sparse experiment of Sec. 6 uses MATLAB sprand
// matrices): Y = S X, S in CSR (the CSR of A for A X, the CSR of A^T for
// A^T X), X and Y dense column-major, FP64.
//
// X is first copied to row-major (row stride xs = cols rounded up to even,
// the pad column zero), so that a half-warp reads one contiguous stretch of
// a row of X per nonzero.  A CTA owns 32 rows of Y and a warp one row at a
// time: its nonzeros' indices and values are loaded 32 at a time and
// broadcast by shuffles, the two half-warps take alternate nonzeros (each
// lane owning every 16th column), and the halves' sums are added at the end
// -- a fixed order, so the result does not depend on the launch.  The pass
// issues one FP64 FMA per nonzero and column, and GB300's FP64 pipe is its
// bound: the 16-column granularity keeps the issued FMAs within 16 columns
// of the useful ones (l = 200: 208 of 200).  The 32 rows are staged in
// shared memory and written to the column-major Y in 256-byte column
// segments.  A column index outside [0, K) or a row pointer outside [0, nnz]
// sets DEV_BADINDEX in the status word and the entry is skipped.
#include "plu_internal.h"

namespace plu {
namespace {

constexpr int SP_ROWS = 32;       // rows of Y per CTA
constexpr int SP_WARPS = 8;
constexpr int SP_CHUNK = 208;     // columns of Y per sweep of a row (13 per lane)
constexpr int SP_SMEM = SP_ROWS * (SP_CHUNK + 1) * int(sizeof(double));
constexpr int SP_CTAS_PER_SM = 2;   // 124 registers x 256 threads: two CTAs an SM

// Xr (K x xs, row-major) = X (K x cols, column-major, ld); Xr[r * xs + cols]
// is zeroed when xs > cols.
__global__ void k_to_rowmajor(int64_t K, int cols, int xs, const double* __restrict__ X,
                              int64_t ld, double* __restrict__ Xr) {
    __shared__ double tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32;
    const int c0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int64_t r = r0 + threadIdx.x;
        const int c = c0 + q;
        tile[q][threadIdx.x] = (r < K && c < cols) ? X[r + int64_t(c) * ld] : 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int64_t r = r0 + q;
        const int c = c0 + threadIdx.x;
        if (r < K && c < xs) Xr[r * xs + c] = tile[threadIdx.x][q];
    }
}

__device__ __forceinline__ void flag_bad_index(int* status) {
    atomicCAS(status, DEV_OK, DEV_BADINDEX);
}

__global__ void __launch_bounds__(SP_WARPS * 32, SP_CTAS_PER_SM)
k_spmm_csr(int64_t rows, int64_t K, int64_t nnz, int cols, int xs,
           const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
           const double* __restrict__ val, const double* __restrict__ Xr,
           double* __restrict__ Y, int64_t ldy, int* status, double* __restrict__ norm_parts) {
    // norm_parts (nullable): the CTA's sum of the squared values it reads
    // (in the first column chunk, where every nonzero is read once)
    double nsq = 0.0;
    extern __shared__ double ys[];            // SP_ROWS x (SP_CHUNK + 1)
    constexpr int YS = SP_CHUNK + 1;
    constexpr int NCM = SP_CHUNK / 16;        // column slots of a lane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the two half-warps take alternate nonzeros; lane `sub` of a half owns
    // the columns sub, sub + 16, ... of the chunk
    const int grp = lane >> 4, sub = lane & 15;
    const unsigned full = 0xffffffffu;
    for (int64_t R0 = int64_t(blockIdx.x) * SP_ROWS; R0 < rows;
         R0 += int64_t(gridDim.x) * SP_ROWS) {
        for (int c0 = 0; c0 < cols; c0 += SP_CHUNK) {
            const int ch = cols - c0 < SP_CHUNK ? cols - c0 : SP_CHUNK;
            const int nc = (ch + 15) >> 4;    // slots in use: a warp-uniform bound,
                                              // so unused slots issue no FMA
            for (int rr = warp; rr < SP_ROWS; rr += SP_WARPS) {
                const int64_t r = R0 + rr;
                double acc[NCM];
#pragma unroll
                for (int i = 0; i < NCM; ++i) acc[i] = 0.0;
                if (r < rows) {
                    int64_t b = row_ptr[r], e = row_ptr[r + 1];
                    if (b < 0 || e > nnz || b > e) {
                        if (lane == 0) flag_bad_index(status);
                        b = e = 0;
                    }
                    const double* xbase = Xr + c0 + sub;
                    for (int64_t t0 = b; t0 < e; t0 += 32) {
                        const int64_t t = t0 + lane;
                        int col = 0;
                        double a = 0.0;
                        if (t < e) {
                            col = col_idx[t];
                            a = val[t];
                            if (col < 0 || int64_t(col) >= K) {
                                flag_bad_index(status);
                                col = 0;
                                a = 0.0;
                            }
                            if (norm_parts && c0 == 0) nsq = fma(a, a, nsq);
                        }
                        const int cnt = e - t0 < 32 ? int(e - t0) : 32;
                        // 2 nonzeros per step, one per half-warp
                        for (int j0 = 0; j0 < cnt; j0 += 2) {
                            const int j = j0 + grp;
                            const int cj = __shfl_sync(full, col, j & 31);
                            const double av = __shfl_sync(full, a, j & 31);
                            const double aj = j < cnt ? av : 0.0;
                            const double* xr = xbase + int64_t(j < cnt ? cj : 0) * xs;
                            double x[NCM];
#pragma unroll
                            for (int i = 0; i < NCM; ++i)
                                if (i < nc) x[i] = (sub + 16 * i < ch) ? xr[16 * i] : 0.0;
#pragma unroll
                            for (int i = 0; i < NCM; ++i)
                                if (i < nc) acc[i] = fma(aj, x[i], acc[i]);
                        }
                    }
                }
                // the second half-warp's sums join the first's
#pragma unroll
                for (int i = 0; i < NCM; ++i)
                    if (i < nc) acc[i] += __shfl_down_sync(full, acc[i], 16);
                if (grp == 0) {
                    double* yrow = ys + rr * YS;
#pragma unroll
                    for (int i = 0; i < NCM; ++i) {
                        const int c = sub + 16 * i;
                        if (i < nc && c < ch) yrow[c] = acc[i];
                    }
                }
            }
            __syncthreads();
            // column-major write-out: a warp writes 32 consecutive rows of one column
            const int nr = rows - R0 < SP_ROWS ? int(rows - R0) : SP_ROWS;
            for (int i = threadIdx.x; i < SP_ROWS * ch; i += SP_WARPS * 32) {
                const int rr = i & 31, c = i >> 5;
                if (rr < nr) Y[R0 + rr + int64_t(c0 + c) * ldy] = ys[rr * YS + c];
            }
            __syncthreads();
        }
    }
    if (norm_parts) {
        const double tot = cta_sum(nsq);
        if (threadIdx.x == 0) norm_parts[blockIdx.x] = tot;
    }
}

}  // namespace

int spmm_row_stride(int cols) { return (cols + 1) & ~1; }

size_t spmm_scratch_bytes(int64_t K, int cols) {
    return size_t(K) * size_t(spmm_row_stride(cols)) * sizeof(double) + 256;
}

cudaError_t launch_spmm_csr(int64_t rows, int64_t K, int64_t nnz, const int64_t* row_ptr,
                            const int32_t* col_idx, const double* val, const double* X,
                            int64_t ldx, int cols, double* Y, int64_t ldy, void* scratch,
                            size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s,
                            const NormOut* norm) {
    if (rows < 1 || K < 1 || cols < 1 || nnz < 0 || !row_ptr || !X || !Y || !dev_status)
        return cudaErrorInvalidValue;
    if (nnz > 0 && (!col_idx || !val)) return cudaErrorInvalidValue;
    if (ldx < K || ldy < rows || cols > 65535 * 32) return cudaErrorInvalidValue;
    if ((K + 31) / 32 > 2147483647LL) return cudaErrorInvalidValue;
    if (scratch_cap < spmm_scratch_bytes(K, cols)) return cudaErrorInvalidValue;
    const int xs = spmm_row_stride(cols);
    double* Xr = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(scratch) + 255) &
                                           ~uintptr_t(255));
    cudaError_t e =
        cudaFuncSetAttribute(k_spmm_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, SP_SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    k_to_rowmajor<<<dim3(unsigned((K + 31) / 32), unsigned((xs + 31) / 32)), dim3(32, 8), 0, s>>>(
        K, cols, xs, X, ldx, Xr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int64_t blocks = (rows + SP_ROWS - 1) / SP_ROWS;
    const int64_t cap = int64_t(num_sms) * SP_CTAS_PER_SM;
    if (blocks > cap) blocks = cap;
    if (norm && (!norm->parts || !norm->out || blocks > norm->cap)) return cudaErrorInvalidValue;
    count_launch();
    k_spmm_csr<<<unsigned(blocks), SP_WARPS * 32, SP_SMEM, s>>>(
        rows, K, nnz, cols, xs, row_ptr, col_idx, val, Xr, Y, ldy, dev_status,
        norm ? norm->parts : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (norm) return launch_sum_partials(norm->parts, int(blocks), norm->out, s);
    return cudaSuccess;
}

int spmm_norm_parts(int64_t rows, int num_sms) {
    const int64_t blocks = (rows + SP_ROWS - 1) / SP_ROWS;
    const int64_t cap = int64_t(num_sms) * SP_CTAS_PER_SM;
    return int(blocks < cap ? blocks : cap);
}

}  // namespace plu
