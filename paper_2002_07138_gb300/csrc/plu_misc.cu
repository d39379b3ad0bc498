// Reductions of the fixed-precision path and small helpers.
//
// ||A||_F^2 (Alg. adaptivewithoutupdating step 1) and the squared column
// norms of G = A V (its step 7) are accumulated in FP64 in a fixed order
// (per-thread strided sums, then a tree in shared memory, then the per-CTA
// partials in CTA order), so they do not depend on scheduling.  The rank scan
// (the loop of Alg. adaptivewithoutupdating, or the per-column loop of
// Sec. 6.4) is a single thread over the <= a few hundred column norms:
// E <- E - ||G(:, t1:t2)||_F^2 until E <= eps^2 ||A||_F^2.
#include "plu_internal.h"

namespace plu {
namespace {

constexpr int RT = 256;

__device__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double out = sh[0];
    __syncthreads();
    return out;
}

template <typename T>
__global__ void __launch_bounds__(RT)
k_norm2_partial(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                double* __restrict__ part) {
    __shared__ double sh[RT];
    double acc = 0.0;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const T* col = A + j * lda;
        for (int64_t i = threadIdx.x; i < m; i += RT) {
            const double x = double(col[i]);
            acc = fma(x, x, acc);
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Sum of squares of a flat array (the nonzeros of a sparse A): CTA b sums
// the entries b*RT + t + i*gridDim.x*RT in a fixed order.
__global__ void __launch_bounds__(RT)
k_sumsq_partial(const double* __restrict__ x, int64_t count, double* __restrict__ part) {
    __shared__ double sh[RT];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * int64_t(RT) + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * RT)
        acc = fma(x[i], x[i], acc);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ part, int count, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < count; ++i) s += part[i];
        *out = s;
    }
}

// *out = sum of part[0 .. count): thread t adds part[t], part[t + 1024], ...,
// then a fixed tree over the threads (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024)
k_sum_partials_wide(const double* __restrict__ part, int count, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 1024) s += part[i];
    s = cta_sum(s);
    if (threadIdx.x == 0) *out = s;
}

__global__ void __launch_bounds__(RT)
k_colnorm2(int64_t rows, const double* __restrict__ G, int64_t ldg, double* __restrict__ out) {
    __shared__ double sh[RT];
    const double* col = G + int64_t(blockIdx.x) * ldg;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += RT) acc = fma(col[i], col[i], acc);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void k_rank_scan(const double* __restrict__ cn, int cols, const double* __restrict__ normA2,
                            const double* __restrict__ E_start, double eps, int b, int precise,
                            int* __restrict__ k_met, double* __restrict__ E_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double E = E_start ? *E_start : *normA2;
    const double acc = eps * eps * *normA2;
    int k = 0, met = 0;
    for (int t1 = 0; t1 < cols && !met; t1 += b) {
        const int t2 = min(cols, t1 + b);
        if (precise) {
            for (int j = t1; j < t2; ++j) {
                E -= cn[j];
                k = j + 1;
                if (E <= acc) { met = 1; break; }
            }
        } else {
            double s = 0.0;
            for (int j = t1; j < t2; ++j) s += cn[j];
            E -= s;
            k = t2;
            if (E <= acc) met = 1;
        }
    }
    k_met[0] = k;
    k_met[1] = met;
    *E_out = E;
}

__global__ void k_copy_cols(int64_t rows, int cols, const double* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        dst[i + j * ldd] = src[i + j * lds];
    }
}

// CTA row blockIdx.y = column j; x strides over the rows.
__global__ void k_scatter_rows(int64_t rows, const int32_t* __restrict__ perm,
                               const double* __restrict__ L, int64_t ldl, double* __restrict__ W,
                               int64_t ldw) {
    const int64_t j = blockIdx.y;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t r = perm[i];
        if (r >= 0 && r < rows) W[r + j * ldw] = L[i + j * ldl];
    }
}

}  // namespace

size_t norm2_scratch_bytes(int num_sms) { return size_t(num_sms) * 4 * sizeof(double) + 256; }

cudaError_t launch_sum_partials(const double* part, int count, double* out, cudaStream_t s) {
    if (count < 0 || !out || (count > 0 && !part)) return cudaErrorInvalidValue;
    count_launch();
    k_sum_partials_wide<<<1, 1024, 0, s>>>(part, count, out);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* x, int64_t count, double* out, void* scratch,
                         int num_sms, cudaStream_t s) {
    if (count < 0 || (count > 0 && !x)) return cudaErrorInvalidValue;
    int64_t blocks = (count + RT - 1) / RT;
    if (blocks > int64_t(num_sms) * 4) blocks = int64_t(num_sms) * 4;
    if (blocks < 1) blocks = 1;
    double* part = static_cast<double*>(scratch);
    count_launch();
    k_sumsq_partial<<<unsigned(blocks), RT, 0, s>>>(x, count, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_sum_partials<<<1, 32, 0, s>>>(part, int(blocks), out);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const void* A, int dtype, int64_t m, int64_t n, int64_t lda,
                         double* out, void* scratch, int num_sms, cudaStream_t s) {
    int blocks = num_sms * 4;
    if (blocks > n) blocks = int(n > 0 ? n : 1);
    double* part = static_cast<double*>(scratch);
    count_launch();
    if (dtype == PLU_F32)
        k_norm2_partial<float><<<blocks, RT, 0, s>>>(static_cast<const float*>(A), m, n, lda, part);
    else
        k_norm2_partial<double><<<blocks, RT, 0, s>>>(static_cast<const double*>(A), m, n, lda, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_sum_partials<<<1, 32, 0, s>>>(part, blocks, out);
    return cudaGetLastError();
}

cudaError_t launch_colnorm2(int64_t rows, int cols, const double* G, int64_t ldg, double* out,
                            cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    count_launch();
    k_colnorm2<<<cols, RT, 0, s>>>(rows, G, ldg, out);
    return cudaGetLastError();
}

cudaError_t launch_rank_scan(const double* colnorm2, int cols, const double* normA2, double eps,
                             int b, int precise, int* k_met, double* E_out, cudaStream_t s,
                             const double* E_start) {
    count_launch();
    k_rank_scan<<<1, 32, 0, s>>>(colnorm2, cols, normA2, E_start, eps, b, precise, k_met, E_out);
    return cudaGetLastError();
}

cudaError_t launch_copy_cols(int64_t rows, int cols, const double* src, int64_t lds, double* dst,
                             int64_t ldd, cudaStream_t s) {
    const int64_t total = rows * int64_t(cols);
    if (total <= 0) return cudaSuccess;
    int64_t b = (total + 255) / 256;
    if (b > 4096) b = 4096;
    count_launch();
    k_copy_cols<<<unsigned(b), 256, 0, s>>>(rows, cols, src, lds, dst, ldd);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows(int64_t rows, int cols, const int32_t* perm, const double* L,
                                int64_t ldl, double* W, int64_t ldw, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (cols > 65535) return cudaErrorInvalidValue;
    int64_t b = (rows + 255) / 256;
    if (b > 64) b = 64;
    count_launch();
    k_scatter_rows<<<dim3(unsigned(b), unsigned(cols)), 256, 0, s>>>(rows, perm, L, ldl, W, ldw);
    return cudaGetLastError();
}

}  // namespace plu
