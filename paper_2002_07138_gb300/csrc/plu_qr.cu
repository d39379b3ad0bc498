// a5: the orthonormal basis [V, ~] = qr(A^T V) that closes Alg. gpowerlu.
//
// FP64 CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014):
//   W = X^T X, W = R1^T R1 (Cholesky), Q1 = X R1^{-1};
//   W = Q1^T Q1, W = R2^T R2,           Q  = Q1 R2^{-1};  R = R2 R1.
// Q equals the Q of the Householder QR with R_ii > 0 up to rounding for
// condition numbers below ~1e7 (the sketches here stay far below that); the
// Gram matrices and the products with R^{-1} are the skinny FP64 GEMMs of
// plu_gemm.cu.  If the first Cholesky meets a non-positive pivot it restarts
// with the shift 11 (rows*cols + cols*(cols+1)) u tr(W) of shifted
// CholeskyQR (Fukaya et al. 2020) and the second pass restores orthogonality;
// a breakdown of the second pass sets the numeric error word.
#include "plu_internal.h"

namespace plu {
namespace {

constexpr int CT = 1024;

// In-place upper Cholesky W = R^T R of the n x n SPD matrix W (ld n),
// one CTA.  The strictly lower triangle is zeroed.  shift_mode 1: on a
// non-positive pivot restart from Wsave with the CholeskyQR shift.
__global__ void __launch_bounds__(CT)
k_cholesky(int n, double* __restrict__ W, const double* __restrict__ Wsave, int64_t rows,
           int shift_mode, int* __restrict__ status, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ int broke;
    __shared__ double rjj;
    const int t = threadIdx.x;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            // tr(W) bounds ||X||_2^2; shift = 11 (rows n + n(n+1)) u tr(W)
            __shared__ double tr;
            if (t == 0) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) s += Wsave[i + int64_t(i) * n];
                tr = s;
            }
            __syncthreads();
            const double shift = 11.0 * (double(rows) * n + double(n) * (n + 1)) * 1.1102230246251565e-16 * tr;
            for (int64_t e = t; e < int64_t(n) * n; e += CT) {
                const int a = int(e % n), c = int(e / n);
                W[e] = Wsave[e] + (a == c ? shift : 0.0);
            }
            __syncthreads();
        }
        if (t == 0) broke = 0;
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            if (t == 0) {
                const double d = W[j + int64_t(j) * n];
                if (!(d > 0.0)) broke = 1;
                rjj = (d > 0.0) ? sqrt(d) : 1.0;
                W[j + int64_t(j) * n] = rjj;
            }
            __syncthreads();
            if (broke) break;
            const double inv = 1.0 / rjj;
            for (int c = j + 1 + t; c < n; c += CT) W[j + int64_t(c) * n] *= inv;
            __syncthreads();
            const int m = n - j - 1;
            for (int64_t e = t; e < int64_t(m) * m; e += CT) {
                const int a = j + 1 + int(e % m), c = j + 1 + int(e / m);
                if (a <= c) W[a + int64_t(c) * n] -= W[j + int64_t(a) * n] * W[j + int64_t(c) * n];
            }
            __syncthreads();
        }
        if (!broke) break;
        if (!shift_mode || attempt == 1) {
            if (t == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
            break;
        }
    }
    __syncthreads();
    for (int64_t e = t; e < int64_t(n) * n; e += CT) {
        const int a = int(e % n), c = int(e / n);
        if (a > c) W[e] = 0.0;
    }
}

// Blocked upper Cholesky W = R^T R over a cooperative grid (n x n, ld n,
// upper triangle read, R written over it, strictly lower part zeroed).
//
// The FP64 pipe of an SM issues one warp instruction about every 64 cycles
// per SM sub-partition, and a dependent FP64 operation waits as long (a
// reciprocal or square root, several operations, ~430 cycles), whether one
// lane or 32 are active.  So the n pivots, which are sequential, decide the
// time, and the kernel keeps per pivot one reciprocal and two CTA barriers
// on the critical path:
//  (A) every CTA factors the diagonal block redundantly in shared memory in
//      LDL^T form (thread 0 takes 1/d_j, all threads apply the rank-1 update
//      with it), then scales: R11 = diag(sqrt d) L^T with the square roots
//      taken in parallel.  No grid barrier is needed before the solves, as
//      every CTA holds R11 and 1/R11(j, j).
//  (B) R12 = R11^{-T} W12, one warp per column (lane i owns row i; x_u is
//      broadcast by a shuffle), grid barrier;
//  (C) W22 -= R12^T R12 (upper part), R12 staged in shared memory when it
//      fits, grid barrier.
// On a non-positive pivot in the first attempt (shift_mode 1) every CTA,
// having met it in its own copy of the diagonal block, restarts from Wsave
// with the shifted-CholeskyQR diagonal shift.
constexpr int CB = 32;
constexpr int CBT = 256;

struct CholCtl {
    unsigned barrier;
    int broke;
};

__global__ void __launch_bounds__(CBT)
k_cholesky_coop(int n, double* __restrict__ W, const double* __restrict__ Wsave, int64_t rows,
                int shift_mode, CholCtl* __restrict__ ctl, int* __restrict__ status,
                int64_t budget, int stage_rows, const int* __restrict__ skip) {
    if (skip && *skip) return;                      // every CTA reads the same flag
    extern __shared__ double S[];                 // [CB][n - kb - b] block rows of R12
    __shared__ double D[CB][CB + 1];
    __shared__ double zinv[CB];                   // 1 / d_j
    __shared__ double yinv[CB];                   // 1 / sqrt(d_j) = 1 / R11(j, j)
    __shared__ int bad;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int nb = gridDim.x;
    const int gtid = blockIdx.x * CBT + t;
    const int gthreads = nb * CBT;
    const int gwarp = blockIdx.x * (CBT / 32) + (t >> 5);
    const int gwarps = nb * (CBT / 32);
    unsigned nbar = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            double tr = 0.0;
            for (int i = 0; i < n; ++i) tr += Wsave[i + int64_t(i) * n];
            const double shift = 11.0 * (double(rows) * n + double(n) * (n + 1)) *
                                 1.1102230246251565e-16 * tr;
            for (int64_t e = gtid; e < int64_t(n) * n; e += gthreads) {
                const int a = int(e % n), c = int(e / n);
                W[e] = Wsave[e] + (a == c ? shift : 0.0);
            }
            if (!grid_barrier(&ctl->barrier, ++nbar * nb, status, budget)) return;
        }
        bool broke = false;
        for (int kb = 0; kb < n; kb += CB) {
            const int b = min(CB, n - kb);
            // (A) the diagonal block, in every CTA
            for (int e = t; e < CB * CB; e += CBT) {
                const int a = e % CB, c = e / CB;
                D[a][c] = (a <= c && c < b) ? __ldcg(&W[(kb + a) + int64_t(kb + c) * n]) : 0.0;
            }
            if (t == 0) bad = 0;
            __syncthreads();
            for (int j = 0; j < b; ++j) {
                if (t == 0) {
                    const double d = D[j][j];
                    if (!(d > 0.0)) bad = 1;
                    zinv[j] = d > 0.0 ? 1.0 / d : 0.0;
                }
                __syncthreads();
                if (bad) break;                     // the same value in every thread
                const double z = zinv[j];
                // D(a, c) -= D(j, a) D(j, c) / d_j for j < a <= c < b: thread t
                // takes columns c = j + 1 + (t % 32) .. and rows a in (j, c]
                // strided by 8 (warps), so all four sub-partitions share the work
                {
                    const int c = j + 1 + lane;
                    if (c < b) {
                        const double wc = D[j][c] * z;
                        for (int a = j + 1 + (t >> 5); a <= c; a += CBT / 32)
                            D[a][c] = fma(-D[j][a], wc, D[a][c]);
                    }
                }
                __syncthreads();
            }
            if (bad) { broke = true; break; }
            // R11 = diag(sqrt d) L^T: row j of the unscaled block times 1/sqrt(d_j)
            if (t < b) yinv[t] = rsqrt(D[t][t]);
            __syncthreads();
            for (int e = t; e < b * b; e += CBT) {
                const int a = e % b, c = e / b;
                if (a <= c) D[a][c] *= yinv[a];
            }
            __syncthreads();
            if (blockIdx.x == 0) {
                for (int e = t; e < b * b; e += CBT) {
                    const int a = e % b, c = e / b;
                    if (a <= c) W[(kb + a) + int64_t(kb + c) * n] = D[a][c];
                }
            }
            // (B) R12(:, c) = R11^{-T} W12(:, c), one warp per column
            const int m = n - kb - b;
            const int c0 = kb + b;
            for (int cc = gwarp; cc < m; cc += gwarps) {
                const int64_t col = int64_t(c0 + cc) * n + kb;
                double acc = lane < b ? __ldcg(&W[col + lane]) : 0.0;
                double x = 0.0;
                for (int u = 0; u < b; ++u) {
                    const double xu = __shfl_sync(0xffffffffu, acc * yinv[u], u);
                    if (lane == u) x = xu;
                    if (lane > u && lane < b) acc = fma(-D[u][lane], xu, acc);
                }
                if (lane < b) W[col + lane] = x;
            }
            if (!grid_barrier(&ctl->barrier, ++nbar * nb, status, budget)) return;
            // (C) W22 -= R12^T R12 (upper triangle), R12 staged in shared memory
            if (stage_rows) {
                for (int e = t; e < b * m; e += CBT) {
                    const int u = e % b, c = e / b;
                    S[u * m + c] = __ldcg(&W[(kb + u) + int64_t(c0 + c) * n]);
                }
                __syncthreads();
            }
            for (int64_t e = gtid; e < int64_t(m) * m; e += gthreads) {
                const int a = int(e % m), c = int(e / m);
                if (a > c) continue;
                double acc = 0.0;
                if (stage_rows) {
                    for (int u = 0; u < b; ++u) acc = fma(S[u * m + a], S[u * m + c], acc);
                } else {
                    for (int u = 0; u < b; ++u)
                        acc = fma(__ldcg(&W[(kb + u) + int64_t(c0 + a) * n]),
                                  __ldcg(&W[(kb + u) + int64_t(c0 + c) * n]), acc);
                }
                W[(c0 + a) + int64_t(c0 + c) * n] -= acc;
            }
            if (!grid_barrier(&ctl->barrier, ++nbar * nb, status, budget)) return;
        }
        if (!broke) break;
        if (!shift_mode || attempt == 1) {
            if (gtid == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
            break;
        }
        if (!grid_barrier(&ctl->barrier, ++nbar * nb, status, budget)) return;
    }
    for (int64_t e = gtid; e < int64_t(n) * n; e += gthreads) {
        const int a = int(e % n), c = int(e / n);
        if (a > c) W[e] = 0.0;
    }
}

// Rinv(:, j) = R^{-1} e_j for upper triangular R (n x n, ld n); CTA j.
__global__ void k_trinv_upper(int n, const double* __restrict__ R, double* __restrict__ Rinv,
                              const int* __restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ double x[];
    double* rd = x + n;                            // 1 / R(i, i), taken in parallel
    const int j = blockIdx.x;
    const int t = threadIdx.x;
    for (int i = t; i < n; i += blockDim.x) {
        x[i] = (i == j) ? 1.0 : 0.0;
        if (i <= j) rd[i] = 1.0 / R[i + int64_t(i) * n];
    }
    __syncthreads();
    for (int i = j; i >= 0; --i) {
        if (t == 0) x[i] *= rd[i];
        __syncthreads();
        const double xi = x[i];
        for (int k = t; k < i; k += blockDim.x) x[k] -= xi * R[k + int64_t(i) * n];
        __syncthreads();
    }
    for (int i = t; i < n; i += blockDim.x) Rinv[i + int64_t(j) * n] = x[i];
}

// As k_trinv_upper, with the columns of R staged in shared memory cw at a
// time (column c, rows 0..c), so a substitution step reads shared memory
// only.  Same operations in the same order, so the same result.
__global__ void k_trinv_upper_staged(int n, const double* __restrict__ R,
                                     double* __restrict__ Rinv, const int* __restrict__ skip,
                                     int cw) {
    if (skip && *skip) return;
    extern __shared__ double sm[];
    double* x = sm;                                // n
    double* rd = sm + n;                           // n: 1 / R(i, i), taken in parallel
    double* Rc = sm + 2 * n;                       // cw columns of n
    const int j = blockIdx.x;
    const int t = threadIdx.x;
    for (int i = t; i < n; i += blockDim.x) {
        x[i] = (i == j) ? 1.0 : 0.0;
        if (i <= j) rd[i] = 1.0 / R[i + int64_t(i) * n];
    }
    for (int hi = j; hi >= 0; hi -= cw) {
        const int lo = hi - cw + 1 > 0 ? hi - cw + 1 : 0;
        __syncthreads();                           // the previous chunk is no longer read
        for (int c = lo; c <= hi; ++c)
            for (int k = t; k <= c; k += blockDim.x) Rc[(c - lo) * n + k] = R[k + int64_t(c) * n];
        __syncthreads();
        for (int i = hi; i >= lo; --i) {
            const double* col = Rc + (i - lo) * n;
            // one thread scales by the reciprocal taken up front (a dependent
            // FP64 division costs ~430 cycles, a multiply ~65); the rest read x_i
            if (t == 0) x[i] *= rd[i];
            __syncthreads();
            const double xi = x[i];
            for (int k = t; k < i; k += blockDim.x) x[k] -= xi * col[k];
            __syncthreads();
        }
    }
    for (int i = t; i < n; i += blockDim.x) Rinv[i + int64_t(j) * n] = x[i];
}

// Rinv = R^{-1}: the staged kernel when cw >= 8 columns of R fit in 64 KB.
cudaError_t trinv_upper(int n, const double* R, double* Rinv, const int* skip, cudaStream_t s) {
    const int tt = n < 256 ? 128 : 256;
    const int cw = 8192 / (n > 0 ? n : 1);
    count_launch();
    if (cw >= 8) {
        const int w = cw > 64 ? 64 : cw;
        const size_t smem = size_t(n) * (w + 2) * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(k_trinv_upper_staged,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        k_trinv_upper_staged<<<n, tt, smem, s>>>(n, R, Rinv, skip, w);
        return cudaGetLastError();
    }
    k_trinv_upper<<<n, tt, 2 * size_t(n) * sizeof(double), s>>>(n, R, Rinv, skip);
    return cudaGetLastError();
}

// skip2 = 1 when the diagonal spread of the first Cholesky factor is at most
// 1e5 (orthogonality loss of one CholeskyQR round ~ (spread)^2 u <= ~1e-6).
__global__ void k_qr_decide(int n, const double* __restrict__ R, int* __restrict__ skip2) {
    double dmax = 0.0, dmin = 1.7976931348623157e308;
    for (int i = threadIdx.x; i < n; i += 32) {
        const double d = fabs(R[i + int64_t(i) * n]);
        dmax = fmax(dmax, d);
        dmin = fmin(dmin, d);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
        dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
    }
    if (threadIdx.x == 0) *skip2 = (dmin > 0.0 && dmax <= 1e5 * dmin) ? 1 : 0;
}

}  // namespace

cudaError_t launch_trinv_upper(int n, const double* R, double* Rinv, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    return trinv_upper(n, R, Rinv, nullptr, s);
}

size_t qr_scratch_bytes(int64_t rows, int cols, int num_sms, int tc_products) {
    const size_t sq = size_t(cols) * cols * sizeof(double);
    size_t p = gemm_f64_partials_bytes(cols, cols, rows, num_sms);
    const size_t p2 = gemm_f64_partials_bytes(rows, cols, cols, num_sms);
    if (p2 > p) p = p2;
    if (tc_products && oz_supported(rows, cols, num_sms)) {
        const size_t oz = oz_scratch_bytes(rows, cols, num_sms);
        if (oz > p) p = oz;
    }
    return 5 * sq + p + 8 * 256;
}

namespace {
thread_local const char* t_cholqr_step = "";
}

const char* cholqr_failed_step() { return t_cholqr_step; }

cudaError_t launch_cholqr2(int64_t rows, int cols, double* X, int64_t ldx, double* R,
                           int64_t ldR, void* scratch, size_t scratch_cap, int* dev_status,
                           int num_sms, cudaStream_t s, int adaptive, int rounds,
                           int tc_products) {
    t_cholqr_step = "arguments";
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (adaptive && R) return cudaErrorInvalidValue;     // R would be R1 or R2 R1
    if (rounds != 1 && rounds != 2) return cudaErrorInvalidValue;
    Workspace ws;
    ws.base = static_cast<char*>(scratch);
    ws.cap = scratch_cap;
    const size_t sq = size_t(cols) * cols * sizeof(double);
    double* W = static_cast<double*>(ws.take(sq));
    double* Wsave = static_cast<double*>(ws.take(sq));
    double* Rinv = static_cast<double*>(ws.take(sq));
    double* R1 = static_cast<double*>(ws.take(sq));
    double* Rtmp = static_cast<double*>(ws.take(sq));
    CholCtl* ctl = static_cast<CholCtl*>(ws.take(sizeof(CholCtl)));
    int* skip2 = static_cast<int*>(ws.take(sizeof(int)));
    // the rest holds the split-K partial sums of the products
    const size_t off = (ws.used + 255) & ~size_t(255);
    const size_t part_cap = scratch_cap > off ? scratch_cap - off : 0;
    void* part = ws.take(part_cap);
    if (!W || !Wsave || !Rinv || !R1 || !Rtmp || !part || !ctl || !skip2)
        return cudaErrorInvalidValue;
    // the products as exact slice products on the tensor cores, except in
    // the second round of the adaptive form (its kernels must return on a
    // device-side flag, which the FP64 kernels do)
    const bool oz = tc_products && oz_supported(rows, cols, num_sms) &&
                    part_cap >= oz_scratch_bytes(rows, cols, num_sms);
    cudaError_t e;
    for (int pass = 0; pass < rounds; ++pass) {
        const int* sk = (pass == 1 && adaptive) ? skip2 : nullptr;
        const bool tc = oz && (pass == 0 || !adaptive);
        // W = X^T X, upper triangle only (the Cholesky reads nothing else;
        // the tensor-core form writes both triangles)
        t_cholqr_step = tc ? "Gram (tensor cores)" : "Gram";
        if (tc)
            e = launch_oz_gram(rows, cols, X, ldx, W, part, part_cap, dev_status, num_sms, s);
        else
            e = launch_gemm_f64_tri(1, 1, cols, cols, rows, X, ldx, X, ldx, W, cols, part,
                                    part_cap, num_sms, s, sk);
        if (e != cudaSuccess) return e;
        if (pass == 0) {
            e = cudaMemcpyAsync(Wsave, W, sq, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
        t_cholqr_step = "Cholesky";
        if (cols <= 128) {
            count_launch();
            k_cholesky<<<1, CT, 0, s>>>(cols, W, Wsave, rows, pass == 0 ? 1 : 0, dev_status, sk);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        } else {
            e = cudaMemsetAsync(ctl, 0, sizeof(CholCtl), s);
            if (e != cudaSuccess) return e;
            // about one CTA per 512 entries of the Gram matrix (the trailing
            // updates and the block-row solves spread over the SMs' FP64
            // pipes), at least 8, at most one per SM
            int grid = int(int64_t(cols) * cols / 512);
            if (grid < 8) grid = 8;
            if (grid > num_sms) grid = num_sms;
            // the block rows of R12 (CB x (cols - CB) doubles) in shared memory when they fit
            const size_t stage_bytes = size_t(CB) * size_t(cols - CB) * sizeof(double);
            int stage = stage_bytes <= 200 * 1024 ? 1 : 0;
            const size_t dsm = stage ? stage_bytes : 0;
            e = cudaFuncSetAttribute(k_cholesky_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(dsm));
            if (e != cudaSuccess) return e;
            int n_ = cols;
            int shift = pass == 0 ? 1 : 0;
            int64_t rows_ = rows;
            int64_t budget = 16LL << 20;
            const int* skp = sk;
            void* args[] = {&n_, &W, &Wsave, &rows_, &shift, &ctl, &dev_status, &budget, &stage,
                            &skp};
            count_launch();
            e = cudaLaunchCooperativeKernel((const void*)k_cholesky_coop, dim3(grid), dim3(CBT),
                                            args, dsm, s);
            if (e != cudaSuccess) return e;
        }
        if (pass == 0 && adaptive) {
            count_launch();
            k_qr_decide<<<1, 32, 0, s>>>(cols, W, skip2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        t_cholqr_step = "triangular inverse";
        if ((e = trinv_upper(cols, W, Rinv, sk, s)) != cudaSuccess) return e;
        t_cholqr_step = tc ? "X R^-1 (tensor cores)" : "X R^-1";
        // X <- X Rinv (the reduction of the partial sums writes X after the
        // product; the tensor-core form reads X's slices, made first)
        if (tc)
            e = launch_oz_xrinv(rows, cols, X, ldx, Rinv, X, ldx, part, part_cap, dev_status,
                                num_sms, s);
        else
            e = launch_gemm_f64_tri(0, 2, rows, cols, cols, X, ldx, Rinv, cols, X, ldx, part,
                                    part_cap, num_sms, s, sk);
        if (e != cudaSuccess) return e;
        if (pass == 0) {
            e = cudaMemcpyAsync(R1, W, sq, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    if (R && rounds == 1) return launch_copy_cols(cols, cols, R1, cols, R, ldR, s);
    if (R) {
        // R = R2 R1 (both upper triangular)
        e = launch_gemm_f64(0, 0, cols, cols, cols, W, cols, R1, cols, Rtmp, cols, part, part_cap,
                            num_sms, s);
        if (e != cudaSuccess) return e;
        e = launch_copy_cols(cols, cols, Rtmp, cols, R, ldR, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace plu
