// Internal declarations shared by the CUDA translation units of the
// library (not part of the C ABI; see include/powerlu.h for that).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "../../include/powerlu.h"

namespace plu {

// Device status word codes (written by kernels, read by the host).
enum DevStatus : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,     // a grid barrier ran out of its spin budget
    DEV_NUMERIC = 2,     // Cholesky breakdown / non-finite value
    DEV_BADINDEX = 3,    // a sparse index or row pointer out of range
};

// Kernels launched by this host thread (the per-call report counts them).
extern thread_local long long g_launches;
inline void count_launch(long long n = 1) { g_launches += n; }

// Largest grid of the cooperative kernels (one candidate slot per CTA).
constexpr int kMaxGrid = 1024;

// ------------------------------------------------ device-side sync helpers
#ifdef __CUDACC__
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Release-add on a grid barrier counter: after a CTA barrier, it publishes the
// CTA's earlier writes (release is cumulative over what the CTA barrier
// ordered before it) without a full fence.
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// LU multiplier as LAPACK's getf2 / getrf2 form it (the LU behind MATLAB's
// lu): x times rinv = 1 / u when |u| is at least the smallest normal number,
// else x / u.  The comparison runs on the integer pipe.
__device__ __forceinline__ double lu_multiplier(double x, double u, double rinv) {
    return (__double_as_longlong(u) & 0x7FFFFFFFFFFFFFFFLL) >= 0x0010000000000000LL ? x * rinv
                                                                                     : x / u;
}

// x rounded to FP32 (to nearest, ties to even) on the integer pipe: a
// conversion on GB300's FP64 pipe holds it like an FMA (~64 cycles per warp
// instruction), and the FP32 GEMMs convert every FP64 operand they load.
// Results in the normal FP32 range (including a rounding up to infinity) are
// formed from the bits (IEEE 754 round to nearest even of the 52-bit
// significand to 23 bits, the carry running into the exponent); zeros,
// subnormal results, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = unsigned(b >> 32);
    const int e = int((hi >> 20) & 0x7FF);
    if (e < 897 || e > 1150) return __double2float_rn(x);     // |x| < 2^-126 or >= 2^128
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    const unsigned long long rem = m & 0x1FFFFFFFULL;           // the 29 bits dropped
    unsigned bits = (unsigned(e - 1023 + 127) << 23) | unsigned(m >> 29);
    if (rem > 0x10000000ULL || (rem == 0x10000000ULL && (bits & 1u))) bits += 1u;
    return __uint_as_float(bits | (hi & 0x80000000u));
}

// x as FP64, exactly, on the integer pipe (zeros and normal numbers; a
// subnormal, infinite or NaN x takes the hardware conversion).
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    if ((u & 0x7FFFFFFFu) == 0) return __hiloint2double(int(u), 0);
    if (e == 0 || e == 255) return double(x);
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double(int(hi), int(u << 29));
}

// A sum of FP32 values kept as an unevaluated pair s + c (Neumaier's
// compensated summation, on the FP32 pipe): s + c equals the exact sum up to
// a relative error of about n * 2^-48, so value() (one FP64 addition) is as
// good as summing in FP64, without an FP64 conversion and addition per term.
struct Sum2f {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        c = fabsf(s) >= fabsf(x) ? __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x))
                                 : __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
        s = t;
    }
    __device__ __forceinline__ double value() const { return f32_to_f64(s) + f32_to_f64(c); }
};

// Sum of squares of FP32 values without the FP64 pipe: each square is split
// exactly into its FP32 product and the product's FMA residual, and the
// products are added with a compensated (error-free) FP32 sum whose errors,
// and the residuals, go to a second word.  value() is accurate to a few units
// of 2^-44 relative for up to ~2^20 terms.  The explicit _rn intrinsics keep
// the compiler from contracting the steps into other FMAs.  Squares above
// ~1.8e38 overflow to inf.
struct SqSum32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a) {
        const float p = __fmul_rn(a, a);
        const float e = __fmaf_rn(a, a, -p);          // a * a = p + e exactly
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;                                          // s + p = t + err exactly
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// Sum over the CTA of one double per thread (blockDim.x a multiple of 32, at
// most 1024), in a fixed order; the result in thread 0.
__device__ __forceinline__ double cta_sum(double v) {
    __shared__ double wsum[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += wsum[w];
    return s;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// Grid-wide barrier over co-resident CTAs (cooperative launch) on a counter
// that only grows: the k-th barrier of a launch waits for k * gridDim.x
// arrivals.  The spin is bounded by `budget` polls; returns false in every
// thread of the CTA when this CTA gave up (it then sets *status) or another
// CTA reported an error.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* status,
                                             int64_t budget) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add_u32(bar, 1u);
        int good = 1;
        int64_t spins = 0;
        // acquire loads: the other CTAs' writes released before their arrival
        // are visible to this CTA after the CTA barrier below
        while (ld_acquire_u32(bar) < target) {
            if (ld_volatile_i32(status) != DEV_OK) { good = 0; break; }
            if (++spins > budget) {
                atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                good = 0;
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}
#endif


// Workspace carved out of the context's device buffer.
struct Workspace {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    void* take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

// ||A||_F^2 of the matrix a pass reads, accumulated by the pass kernel from
// the entries it stages (every entry once, Alg. adaptivewithoutupdating step
// 1 fused into the first pass): the kernel writes one FP64 partial per CTA to
// parts (room for cap), the launcher then sums them in a fixed order into
// *out (a device double).
struct NormOut {
    double* parts = nullptr;
    int cap = 0;
    double* out = nullptr;
};
// *out = the sum of part[0 .. count-1] in a fixed order (one CTA).
cudaError_t launch_sum_partials(const double* part, int count, double* out, cudaStream_t s);

// ---------------------------------------------------------------- RNG (a1)
cudaError_t launch_gaussian(int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                            double* out, int64_t ld, cudaStream_t s);

// ----------------------------------------------------------- SIMT passes
// C (M x N, FP64, ldc) = op(A) * B with op(A) = A (trans = 0, A is M x K) or
// A^T (trans = 1, A is K x M); A of element type dtype (lda), B FP64 (K x N).
// prec selects FP64 FMA or FP32 FMA (B converted to FP32).  `partials`
// (part_cap bytes) receives the split-K partial sums: gemm_partials_bytes(...)
// is the size for the preferred split count; a smaller buffer lowers the
// split count, one without room for a single M x N partial is an error.
size_t gemm_partials_bytes(int64_t M, int64_t N, int64_t K, int prec, int num_sms);
cudaError_t launch_gemm_simt(int trans, int64_t M, int64_t N, int64_t K, const void* A,
                             int dtype, int64_t lda, const double* B, int64_t ldb,
                             double* C, int64_t ldc, int prec, void* partials,
                             size_t part_cap, float* b32_scratch, int num_sms, cudaStream_t s,
                             int accum = 0, const NormOut* norm = nullptr);
// Partials a pass with the NormOut needs (one per CTA of the first column tile).
int gemm_norm_parts(int64_t M, int64_t N, int64_t K, int num_sms);
// accum > 0: C += op(A) B; accum < 0: C -= op(A) B; 0: C = op(A) B.
// FP64 GEMM with transposed-B option for the small products of the tail:
// C = A * op(B), op(B) = B (K x N) or B^T (B is N x K).
cudaError_t launch_gemm_f64(int transA, int transB, int64_t M, int64_t N, int64_t K,
                            const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc, void* partials, size_t part_cap,
                            int num_sms, cudaStream_t s);
size_t gemm_f64_partials_bytes(int64_t M, int64_t N, int64_t K, int num_sms);
// As launch_gemm_f64 (no B transpose) with a triangular shortcut: tri 1 computes
// only the upper triangle of C (the rest is zero), tri 2 takes op(B) upper
// triangular, tri 3 lower triangular.
// skip (nullable, device): when *skip != 0 at run time the kernels return
// without touching C.
cudaError_t launch_gemm_f64_tri(int transA, int tri, int64_t M, int64_t N, int64_t K,
                                const double* A, int64_t lda, const double* B, int64_t ldb,
                                double* C, int64_t ldc, void* partials, size_t part_cap,
                                int num_sms, cudaStream_t s, const int* skip = nullptr);

// As launch_gemm_f64_tri without the A transpose, with FP32 FMAs: A and B are
// read as FP64 and rounded to FP32, each split sums in FP32 and the splits are
// added in FP64.  The partial sums take half the bytes of the FP64 version.
cudaError_t launch_gemm_f32_tri(int tri, int64_t M, int64_t N, int64_t K, const double* A,
                                int64_t lda, const double* B, int64_t ldb, double* C,
                                int64_t ldc, void* partials, size_t part_cap, int num_sms,
                                cudaStream_t s);

// ----------------------------------------------- tensor-core passes (TF32)
// Y (FP64) = A X (trans 0) or A^T X (trans 1) with FP32 A (m x n, lda) on
// tcgen05 tensor cores; X is FP64 (K x cols).  tc_supported() tells whether
// the shape / alignment is handled (cols <= 512, lda % 4 == 0, A 16-byte
// aligned).  scratch holds scratch_cap bytes, at least tc_scratch_bytes(M, K,
// cols, num_sms) (an error otherwise).
bool tc_supported(int64_t M, int64_t K, int cols, const void* A, int64_t lda, int trans);
size_t tc_scratch_bytes(int64_t M, int64_t K, int cols, int num_sms);
// xq_pre (nullable): X already in operand form (launch_tc_operand with the
// same K and cols); the pass then reads it instead of converting X.
cudaError_t launch_tc_pass(int trans, int64_t m, int64_t n, const float* A, int64_t lda,
                           const double* X, int64_t ldx, int cols, double* Y, int64_t ldy,
                           void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                           cudaStream_t s, int accum = 0, const void* xq_pre = nullptr,
                           const NormOut* norm = nullptr);
// The TF32 operand image of X (K x cols, FP64): the tiled, swizzled layout the
// pass kernel copies one K step at a time.  out holds tc_operand_bytes(K, cols).
size_t tc_operand_bytes(int64_t K, int cols);
cudaError_t launch_tc_operand(int64_t K, int cols, const double* X, int64_t ldx, void* out,
                              int num_sms, cudaStream_t s);
// Quantized copy of A for the BF16 / FP8-E4M3 passes: column-major, ld a
// multiple of 16 elements; FP8 carries rank-1 tile scales s_r (per 128 rows)
// and s_c (per 128 columns) with A(i, j) ~= Aq(i, j) s_r[i/128] s_c[j/128].
struct QuantA {
    const void* data = nullptr;
    int64_t ld = 0, m = 0, n = 0;
    int prec = 0;
    const float* s_r = nullptr;
    const float* s_c = nullptr;
};
size_t tc_quant_bytes(int64_t m, int64_t n, int prec);
cudaError_t launch_tc_quantize(int prec, const float* A, int64_t m, int64_t n, int64_t lda,
                               void* qbuf, QuantA* out, int num_sms, cudaStream_t s,
                               const NormOut* norm = nullptr);
// Partials the quantisation (or a tensor-core pass) needs for the NormOut.
int quant_norm_parts(int num_sms);
// The stream-K partial tiles of one pass, left in its scratch for a later
// reduction: CTA c's segment for row block b at part + ((c max_segs + b -
// c per / ksteps) npad) 128.
constexpr int kMaxBands = 16;
struct TcPartials {
    const float* part = nullptr;
    int npad = 0, ksteps = 0, max_segs = 0, grid = 0;
    int64_t total = 0, per = 0;
};
// xq_pre (BF16 only): X already in BF16 operand form, as for launch_tc_pass.
// keep (BF16 only, non-null): the pass leaves its partial tiles in scratch,
// described by *keep, and does not write Y.
cudaError_t launch_tc_pass_q(int trans, const QuantA& q, const double* X, int64_t ldx, int cols,
                             double* Y, int64_t ldy, void* scratch, size_t scratch_cap,
                             int* dev_status, int num_sms, cudaStream_t s, int accum = 0,
                             const void* xq_pre = nullptr, TcPartials* keep = nullptr);
// Y (M x cols, ldy) = (accum != 0: Y +, else) the FP64 sum of
// the stream-K partial tiles P in CTA order.
cudaError_t launch_tc_reduce(const TcPartials& P, int64_t M, int cols, double* Y, int64_t ldy,
                             int accum, int num_sms, cudaStream_t s);
// A 2-D tensor map (128-byte swizzle) over a column-major matrix: element
// size dtype_code (4 FP32, 2 BF16, 1 one-byte), dim0 contiguous.
bool tc_make_map_2d(CUtensorMap* map, int dtype_code, const void* base, uint64_t dim0,
                    uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1);

// Split-precision passes (3xTF32, plu_tcsplit.cu): Y = op(A) X with FP32 A
// = A_hi + A_lo and X = X_hi + X_lo (hi the TF32 rounding, lo the TF32
// rounding of the remainder), Y = A_hi X_hi + A_lo X_hi + A_hi X_lo on the
// tensor cores with FP32 accumulation: FP32-accurate products.
bool tcs_supported(int64_t M, int64_t K, int cols, const void* A, int64_t lda, int trans);
size_t tcs_scratch_bytes(int64_t M, int64_t K, int cols, int num_sms);
// The small operand X (K x cols) in the split pass's hi/lo operand form, made
// once for several passes that share it (ximg_pre).
size_t tcs_operand_bytes(int64_t K, int cols);
cudaError_t launch_tcs_operand(int64_t K, int cols, const double* X, int64_t ldx, void* out,
                               int num_sms, cudaStream_t s);
// Y (rows x k) = X T with X FP64 (rows x k) and T FP64 (k x k) as split-precision
// tensor-core products: X is rounded to an FP32 copy in scratch (ld a
// multiple of 4) and taken through launch_tc_split_pass (FP32-accurate).
size_t tcs_product_scratch_bytes(int64_t rows, int k, int num_sms);
cudaError_t launch_tcs_product(int64_t rows, int k, const double* X, int64_t ldx, const double* T,
                               int64_t ldt, double* Y, int64_t ldy, void* scratch,
                               size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s);
// norm (nullable): ||A||_F^2 of the entries the pass reads, summed into *norm->out.
cudaError_t launch_tc_split_pass(int trans, int64_t m, int64_t n, const float* A, int64_t lda,
                                 const double* X, int64_t ldx, int cols, double* Y, int64_t ldy,
                                 void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                                 cudaStream_t s, int accum = 0, const void* ximg_pre = nullptr,
                                 const NormOut* norm = nullptr);

// Y (M x cols, ldy) = the bands' FP64 reductions added in order (one write).
cudaError_t launch_tc_reduce_bands(const TcPartials* bands, int nbands, int64_t M, int cols,
                                   double* Y, int64_t ldy, cudaStream_t s);

// FP64-accurate X^T X and X R^{-1} on the BF16 tensor cores (sums of exact
// slice products; plu_ozaki.cu).  X is rows x cols (ldx), R^{-1} cols x cols
// (ld cols); W (cols x cols, ld cols) receives the whole Gram matrix.
// oz_supported() tells whether the shape keeps every FP32 partial sum exact
// (cols <= 512 and a bounded stream-K segment); the launchers return an error
// otherwise.  scratch holds oz_scratch_bytes().
bool oz_supported(int64_t rows, int cols, int num_sms);
size_t oz_scratch_bytes(int64_t rows, int cols, int num_sms);
cudaError_t launch_oz_gram(int64_t rows, int cols, const double* X, int64_t ldx, double* W,
                           void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                           cudaStream_t s);
cudaError_t launch_oz_xrinv(int64_t rows, int cols, const double* X, int64_t ldx,
                            const double* Rinv, double* Y, int64_t ldy, void* scratch,
                            size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s);

// ------------------------------------------------------- panel LU (a3, a8)
struct PanelScratch;   // defined in plu_panel.cu; starts with a PanelHead
// Head of a panel LU's scratch: the grid-barrier counter, the first exactly
// zero pivot column (1-based, as LAPACK's info) and the non-finite flag.
struct PanelHead {
    unsigned int barrier;
    int info;
    int any_nan;
    int pad;
};
size_t panel_head_bytes();
size_t panel_scratch_bytes(int64_t rows, int cols);
// Factor X (rows x cols) in place with partial pivoting (virtual row order).
// mode 0: leave X = P^T L (reorthogonalisation).
// mode 1: write perm, L (pivoted order) and U (or U^T when u_trans), or L^T
//         when l_trans; X is destroyed.
cudaError_t launch_panel_lu(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                            int32_t* perm, double* L, int64_t ldL, int l_trans,
                            double* U, int64_t ldU, int u_trans, int32_t* info,
                            void* scratch, int* dev_status, int64_t spin_budget,
                            int num_sms, cudaStream_t s);

// After a factorisation with rows in place: info and the non-finite flag;
// mode 0 writes P^T L into X, mode 1 writes perm, L (or L^T) and U (or U^T)
// from the U rows in Ubuf (steps x cols, ld steps; nullptr: from X).
cudaError_t launch_panel_finish(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                                int32_t* perm, double* L, int64_t ldL, int l_trans, double* U,
                                int64_t ldU, int u_trans, int32_t* info, const void* head,
                                const int* pos, const int* pivstep, const double* Ubuf,
                                int* dev_status, int num_sms, cudaStream_t s);

// The same factorisation as launch_panel_lu (same pivots, rows in place),
// with the trailing updates between 32-column leaves computed on the tensor
// cores as FP64-accurate sums of exact FP16 digit products (plu_tclu.cu).
// tclu_supported() tells whether the shape fits its kernels.
bool tclu_supported(int64_t rows, int cols, int num_sms);
size_t tclu_scratch_bytes(int64_t rows, int cols);
cudaError_t launch_panel_lu_tc(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                               int32_t* perm, double* L, int64_t ldL, int l_trans, double* U,
                               int64_t ldU, int u_trans, int32_t* info, void* scratch,
                               int* dev_status, int64_t spin_budget, int num_sms, cudaStream_t s);

// --------------------------------------------------------------- QR (a5)
// scratch holds scratch_cap >= qr_scratch_bytes(rows, cols, num_sms) bytes
// (less works down to one split of each product; too little is an error).
size_t qr_scratch_bytes(int64_t rows, int cols, int num_sms, int tc_products = 0);
// adaptive != 0: the second CholeskyQR round runs only when the first
// Cholesky factor's diagonal spread max|r_ii| / min|r_ii| exceeds 1e5 (the
// decision is taken on the device; the second round's kernels return at once
// otherwise); R cannot be requested then.  rounds = 1 runs one CholeskyQR
// round (X <- X R1^{-1}, R = R1, with R1^T R1 = X^T X).  tc_products != 0
// computes X^T X and X R^{-1} as exact slice products on the BF16 tensor
// cores (launch_oz_gram / launch_oz_xrinv; in every round, except the
// device-skippable second round of the adaptive form) when the shape allows
// it and the scratch holds qr_scratch_bytes(..., 1).
cudaError_t launch_cholqr2(int64_t rows, int cols, double* X, int64_t ldx, double* R,
                           int64_t ldR, void* scratch, size_t scratch_cap, int* dev_status,
                           int num_sms, cudaStream_t s, int adaptive = 0, int rounds = 2,
                           int tc_products = 0);

// The step of the calling thread's last launch_cholqr2 that returned an error.
const char* cholqr_failed_step();

// Rinv = R^{-1} for an upper triangular n x n R (ld n); Rinv is upper triangular.
cudaError_t launch_trinv_upper(int n, const double* R, double* Rinv, cudaStream_t s);

// -------------------------------------------------------- sparse passes
// Y (rows x cols, ld ldy) = S X for S rows x K in CSR (row_ptr rows + 1,
// col_idx / val nnz entries) and X K x cols (ld ldx), FP64.  The scratch
// holds the row-major copy of X.  A column index outside [0, K) or a row
// pointer outside [0, nnz] sets DEV_BADINDEX and the entry is skipped.
int spmm_row_stride(int cols);
size_t spmm_scratch_bytes(int64_t K, int cols);
cudaError_t launch_spmm_csr(int64_t rows, int64_t K, int64_t nnz, const int64_t* row_ptr,
                            const int32_t* col_idx, const double* val, const double* X,
                            int64_t ldx, int cols, double* Y, int64_t ldy, void* scratch,
                            size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s,
                            const NormOut* norm = nullptr);
// Partials the sparse pass needs for the NormOut (the sum of the squared
// values of the CSR it reads).
int spmm_norm_parts(int64_t rows, int num_sms);

// -------------------------------------------------------- rank and norms
size_t norm2_scratch_bytes(int num_sms);
cudaError_t launch_norm2(const void* A, int dtype, int64_t m, int64_t n, int64_t lda,
                         double* out, void* scratch, int num_sms, cudaStream_t s);
// *out = sum of x[i]^2 over count entries (scratch: norm2_scratch_bytes).
cudaError_t launch_sumsq(const double* x, int64_t count, double* out, void* scratch,
                         int num_sms, cudaStream_t s);
cudaError_t launch_colnorm2(int64_t rows, int cols, const double* G, int64_t ldg,
                            double* out, cudaStream_t s);
// k/E/met from column norms (one thread): out[0] = k, out[1] = met (ints);
// E written to *E_out (device double).  The scan starts from *E_start when
// given (an indicator carried over from an earlier round), else from *normA2;
// the tolerance is eps^2 *normA2 either way.
cudaError_t launch_rank_scan(const double* colnorm2, int cols, const double* normA2,
                             double eps, int b, int precise, int* k_met, double* E_out,
                             cudaStream_t s, const double* E_start = nullptr);

// -------------------------------------------------------------- helpers
cudaError_t launch_copy_cols(int64_t rows, int cols, const double* src, int64_t lds,
                             double* dst, int64_t ldd, cudaStream_t s);
// W(perm[i], j) = L(i, j) for i < rows, j < cols: the rows of an LU's L (in
// pivoted order) moved back to the row order of the factored matrix.
// perm must be a permutation of 0 .. rows-1 (entries outside are skipped).
cudaError_t launch_scatter_rows(int64_t rows, int cols, const int32_t* perm, const double* L,
                                int64_t ldl, double* W, int64_t ldw, cudaStream_t s);

// ------------------------------------------------------------- batched
size_t batch_workspace_bytes(const plu_batch_problem* P, int count);
size_t batch_tables_bytes(int count);
// tuned: the tile shape and split-K choice of every grouped GEMM of the
// plan; when it does not match the plan's GEMM count the autotuner times the
// choices and fills it.  forced >= 0 takes that tile shape, unsplit, for every
// grouped GEMM instead.  *part / *part_cap: the split-K partial buffer (device,
// owned by the caller, grown here with cudaMalloc when too small).
cudaError_t run_batch(const plu_batch_problem* P, int count, int prec, char* ws, char* tables,
                      size_t tables_cap, int* dev_status, int num_sms, cudaStream_t s,
                      cudaStream_t capture_stream, int* nlaunch, float* ms_graph,
                      std::vector<int>* tuned, int forced, double** part, size_t* part_cap);
// Tile shape (rows, columns) of grouped-GEMM choice c; 0 for a bad index.
int batch_gemm_tile(int choice, int* bm, int* bn);
// K-chunk length of choice c (0: no split-K); -1 for a bad index.
int batch_gemm_splitk(int choice);
// Number of grouped-GEMM choices (tile shapes x split-K lengths).
int batch_gemm_choices();

}  // namespace plu
