// FP64-accurate products on the BF16 tensor cores for CholeskyQR's Gram
// matrix X^T X and its product X R^{-1} (the a5 step of the mixed modes).
//
// GB300 runs FP64 FMAs at 1.25 TFLOP/s, so these two n x k x k products are
// bound by the FP64 pipe.  Here every FP64 operand is split into OZ_S slices:
// with a common exponent E per row (or per column), x = sum_i n_i 2^(E - 7 i)
// + r, |n_i| <= 64 integers, |r| <= 2^(E - 57) (8 slices of 7 bits after one
// bit of headroom).  A slice value n_i 2^(E - 7 i) is exact in BF16.
//
// The product of slice i of one operand and slice j of the other is exact in
// FP32 accumulation: every term is a multiple of the same power of two (the
// row and column exponents and 7 (i + j) fix it), each term is at most
// 64 * 64 = 2^12 of those units, and every FP32 partial sum the tensor-core
// pass forms covers at most 4096 terms (asserted on the host), so it stays
// within 2^24 units.  The pass sums its partial tiles in FP64, which is also
// exact here.  Pairs with the same i + j = t share their units, so they are
// stacked along the reduction index and computed by one pass per t; the
// passes for t = 2 .. OZ_S + 1 are added in FP64.  The pairs dropped (i + j >
// OZ_S + 1) and the remainders r contribute below 2^-50 of |X| |Y| k, within
// the bound of an FP64 product.  Slices are cut with integer operations (the
// FP64 pipe is the one being avoided).  The slice values must lie in BF16's
// exponent range: row and column maxima between about 2^-70 and 2^120, which
// holds for the orthonormalised bases and triangular inverses these products
// see; smaller entries only lose bits below 2^-126 absolute.
#include "plu_internal.h"

#include <cuda_bf16.h>
#include <climits>

namespace plu {
namespace {

constexpr int OZ_S = 8;          // slices per operand
constexpr int OZ_BITS = 7;       // bits per slice (|n_i| <= 64)

// E with max|x| < 2^(E-1), so the first slice's integer is at most 64; INT_MIN
// for an all-zero line, INT_MAX for a line holding an inf or a NaN (its slices
// are NaN, so the products report it).
__device__ __forceinline__ int oz_exponent(double maxabs) {
    if (!(maxabs <= 1.7976931348623157e308)) return INT_MAX;
    if (!(maxabs > 0.0)) return INT_MIN;
    int e;
    frexp(maxabs, &e);               // maxabs < 2^e
    return e + 1;
}

// The slice integers of x with exponent E, on the integer pipe: N = x
// 2^(56 - E) rounded to an integer (|N| < 2^55, so |x - N 2^(E - 56)| <=
// 2^(E - 57)), written in balanced base 128: N = sum_i n_i 128^(7 - i),
// n_7..n_1 in [-64, 63] and n_0 in [-64, 64].
__device__ __forceinline__ void oz_digits(double x, int E, int dig[OZ_S]) {
    const long long bits = __double_as_longlong(x);
    const int ex = int((bits >> 52) & 0x7FF);
    long long N = 0;
    if (E != INT_MIN && ex != 0) {                 // zero and subnormal x give N = 0
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        // x = mant 2^(ex - 1075), N = mant 2^(ex - 1075 + 56 - E)
        const int sh = ex - 1019 - E;
        if (sh >= 0) {
            N = sh < 3 ? (mant << sh) : 0;       // |x| < 2^(E-1) bounds sh <= 2
        } else if (sh > -63) {
            const long long half = 1LL << (-sh - 1);
            N = (mant + half) >> (-sh);          // round half up
        }
        if (bits < 0) N = -N;
    }
#pragma unroll
    for (int i = OZ_S - 1; i > 0; --i) {
        long long d = N & 127;                   // N mod 128 in [0, 128)
        if (d >= 64) d -= 128;                   // centred: [-64, 63]
        dig[i] = int(d);
        N = (N - d) >> 7;                        // exact division by 128
    }
    dig[0] = int(N);
}

// The slices of x with exponent E: out[i] = n_i 2^(E - 7 (i + 1)).
__device__ __forceinline__ void oz_split(double x, int E, double out[OZ_S]) {
    if (E == INT_MIN || E == INT_MAX) {
        const double v = E == INT_MAX ? __longlong_as_double(0x7FF8000000000000LL) : 0.0;
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) out[i] = v;
        return;
    }
    double y = ldexp(x, OZ_BITS - E);                 // |y| < 64, exact scaling
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
        const double ni = rint(y);                    // |ni| <= 64
        out[i] = ldexp(ni, E - OZ_BITS * (i + 1));
        y = (y - ni) * double(1 << OZ_BITS);          // exact: |y - ni| <= 1/2
    }
}

// |x| as the 64-bit pattern of its absolute value: for finite values these
// order like the values, so maxima run on the integer pipe.
__device__ __forceinline__ long long abs_bits(double x) {
    return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
}

// Per-column exponents of X (rows x cols): one CTA per column.
__global__ void k_oz_colexp(int64_t rows, const double* __restrict__ X, int64_t ldx,
                            int* __restrict__ Ecol) {
    __shared__ long long red[256];
    const int a = blockIdx.x;
    long long mx = 0;
    for (int64_t r = threadIdx.x; r < rows; r += 256) mx = max(mx, abs_bits(X[r + a * ldx]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + s2]);
        __syncthreads();
    }
    if (threadIdx.x == 0) Ecol[a] = oz_exponent(__longlong_as_double(red[0]));
}

// Per-row exponents of X (rows x cols): 64 rows per CTA, four threads per
// row, each scanning every fourth column (more loads in flight than one
// thread per row), their maxima combined in shared memory.
constexpr int RX_ROWS = 64;
__global__ void __launch_bounds__(RX_ROWS * 4) k_oz_rowexp(int64_t rows, int cols,
                                                          const double* __restrict__ X,
                                                          int64_t ldx, int* __restrict__ Erow) {
    __shared__ long long part[4][RX_ROWS];
    const int lr = threadIdx.x % RX_ROWS, q = threadIdx.x / RX_ROWS;
    const int64_t r = int64_t(blockIdx.x) * RX_ROWS + lr;
    long long mx = 0;
    if (r < rows) {
#pragma unroll 8
        for (int a = q; a < cols; a += 4) mx = max(mx, abs_bits(X[r + a * ldx]));
    }
    part[q][lr] = mx;
    __syncthreads();
    if (q == 0 && r < rows) {
        mx = max(max(part[0][lr], part[1][lr]), max(part[2][lr], part[3][lr]));
        Erow[r] = oz_exponent(__longlong_as_double(mx));
    }
}

// Gram operands, column exponents.  Slice i of X goes (a) to rows
// [i nr, i nr + rows) of the tall BF16 matrix Sv (ld ldv, column-major; rows
// rows..nr-1 of each block are zero) and (b) to block OZ_S - 1 - i of the
// reversed operand image img: nr / 64 K steps per block, each step npad rows
// (columns of X) of 128 bytes holding 64 consecutive rows of X, 16-byte chunk
// c of row j stored at chunk c ^ (j % 8) (the layout the pass kernel copies).
// CTA row blockIdx.y = column a; a thread takes the row pairs (r, r + 1), r
// even, x strided over nr / 2, and stores each slice's pair as one 4-byte word
// (adjacent in Sv, and in one 16-byte chunk of the image).
__device__ __forceinline__ __nv_bfloat16 oz_slice_value(int dig, int Es, int i, bool bad) {
    return __float2bfloat16_rn(bad ? __int_as_float(0x7FC00000)
                                   : ldexpf(float(dig), Es - OZ_BITS * (i + 1)));
}

__global__ void k_oz_slice_gram(int64_t rows, int64_t nr, const double* __restrict__ X,
                                int64_t ldx, const int* __restrict__ Ecol,
                                __nv_bfloat16* __restrict__ Sv, int64_t ldv,
                                unsigned char* __restrict__ img, int npad) {
    const int a = blockIdx.y;
    const int E = Ecol[a];
    const int64_t steps = nr / 64;
    const int Es = (E == INT_MIN || E == INT_MAX) ? 0 : E;   // digits 0 then
    for (int64_t pr = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; pr < nr / 2;
         pr += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = 2 * pr;
        int d0[OZ_S], d1[OZ_S];
        oz_digits(r < rows ? X[r + a * ldx] : 0.0, (r < rows && E != INT_MAX) ? E : INT_MIN, d0);
        oz_digits(r + 1 < rows ? X[r + 1 + a * ldx] : 0.0,
                  (r + 1 < rows && E != INT_MAX) ? E : INT_MIN, d1);
        const bool bad0 = E == INT_MAX && r < rows;             // inf / NaN column
        const bool bad1 = E == INT_MAX && r + 1 < rows;
        const int64_t s = r / 64;
        const int kk = int(r % 64);
        const int64_t in_step = int64_t(a) * 128 + (((kk / 8) ^ (a & 7)) << 4) + (kk % 8) * 2;
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
            __nv_bfloat162 v;
            v.x = oz_slice_value(d0[i], Es, i, bad0);
            v.y = oz_slice_value(d1[i], Es, i, bad1);
            *reinterpret_cast<__nv_bfloat162*>(Sv + int64_t(i) * nr + r + a * ldv) = v;
            const int64_t step = int64_t(OZ_S - 1 - i) * steps + s;
            *reinterpret_cast<__nv_bfloat162*>(img + step * int64_t(npad) * 128 + in_step) = v;
        }
    }
}

// X R^{-1} left operand, row exponents: slice i of X to columns
// [i cols, (i + 1) cols) of Sh (rows x OZ_S cols, BF16, ld lds, a multiple of
// 16).  A thread takes the row pairs (r, r + 1), r even, and stores each
// slice's pair as one 4-byte word (a zero for row r + 1 = rows, inside lds).
__global__ void k_oz_slice_rows(int64_t rows, int cols, const double* __restrict__ X,
                                int64_t ldx, const int* __restrict__ Erow,
                                __nv_bfloat16* __restrict__ Sh, int64_t lds) {
    const int a = blockIdx.y;
    for (int64_t pr = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; pr < (rows + 1) / 2;
         pr += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = 2 * pr;
        const bool has1 = r + 1 < rows;
        int d0[OZ_S], d1[OZ_S];
        const int E0 = Erow[r];
        const int E1 = has1 ? Erow[r + 1] : INT_MIN;
        oz_digits(X[r + a * ldx], E0 == INT_MAX ? INT_MIN : E0, d0);
        oz_digits(has1 ? X[r + 1 + a * ldx] : 0.0, E1 == INT_MAX ? INT_MIN : E1, d1);
        const int Es0 = (E0 == INT_MIN || E0 == INT_MAX) ? 0 : E0;   // digits 0 then
        const int Es1 = (E1 == INT_MIN || E1 == INT_MAX) ? 0 : E1;
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
            __nv_bfloat162 v;
            v.x = oz_slice_value(d0[i], Es0, i, E0 == INT_MAX);
            v.y = oz_slice_value(d1[i], Es1, i, E1 == INT_MAX);
            *reinterpret_cast<__nv_bfloat162*>(Sh + r + (int64_t(i) * cols + a) * lds) = v;
        }
    }
}

// X R^{-1} right operand, column exponents of R^{-1} (n x n): slice j of
// column c to block OZ_S - 1 - j of Trev (OZ_S n x n, FP64, ld OZ_S n), so
// that the pass for i + j = t reads the suffix starting at block OZ_S + 1 - t.
// One CTA per column.
__global__ void k_oz_slice_rinv(int n, const double* __restrict__ Rinv,
                                double* __restrict__ Trev) {
    __shared__ long long red[256];
    __shared__ int Es;
    const int c = blockIdx.x;
    long long mx = 0;
    for (int r = threadIdx.x; r < n; r += 256) mx = max(mx, abs_bits(Rinv[r + int64_t(c) * n]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + s2]);
        __syncthreads();
    }
    if (threadIdx.x == 0) Es = oz_exponent(__longlong_as_double(red[0]));
    __syncthreads();
    const int64_t ldt = int64_t(OZ_S) * n;
    for (int r = threadIdx.x; r < n; r += 256) {
        double sl[OZ_S];
        oz_split(Rinv[r + int64_t(c) * n], Es, sl);
#pragma unroll
        for (int j = 0; j < OZ_S; ++j) Trev[int64_t(OZ_S - 1 - j) * n + r + int64_t(c) * ldt] = sl[j];
    }
}

struct OzLayout {
    int64_t nr, ldv, lds;
    int npad;
    size_t e_off, a_off, b_off, pass_off, total;
    size_t xr_band;            // X R^{-1}: one pass scratch per band (kept partials)
};

// Both phases share one region: the Gram's Sv + img, then (after the
// Cholesky) X R^{-1}'s Sh + Trev.  The pass scratch follows.
OzLayout oz_layout(int64_t rows, int cols, int num_sms) {
    OzLayout L{};
    L.nr = (rows + 63) / 64 * 64;
    L.ldv = int64_t(OZ_S) * L.nr;
    L.lds = (rows + 15) / 16 * 16;
    L.npad = cols <= 256 ? (cols + 15) / 16 * 16 : (cols + 31) / 32 * 32;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    L.e_off = off;
    off = up(off + size_t(rows > cols ? rows : cols) * sizeof(int));
    L.a_off = off;
    const size_t gram_a = size_t(L.ldv) * cols * 2;                        // Sv
    const size_t xr_a = size_t(L.lds) * size_t(OZ_S) * cols * 2;          // Sh
    off = up(off + (gram_a > xr_a ? gram_a : xr_a));
    L.b_off = off;
    const size_t gram_b = size_t(OZ_S) * size_t(L.nr / 64) * L.npad * 128;  // img
    const size_t xr_b = size_t(OZ_S) * cols * size_t(cols) * sizeof(double);  // Trev
    off = up(off + (gram_b > xr_b ? gram_b : xr_b));
    L.pass_off = off;
    // the pass scratch of every band t (it is not monotone in the reduction
    // length: the stream-K grid changes with it)
    size_t pg = 0, px = 0;
    for (int t = 2; t <= OZ_S + 1; ++t) {
        const size_t p1 = tc_scratch_bytes(cols, int64_t(t - 1) * L.nr, cols, num_sms);
        const size_t p2 = tc_scratch_bytes(rows, int64_t(t - 1) * cols, cols, num_sms);
        if (p1 > pg) pg = p1;
        if (p2 > px) px = p2;
    }
    L.xr_band = up(px);
    const size_t xr_all = L.xr_band * OZ_S;
    off = up(off + (pg > xr_all ? pg : xr_all));
    L.total = off;
    return L;
}

// The longest FP32 partial sum of the pass Y = A^T X with A = K x M (stream-K
// over (128-row block, 64-element K step) units, one CTA per SM): the units of
// one CTA within one block.
int64_t oz_seg_terms(int64_t M, int64_t K, int num_sms) {
    const int64_t ksteps = (K + 63) / 64;
    const int64_t total = ((M + 127) / 128) * ksteps;
    const int64_t grid = total < num_sms ? total : num_sms;
    const int64_t per = (total + grid - 1) / grid;
    return (per < ksteps ? per : ksteps) * 64;
}

int grid_rows(int64_t rows, int cols, int num_sms) {
    int64_t b = (rows + 255) / 256;
    const int64_t cap = (int64_t(num_sms) * 16 + cols - 1) / cols;
    if (b > cap) b = cap;
    return int(b < 1 ? 1 : b);
}

}  // namespace

bool oz_supported(int64_t rows, int cols, int num_sms) {
    if (cols < 1 || cols > 512 || rows < cols) return false;
    // every FP32 partial sum covers at most 4096 terms of at most 2^12 units,
    // so every partial sum is an integer number of units below 2^24 + 1
    if (int64_t(OZ_S) * cols > 4096) return false;
    const OzLayout L = oz_layout(rows, cols, num_sms);
    for (int t = 2; t <= OZ_S + 1; ++t)
        if (oz_seg_terms(cols, int64_t(t - 1) * L.nr, num_sms) > 4096) return false;
    return true;
}

size_t oz_scratch_bytes(int64_t rows, int cols, int num_sms) {
    return oz_layout(rows, cols, num_sms).total;
}

cudaError_t launch_oz_gram(int64_t rows, int cols, const double* X, int64_t ldx, double* W,
                           void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                           cudaStream_t s) {
    if (!oz_supported(rows, cols, num_sms)) return cudaErrorInvalidValue;
    const OzLayout L = oz_layout(rows, cols, num_sms);
    if (scratch_cap < L.total) return cudaErrorInvalidValue;
    char* base = static_cast<char*>(scratch);
    int* Ecol = reinterpret_cast<int*>(base + L.e_off);
    __nv_bfloat16* Sv = reinterpret_cast<__nv_bfloat16*>(base + L.a_off);
    unsigned char* img = reinterpret_cast<unsigned char*>(base + L.b_off);
    cudaError_t e;
    if (L.npad > cols) {           // operand rows beyond cols are zero
        e = cudaMemsetAsync(img, 0, size_t(OZ_S) * size_t(L.nr / 64) * L.npad * 128, s);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    k_oz_colexp<<<cols, 256, 0, s>>>(rows, X, ldx, Ecol);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_oz_slice_gram<<<dim3(unsigned(grid_rows(L.nr / 2, cols, num_sms)), unsigned(cols)), 256, 0, s>>>(
        rows, L.nr, X, ldx, Ecol, Sv, L.ldv, img, L.npad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t step_bytes = size_t(L.npad) * 128;
    for (int t = 2; t <= OZ_S + 1; ++t) {
        // sum over i + j = t: [S_1; ..; S_{t-1}]^T [S_{t-1}; ..; S_1]
        QuantA q;
        q.data = Sv;
        q.ld = L.ldv;
        q.m = int64_t(t - 1) * L.nr;
        q.n = cols;
        q.prec = PLU_BF16;
        const unsigned char* pre = img + size_t(OZ_S + 1 - t) * size_t(L.nr / 64) * step_bytes;
        e = launch_tc_pass_q(1, q, nullptr, 0, cols, W, cols, base + L.pass_off,
                             scratch_cap - L.pass_off, dev_status, num_sms, s, t > 2 ? 1 : 0, pre);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_oz_xrinv(int64_t rows, int cols, const double* X, int64_t ldx,
                            const double* Rinv, double* Y, int64_t ldy, void* scratch,
                            size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s) {
    if (!oz_supported(rows, cols, num_sms)) return cudaErrorInvalidValue;
    const OzLayout L = oz_layout(rows, cols, num_sms);
    if (scratch_cap < L.total) return cudaErrorInvalidValue;
    char* base = static_cast<char*>(scratch);
    int* Erow = reinterpret_cast<int*>(base + L.e_off);
    __nv_bfloat16* Sh = reinterpret_cast<__nv_bfloat16*>(base + L.a_off);
    double* Trev = reinterpret_cast<double*>(base + L.b_off);
    cudaError_t e;
    count_launch();
    k_oz_rowexp<<<unsigned((rows + RX_ROWS - 1) / RX_ROWS), RX_ROWS * 4, 0, s>>>(rows, cols, X,
                                                                              ldx, Erow);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_oz_slice_rows<<<dim3(unsigned(grid_rows((rows + 1) / 2, cols, num_sms)), unsigned(cols)), 256, 0, s>>>(
        rows, cols, X, ldx, Erow, Sh, L.lds);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_oz_slice_rinv<<<cols, 256, 0, s>>>(cols, Rinv, Trev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // every band's partial tiles stay in their own scratch; one reduction then
    // adds the bands (in order) and writes Y once
    TcPartials bands[OZ_S];
    for (int t = 2; t <= OZ_S + 1; ++t) {
        // sum over i + j = t: [S_1 .. S_{t-1}] [T_{t-1}; ..; T_1]
        QuantA q;
        q.data = Sh;
        q.ld = L.lds;
        q.m = rows;
        q.n = int64_t(t - 1) * cols;
        q.prec = PLU_BF16;
        const double* Tt = Trev + size_t(OZ_S + 1 - t) * cols;
        e = launch_tc_pass_q(0, q, Tt, int64_t(OZ_S) * cols, cols, Y, ldy,
                             base + L.pass_off + size_t(t - 2) * L.xr_band, L.xr_band, dev_status,
                             num_sms, s, 0, nullptr, &bands[t - 2]);
        if (e != cudaSuccess) return e;
    }
    return launch_tc_reduce_bands(bands, OZ_S, rows, cols, Y, ldy, s);
}

}  // namespace plu
