// Partial-pivoting LU of a tall FP64 panel (rows >= cols) with the trailing
// updates on the tensor cores: the re-orthogonalising [X, ~] = lu(X) of
// Alg. gpowerlu and the [L, U, P] = lu(Y), lu(B^T) of Alg. bpowerlu steps 4
// and 6, as the mixed-precision modes run them.  Pivots, tie rule, zero
// columns and outputs are those of launch_panel_lu (plu_panel.cu): rows stay
// in place and carry their current position (virtual pivoting); the pivot of
// column j is the largest |x| among the rows not yet pivoted, ties to the
// smallest current position (LAPACK's order).
//
// The columns are factored 32 at a time ("leaves").
//
// Leaf (k_lu_leaf, cooperative, one CTA per SM).  Each CTA keeps its rows of
// the leaf's columns in shared memory.  A column step is one grid-wide
// candidate exchange: every CTA stores a tagged key, one warp per CTA polls
// all keys until every tag is the step's, then reads the winner's record.
// Warp 0 runs the exchange; the other warps own the rows.  Per step they eliminate only the next column, so that the next
// candidate is ready, and apply the rest of the step's elimination to the
// leaf's later columns while the exchange is in flight.  The candidate row's
// later columns travel with its candidate, so the winner's U row needs no
// second read.  After the leaf, every warp of the grid forms one column of
// U12 = L11^{-1} X(pivot rows, later columns) by FP64 forward substitution,
// and cuts it into the digits the update kernel multiplies.
//
// Update (k_lu_update, tcgen05).  X(active rows, later columns) -=
// L(rows, leaf) U12 as a sum of exact products on the tensor cores.  Every
// multiplier row and every U12 column is scaled by its largest binary
// exponent and cut into six signed digits of 9 bits, each exact in FP16:
// x = sum_k n_k 2^(E - 1030 - 9(k-1)), |n_k| <= 256, up to a rounding of
// 2^(E - 1076).  A digit product is at most 2^16 and the digit pairs of equal
// weight (band t = k + j) add at most 6 x 32 of them, so the FP32 sums in
// TMEM are exact.  Bands 2..7 (21 digit pairs, 42 MMAs of K = 16 per 64
// columns) are combined in integers and rounded once to FP64; the dropped
// bands and the digit rounding leave less than 2^-51 of 32 max|l| max|u|,
// which is the size of an FP64 dot product's own rounding error bound.  (An
// error-free splitting in the manner of Ozaki's scheme, written for this
// operand shape.)  This replaces 32 FP64 FMAs per updated entry (GB300's FP64
// pipe retires under two per cycle per SM) by integer work and one FP64
// subtraction.
#include "plu_internal.h"
#include "plu_ptx.cuh"

#include <cuda_fp16.h>

#include <climits>

namespace plu {
namespace {

constexpr int LW = 32;          // leaf width (columns)
constexpr int LT = 256;         // leaf threads: warp 0 exchanges, warps 1-7 own rows
constexpr int LROWT = LT - 32;  // row-owning threads
constexpr int LMAXG = 256;      // largest leaf grid (one key per CTA, 8 per lane)
constexpr int RECW = 3 + LW;    // record (uint4): |x|, (pos, row), the row's leaf columns, 1 / pivot

constexpr int UM = 128;         // update tile rows (MMA M)
constexpr int UNC = 32;         // update columns per MMA chunk (MMA N)
constexpr int UMAXC = 8;        // chunks per update launch (256 columns)
constexpr int UBUF = 6 * UNC;   // TMEM columns of one chunk's six bands (two buffers)
constexpr int UEW = 16;         // update epilogue warps: 4 per TMEM lane quarter
constexpr int UT = (UEW + 2) * 32;   // update threads: epilogue warps, MMA warp, copy warp
constexpr int NDIG = 6;         // digits per value
constexpr int A_KSTEP = UM * 128;           // one 128-byte K step of the A image
constexpr int B_KSTEP = UNC * 128;
constexpr int B_CHUNK = 3 * B_KSTEP;        // 3 K steps: 6 digits x 32 values x 2 bytes
constexpr int A_IMG = 3 * A_KSTEP;

struct Cand {
    double v;
    int pos;
    int row;
};

__device__ __forceinline__ bool is_nan_abs(double a) {
    return __double_as_longlong(a) > 0x7FF0000000000000LL;
}

// true when a should be the pivot rather than b (see plu_panel.cu)
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
    if (a.row < 0) return false;
    if (b.row < 0) return true;
    const long long ab = __double_as_longlong(a.v), bb = __double_as_longlong(b.v);
    const bool an = ab > 0x7FF0000000000000LL, bn = bb > 0x7FF0000000000000LL;
    if (an || bn) return an && bn ? a.pos < b.pos : bn;
    if (ab > bb) return true;
    if (ab < bb) return false;
    return a.pos < b.pos;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int x) {
    Cand o;
    o.v = __shfl_xor_sync(0xffffffffu, c.v, x);
    o.pos = __shfl_xor_sync(0xffffffffu, c.pos, x);
    o.row = __shfl_xor_sync(0xffffffffu, c.row, x);
    return o;
}

// Lane of the warp's best candidate under `better`, in few steps:
// the largest |x| bit pattern by two redux maxima (high word, then low word
// among the lanes holding it), then the smallest position among the equal
// ones.  NaN candidates lose to every number, so they are left out; a warp
// without a finite candidate takes the full comparison rule.
__device__ __forceinline__ int warp_winner_lane(const Cand& c) {
    const int lane = threadIdx.x & 31;
    const bool fin = c.row >= 0 && !is_nan_abs(c.v);
    const unsigned long long b = fin ? (unsigned long long)__double_as_longlong(c.v) : 0ull;
    const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
    const unsigned mh = __reduce_max_sync(0xffffffffu, fin ? hi + 1u : 0u);   // |x| < 2^63: no wrap
    if (mh == 0) {
        Cand g = c;
        int gl = lane;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Cand o = shfl_cand(g, off);
            const int ol = __shfl_xor_sync(0xffffffffu, gl, off);
            if (better(o, g) || (!better(g, o) && ol < gl)) {
                g = o;
                gl = ol;
            }
        }
        return __shfl_sync(0xffffffffu, gl, 0);
    }
    const bool h1 = fin && hi + 1u == mh;
    const unsigned ml = __reduce_max_sync(0xffffffffu, h1 ? lo : 0u);
    const bool h2 = h1 && lo == ml;
    const unsigned mp = __reduce_min_sync(0xffffffffu, h2 ? unsigned(c.pos) : 0xFFFFFFFFu);
    return __ffs(__ballot_sync(0xffffffffu, h2 && unsigned(c.pos) == mp)) - 1;
}

__device__ __forceinline__ Cand shfl_cand_from(const Cand& c, int src) {
    Cand o;
    o.v = __shfl_sync(0xffffffffu, c.v, src);
    o.pos = __shfl_sync(0xffffffffu, c.pos, src);
    o.row = __shfl_sync(0xffffffffu, c.row, src);
    return o;
}

__device__ __forceinline__ uint4 ld_relaxed_v4(const void* p) {
    uint4 r;
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p)
                 : "memory");
    return r;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(void* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 32-bit key of a candidate for the exchange: the high word of |x| (monotone
// in |x|); 0 for no candidate and for NaN (both lose to every number).  Equal
// keys are resolved with the full records.
__device__ __forceinline__ unsigned cand_key(const Cand& c) {
    if (c.row < 0 || is_nan_abs(c.v)) return 0u;
    return unsigned((unsigned long long)__double_as_longlong(c.v) >> 32);
}
__device__ __forceinline__ void st_relaxed_v4(void* p, uint4 v) {
    asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 tagged(unsigned long long b, unsigned tag) {
    return make_uint4(unsigned(b), tag, unsigned(b >> 32), tag);
}
__device__ __forceinline__ unsigned long long untag(const uint4& q) {
    return (unsigned long long)q.x | ((unsigned long long)q.z << 32);
}
__device__ __forceinline__ bool has_tag(const uint4& q, unsigned tag) {
    return q.y == tag && q.w == tag;
}

// Six signed 9-bit digits of x relative to the biased exponent E (the largest
// biased exponent of its row or column, subnormals counted as 1):
// x = sum_k n_k 2^(E - 1030 - 9k) (k = 0..5) up to the rounding of x to a
// multiple of 2^(E - 1075), |n_k| <= 256.  Integer operations only.
__device__ __forceinline__ void digits9(double x, int E, int (&n)[NDIG]) {
    const long long b = __double_as_longlong(x);
    const int ex = int((b >> 52) & 0x7FF);
    long long m = b & 0xFFFFFFFFFFFFFLL;
    int e = 1;
    if (ex != 0) {
        m |= 1LL << 52;
        e = ex;
    }
    const int d = E - e;            // >= 0 for every value of the row
    long long F;
    if (m == 0 || d > 54) F = 0;
    else if (d <= 0) F = m;
    else F = (m + (1LL << (d - 1))) >> d;
    if (b < 0) F = -F;              // |F| <= 2^53
    long long R = F;
    n[0] = int((R + (1LL << 44)) >> 45);
    R -= (long long)n[0] << 45;
    n[1] = int((R + (1LL << 35)) >> 36);
    R -= (long long)n[1] << 36;
    n[2] = int((R + (1LL << 26)) >> 27);
    R -= (long long)n[2] << 27;
    n[3] = int((R + (1LL << 17)) >> 18);
    R -= (long long)n[3] << 18;
    n[4] = int((R + (1LL << 8)) >> 9);
    R -= (long long)n[4] << 9;
    n[5] = int(R);
}

__device__ __forceinline__ int biased_exp(double x) {
    const int ex = int((__double_as_longlong(x) >> 52) & 0x7FF);
    return ex == 0 ? 1 : ex;
}

// x - S 2^e2 with S = sum_t b_t 2^(9(7-t)), t = 2..7 (b[0] is band 2), the
// band sums exact integers below 2^24 in FP32.  S is formed exactly as a
// 128-bit integer and rounded once to FP64 (to nearest, ties away from
// zero), then subtracted: one FP64 operation.  Outside the normal exponent
// range the FP64 pipe forms the product instead.
__device__ __forceinline__ double sub_bands(const float (&b)[NDIG], double x, int e2) {
    const int i2 = __float2int_rn(b[0]), i3 = __float2int_rn(b[1]), i4 = __float2int_rn(b[2]);
    const int i5 = __float2int_rn(b[3]), i6 = __float2int_rn(b[4]), i7 = __float2int_rn(b[5]);
    const long long H = ((long long)i2 << 18) + ((long long)i3 << 9) + i4;   // |H| < 2^43
    const long long L = ((long long)i5 << 18) + ((long long)i6 << 9) + i7;   // |L| < 2^43
    const unsigned long long lo0 = (unsigned long long)H << 27;
    long long hi = H >> 37;
    unsigned long long lo = lo0 + (unsigned long long)L;
    hi += (L >> 63) + (lo < lo0 ? 1 : 0);
    const bool neg = hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0 ? 1 : 0);
    }
    const unsigned long long uh = (unsigned long long)hi;
    if (uh == 0 && lo == 0) return x;
    int p;
    unsigned long long top;
    if (uh != 0) {
        const int lz = __clzll((long long)uh);
        p = 127 - lz;
        top = lz == 0 ? uh : ((uh << lz) | (lo >> (64 - lz)));
    } else {
        const int lz = __clzll((long long)lo);
        p = 63 - lz;
        top = lo << lz;
    }
    unsigned long long m = (top >> 11) + ((top >> 10) & 1ull);
    int ex = p + e2 + 1023;
    if (m >> 53) {
        m >>= 1;
        ++ex;
    }
    if (ex < 1 || ex > 2046) {
        const double D = fma(__ll2double_rn(H), 134217728.0, __ll2double_rn(L));
        return x - ldexp(D, e2);
    }
    const unsigned long long bits = ((unsigned long long)(neg ? 1 : 0) << 63) |
                                    ((unsigned long long)ex << 52) | (m & ((1ull << 52) - 1));
    return x - __longlong_as_double((long long)bits);
}

// FP16 bit pattern of the integer v, |v| <= 256 (exact).
__device__ __forceinline__ unsigned short half_bits(int v) {
    return __half_as_ushort(__int2half_rn(v));
}

// Byte offset of digit k of K index c (0..31) in row r of a 128-byte-swizzled
// K-major operand image with 3 K steps of kstep bytes: digit k occupies
// bytes (k % 2) 64 + 2c of K step k / 2.
__device__ __forceinline__ uint32_t img_off(int r, int k, int c, int kstep) {
    const int boff = (k & 1) * 64 + 2 * c;
    const int ch = (boff >> 4) ^ (r & 7);
    return uint32_t((k >> 1) * kstep + r * 128 + (ch << 4) + (boff & 15));
}

// ------------------------------------------------------------------- leaf
// smem: P[LW][per] | PR[LW][LW] | L11[LW][LW] | pos_s[per] | piv_s[per] | prow_id[LW]
__global__ void __launch_bounds__(LT, 1)
k_lu_leaf(int64_t rows, int cols, double* __restrict__ X, int64_t ldx, int c0, int w,
          PanelHead* __restrict__ head, unsigned long long* __restrict__ keys,
          uint4* __restrict__ recs, double* __restrict__ Ubuf,
          int steps, int* __restrict__ pos_g, int* __restrict__ piv_g, int* __restrict__ status,
          int64_t budget, int per, unsigned bar_base, int first, unsigned char* __restrict__ bimg,
          int* __restrict__ fexp) {
    extern __shared__ __align__(16) double lsm[];
    double* P = lsm;
    double* PR = P + int64_t(LW) * per;
    double* L11 = PR + LW * LW;
    int* pos_s = reinterpret_cast<int*>(L11 + LW * LW);
    int* piv_s = pos_s + per;
    int* prow_id = piv_s + per;
    __shared__ Cand red[LT / 32];
    __shared__ Cand piv;
    __shared__ int ok_s;
    __shared__ int nan_seen;
    __shared__ double rinv_s;

    const int nb = gridDim.x;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = min(rows, r0 + per);
    const int R = int(r1 > r0 ? r1 - r0 : 0);
    unsigned nbar = bar_base;

    // ---- row state and the leaf's columns of own rows
    for (int r = t; r < R; r += LT) {
        if (first) {
            pos_s[r] = int(r0 + r);
            piv_s[r] = -1;
        } else {
            pos_s[r] = pos_g[r0 + r];
            piv_s[r] = piv_g[r0 + r];
        }
    }
    if (t == 0) nan_seen = 0;
    __syncthreads();
    for (int e = t; e < w * R; e += LT) {
        const int r = e % R, c = e / R;
        if (piv_s[r] < 0) P[c * per + r] = X[(r0 + r) + int64_t(c0 + c) * ldx];
    }
    __syncthreads();
    // each warp's candidate for the leaf's first column (warp 0 owns no rows)
    Cand best{-1.0, INT_MAX, -1};
    if (warp > 0) {
        for (int r = t - 32; r < R; r += LROWT) {
            if (piv_s[r] >= 0) continue;
            const double a = fabs(P[r]);
            if (is_nan_abs(a)) nan_seen = 1;
            const Cand c{a, pos_s[r], int(r0 + r)};
            if (better(c, best)) best = c;
        }
    }
    {
        const int wl = warp_winner_lane(best);
        const Cand wb = shfl_cand_from(best, wl);
        if (lane == 0) red[warp] = wb;
    }
    __syncthreads();
    bool pend = false;            // an elimination of the previous step is pending
    for (int sc = 0; sc < w; ++sc) {
        const int j = c0 + sc;
        const unsigned tag = unsigned(j) + 1u;
        const int64_t par = int64_t(j & 1) * nb;
        // ---- (1) the CTA's candidate for column sc (every warp reduces the
        // warps' candidates itself: no barrier)
        Cand cb = lane < LT / 32 ? red[lane] : Cand{-1.0, INT_MAX, -1};
        cb = shfl_cand_from(cb, warp_winner_lane(cb));
        const int rc = (cb.row >= 0) ? int(cb.row - r0) : -1;
        if (warp == 0) {
            // ---- (2) publish the candidate, its row's columns sc.. of the leaf
            // (with the pending elimination applied, and kept in P: this warp
            // owns that update of the candidate row) and its key.  Every word
            // carries the step's tag next to its value, so the arrival needs
            // no release and the reads no acquire: a reader polls until the
            // tags match.
            // The key goes out first: the readers poll the keys before they
            // read a record, so the record's stores and the reciprocal of the
            // pivot (one FP64 division, here instead of on every reader's
            // path) land while they poll.
            uint4* myrec = recs + (par + blockIdx.x) * RECW;
            if (lane == 0)
                st_relaxed_u64(keys + par + blockIdx.x,
                               (unsigned long long)cand_key(cb) | ((unsigned long long)tag << 32));
            double v = 0.0;
            if (rc >= 0 && lane >= sc && lane < w) {
                v = P[lane * per + rc];
                if (pend && lane > sc) {
                    v = fma(-P[(sc - 1) * per + rc], PR[(sc - 1) * LW + lane], v);
                    P[lane * per + rc] = v;
                }
                st_relaxed_v4(myrec + 2 + lane, tagged(__double_as_longlong(v), tag));
            }
            if (lane == 0) {
                st_relaxed_v4(myrec, tagged(__double_as_longlong(cb.v), tag));
                st_relaxed_v4(myrec + 1,
                              tagged((unsigned long long)unsigned(cb.pos) |
                                         ((unsigned long long)unsigned(cb.row) << 32),
                                     tag));
            }
            if (rc >= 0 && lane == sc)
                st_relaxed_v4(myrec + 2 + LW, tagged(__double_as_longlong(1.0 / v), tag));
            // ---- (3) every key (slot lane + 32 k), all loads in flight, polled
            // until each carries this step's tag (every CTA has published);
            // then the records of the slots holding the largest key
            int good = 1;
            constexpr int KPL = LMAXG / 32;
            unsigned kv[KPL];
            int64_t spins = 0;
            {
                unsigned ready = 0;
#pragma unroll
                for (int k = 0; k < KPL; ++k) {
                    kv[k] = 0;
                    if (lane + 32 * k >= nb) ready |= 1u << k;
                }
                while (true) {
                    unsigned long long wv[KPL];
#pragma unroll
                    for (int k = 0; k < KPL; ++k)
                        wv[k] = (ready & (1u << k)) ? 0ull : ld_relaxed_u64(keys + par + lane + 32 * k);
#pragma unroll
                    for (int k = 0; k < KPL; ++k) {
                        if (!(ready & (1u << k)) && unsigned(wv[k] >> 32) == tag) {
                            kv[k] = unsigned(wv[k]);
                            ready |= 1u << k;
                        }
                    }
                    if (__all_sync(0xffffffffu, ready == (1u << KPL) - 1u)) break;
                    if (++spins > budget) { good = 0; break; }
                    if ((spins & 63) == 0 &&
                        __any_sync(0xffffffffu, lane == 0 && ld_volatile_i32(status) != DEV_OK)) {
                        good = 0;     // another CTA gave up
                        break;
                    }
                }
                good = __all_sync(0xffffffffu, good);
            }
            Cand g{-1.0, INT_MAX, -1};
            int gs = -1;
            if (good) {
                unsigned mk = 0;
#pragma unroll
                for (int k = 0; k < KPL; ++k)
                    if (lane + 32 * k < nb) mk = max(mk, kv[k]);
                mk = __reduce_max_sync(0xffffffffu, mk);
                int nhit = 0;
#pragma unroll
                for (int k = 0; k < KPL; ++k) {
                    const unsigned bal = __ballot_sync(0xffffffffu, lane + 32 * k < nb && kv[k] == mk);
                    nhit += __popc(bal);
                    if (bal) gs = (__ffs(bal) - 1) + 32 * k;
                }
                if (nhit > 1) {
                    // equal keys: every lane reads the records of its tied slots
                    gs = -1;
#pragma unroll
                    for (int k = 0; k < KPL; ++k) {
                        const int b = lane + 32 * k;
                        if (b >= nb || kv[k] != mk || !good) continue;
                        const uint4* rb = recs + (par + b) * RECW;
                        uint4 q0, q1;
                        while (true) {
                            q0 = ld_relaxed_v4(rb);
                            q1 = ld_relaxed_v4(rb + 1);
                            if (has_tag(q0, tag) && has_tag(q1, tag)) break;
                            if (++spins > budget) { good = 0; break; }
                        }
                        const unsigned long long pr = untag(q1);
                        const Cand c{__longlong_as_double((long long)untag(q0)), int(unsigned(pr)),
                                     int(unsigned(pr >> 32))};
                        if (better(c, g)) { g = c; gs = b; }
                    }
                    good = __all_sync(0xffffffffu, good);
                    const int wl = warp_winner_lane(g);
                    gs = __shfl_sync(0xffffffffu, gs, wl);
                }
            }
            if (good && gs >= 0) {
                // the winning record, its row (lane c: column c) and the
                // reciprocal of its pivot in one round
                const uint4* rb = recs + (par + gs) * RECW;
                const bool want = lane >= sc && lane < w;
                uint4 q0 = make_uint4(0, tag, 0, tag), q1 = q0, qi = q0, qr = q0;
                while (true) {
                    if (lane == 0) {
                        q0 = ld_relaxed_v4(rb);
                        q1 = ld_relaxed_v4(rb + 1);
                        qi = ld_relaxed_v4(rb + 2 + LW);
                    }
                    if (want) qr = ld_relaxed_v4(rb + 2 + lane);
                    const bool ok = has_tag(q0, tag) && has_tag(q1, tag) && has_tag(qi, tag) &&
                                    has_tag(qr, tag);
                    if (__all_sync(0xffffffffu, ok)) break;
                    if (++spins > budget) { good = 0; break; }
                }
                good = __all_sync(0xffffffffu, good);
                const unsigned long long pr = untag(q1);
                g.v = __shfl_sync(0xffffffffu, __longlong_as_double((long long)untag(q0)), 0);
                g.pos = __shfl_sync(0xffffffffu, int(unsigned(pr)), 0);
                g.row = __shfl_sync(0xffffffffu, int(unsigned(pr >> 32)), 0);
                if (want) PR[sc * LW + lane] = __longlong_as_double((long long)untag(qr));
                if (lane == 0) rinv_s = __longlong_as_double((long long)untag(qi));
            }
            if (!good && lane == 0) atomicCAS(status, DEV_OK, DEV_TIMEOUT);
            if (lane == 0) {
                piv = g;
                prow_id[sc] = g.row;
                ok_s = good;
            }
        } else if (pend) {
            // ---- (3') the pending elimination of the later columns (not the
            // candidate row's: warp 0 did that one)
            for (int r = t - 32; r < R; r += LROWT) {
                if (piv_s[r] >= 0 || r == rc) continue;
                const double l = P[(sc - 1) * per + r];
                for (int c = sc + 1; c < w; ++c)
                    P[c * per + r] = fma(-l, PR[(sc - 1) * LW + c], P[c * per + r]);
            }
        }
        __syncthreads();
        if (!ok_s) return;
        const Cand pv = piv;
        if (pv.row < 0) {                 // no comparable candidate (non-finite panel)
            if (blockIdx.x == 0 && t == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
            return;
        }
        if (blockIdx.x == 0 && t == 0) {
            if (pv.v == 0.0 && head->info == 0) head->info = j + 1;
            if (!(pv.v <= 1.7976931348623157e308)) head->any_nan = 1;
        }
        const double ujj = PR[sc * LW + sc];
        const bool elim = ujj != 0.0;
        if (warp > 0) {
            // ---- (5) interchange on the positions of own rows, retire the
            // pivot row, multipliers of column sc and column sc + 1 of own
            // active rows, and the warp's candidate for column sc + 1
            best = Cand{-1.0, INT_MAX, -1};
            for (int r = t - 32; r < R; r += LROWT) {
                if (r0 + r == pv.row) {
                    pos_s[r] = j;
                    piv_s[r] = j;
                    continue;
                }
                if (pos_s[r] == j) pos_s[r] = pv.pos;
                if (piv_s[r] >= 0) continue;
                if (elim) {
                    const double l = lu_multiplier(P[sc * per + r], ujj, rinv_s);
                    P[sc * per + r] = l;
                    if (sc + 1 < w)
                        P[(sc + 1) * per + r] = fma(-l, PR[sc * LW + sc + 1], P[(sc + 1) * per + r]);
                }   // a zero pivot column keeps its zero multipliers and no update
                if (sc + 1 < w) {
                    const double a = fabs(P[(sc + 1) * per + r]);
                    if (is_nan_abs(a)) nan_seen = 1;
                    const Cand c{a, pos_s[r], int(r0 + r)};
                    if (better(c, best)) best = c;
                }
            }
            const int wl = warp_winner_lane(best);
            const Cand wb = shfl_cand_from(best, wl);
            if (lane == 0) red[warp] = wb;
        }
        pend = elim;
        // the warps' candidates, the pivot row and the new multipliers are
        // read by the next step
        __syncthreads();
        if (!ok_s) return;
    }
    // ---- leaf columns of own rows back to X (multipliers; pivot rows keep U11)
    for (int e = t; e < w * R; e += LT) {
        const int r = e % R, c = e / R;
        const int ps_r = piv_s[r];
        if (ps_r < 0 || ps_r >= c0) X[(r0 + r) + int64_t(c0 + c) * ldx] = P[c * per + r];
    }
    if (blockIdx.x == 0) {
        for (int e = t; e < w * w; e += LT) {
            const int sr = e % w, c = e / w;
            if (c >= sr) Ubuf[(c0 + sr) + int64_t(c0 + c) * steps] = PR[sr * LW + c];
        }
    }
    for (int r = t; r < R; r += LT) {
        pos_g[r0 + r] = pos_s[r];
        piv_g[r0 + r] = piv_s[r];
    }
    if (nan_seen) atomicExch(&head->any_nan, 1);
    const int c1 = c0 + w;
    if (c1 >= cols) return;
    // ---- every CTA's multipliers are in X after this barrier
    ++nbar;
    if (!grid_barrier(&head->barrier, nbar * unsigned(nb), status, budget)) return;
    // L11 (unit lower): rows prow_id[s], leaf columns t < s
    for (int e = t; e < w * w; e += LT) {
        const int s = e % w, c = e / w;
        L11[s * LW + c] = c < s ? __ldcg(&X[prow_id[s] + int64_t(c0 + c) * ldx]) : 0.0;
    }
    __syncthreads();
    // ---- U12, one column per warp of the grid, and its digit image
    const int N = cols - c1;
    const int npad = (N + UNC - 1) / UNC * UNC;
    const int gwarps = nb * (LT / 32);
    for (int n = blockIdx.x * (LT / 32) + warp; n < npad; n += gwarps) {
        double u = 0.0;
        if (n < N) {
            const int c = c1 + n;
            double x = lane < w ? __ldcg(&X[prow_id[lane] + int64_t(c) * ldx]) : 0.0;
            // forward substitution: after step s lane s holds u_s
            for (int s = 0; s < w; ++s) {
                const double us = __shfl_sync(0xffffffffu, x, s);
                if (lane > s && lane < w) x = fma(-L11[lane * LW + s], us, x);
            }
            u = lane < w ? x : 0.0;
            if (lane < w) Ubuf[(c0 + lane) + int64_t(c) * steps] = u;
        }
        const int E = __reduce_max_sync(0xffffffffu, u != 0.0 ? biased_exp(u) : 0);
        int dg[NDIG];
        digits9(u, E, dg);
        // digit image row n % UNC of chunk n / UNC; K index = lane
        unsigned char* img = bimg + int64_t(n / UNC) * B_CHUNK;
        const int rr = n % UNC;
#pragma unroll
        for (int k = 0; k < NDIG; ++k)
            *reinterpret_cast<unsigned short*>(img + img_off(rr, k, lane, B_KSTEP)) = half_bits(dg[k]);
        if (lane == 0) fexp[n] = E;
    }
}

// ----------------------------------------------------------------- update
struct UpdParams {
    int64_t rows;
    double* X;
    int64_t ldx;
    int c0, w;          // the leaf's columns (the multipliers)
    int c1;             // first column after the leaf
    int n0, ncols;      // this launch's columns: c1 + n0 .. c1 + n0 + ncols - 1
    int nchunks;        // ceil(ncols / UNC)
    const int* piv;     // pivot step per row (-1: not pivoted)
    const unsigned char* bimg;   // digit image of U12, chunk n0 / UNC onwards
    const int* fexp;    // column exponents, index n0 onwards
    int* status;
};

// Warps 0-15 build the digit image of a 128-row tile of multipliers (thread
// = row r = t % 128 and 8 of its 32 values) and then drain TMEM: warp e takes
// TMEM lane quarter e % 4 (its 32 rows) and 16 of the chunk's 64 columns.
// Warp 16 issues the MMAs, warp 17 copies the U12 digit image once.
__global__ void __launch_bounds__(UT, 1) k_lu_update(const UpdParams P) {
    extern __shared__ __align__(1024) unsigned char usm_raw[];
    __shared__ __align__(8) uint64_t b_full;
    __shared__ __align__(8) uint64_t mma_done[2];
    __shared__ __align__(8) uint64_t tmem_free[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int fex_s[UMAXC * UNC];
    __shared__ unsigned short htab[513];
    __shared__ int emax_s[4][UM];
    __shared__ int erow_s[UM];
    __shared__ int rflag_s[UM];          // bit 0: active row, bit 1: non-finite multipliers
    __shared__ volatile int abort_flag;

    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(usm_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* aimg = smem;
    unsigned char* bimg = smem + A_IMG;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    constexpr int MMA_WARP = UEW, COPY_WARP = UEW + 1;
    const uint32_t tcols = 512;

    if (t == 0) {
        abort_flag = 0;
        mbar_init(&b_full, 1);
        for (int q = 0; q < 2; ++q) {
            mbar_init(&mma_done[q], 1);
            mbar_init(&tmem_free[q], UEW);
        }
        mbar_init(&drain_bar, 1);
        fence_barrier_init();
    }
    for (int v = t; v < 513; v += UT) htab[v] = half_bits(v - 256);
    for (int n = t; n < P.nchunks * UNC; n += UT) fex_s[n] = n < P.ncols ? P.fexp[n] : 0;
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    if (warp == COPY_WARP && lane == 0) {
        const uint32_t bytes = uint32_t(P.nchunks) * B_CHUNK;
        mbar_arrive_expect_tx(&b_full, bytes);
        bulk_load(bimg, P.bimg, bytes, &b_full, policy_evict_last());
    }
    const int64_t ntiles = (P.rows + UM - 1) / UM;
    const int E_BIAS = 2105;      // 2 x 1030 + 45: S (band 7 units) to the product's scale
    uint32_t nround = 0;          // MMA rounds (chunks) issued by this CTA
    const int br = t & (UM - 1), bg = t >> 7;          // digit build: row, 8-value group
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- digit image of the tile's multiplier rows
        double x[8];
        const int64_t ib = tile * UM + br;
        bool act = false;
        if (warp < UEW) {
            act = ib < P.rows && P.piv[ib] < 0;
            int E = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * bg + q;
                x[q] = (act && c < P.w) ? P.X[ib + int64_t(P.c0 + c) * P.ldx] : 0.0;
                if (x[q] != 0.0) E = max(E, biased_exp(x[q]));
            }
            emax_s[bg][br] = E;
        }
        __syncthreads();
        if (warp < UEW) {
            const int E = max(max(emax_s[0][br], emax_s[1][br]), max(emax_s[2][br], emax_s[3][br]));
            const bool bad = E >= 2047;
            if (bg == 0) {
                erow_s[br] = E;
                rflag_s[br] = (act ? 1 : 0) | (bad ? 2 : 0);
            }
            uint32_t pk[NDIG][4];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int dg[NDIG];
                digits9(bad ? 0.0 : x[q], E, dg);
#pragma unroll
                for (int k = 0; k < NDIG; ++k) {
                    const uint32_t h = htab[dg[k] + 256];
                    if (q & 1) pk[k][q >> 1] |= h << 16;
                    else pk[k][q >> 1] = h;
                }
            }
#pragma unroll
            for (int k = 0; k < NDIG; ++k)
                *reinterpret_cast<uint4*>(aimg + img_off(br, k, 8 * bg, A_KSTEP)) =
                    make_uint4(pk[k][0], pk[k][1], pk[k][2], pk[k][3]);
            fence_proxy_async_smem();
        }
        __syncthreads();
        const int row = 32 * (warp & 3) + lane;        // epilogue: TMEM lane = tile row
        const int64_t i = tile * UM + row;
        const int cq = (warp >> 2) * 8;                 // epilogue: first column within a chunk
        for (int q = 0; q < P.nchunks; ++q) {
            if (warp == MMA_WARP) {
                if (lane == 0 && !abort_flag) {
                    // TMEM buffer nround % 2; its previous round (nround - 2) drained
                    const uint32_t buf = nround & 1u;
                    bool ok = mbar_wait(&b_full, 0, &abort_flag);
                    if (ok && nround >= 2)
                        ok = mbar_wait(&tmem_free[buf], ((nround >> 1) - 1) & 1u, &abort_flag);
                    if (!ok) {
                        abort_flag = 1;
                    } else {
                        tc_fence_after();
                        const uint32_t idesc = idesc_make(0 /* F16 */, UM, UNC);
                        const uint32_t abase = smem_u32(aimg);
                        const uint32_t bbase = smem_u32(bimg + q * B_CHUNK);
                        for (int tb = 2; tb <= 7; ++tb) {
                            int acc = 0;
                            for (int k = 1; k <= NDIG; ++k) {
                                const int jd = tb - k;
                                if (jd < 1 || jd > NDIG) continue;
                                const uint64_t ad = smem_desc(abase + ((k - 1) >> 1) * A_KSTEP, 16, 1024) +
                                                    uint64_t(((k - 1) & 1) * 4);
                                const uint64_t bd = smem_desc(bbase + ((jd - 1) >> 1) * B_KSTEP, 16, 1024) +
                                                    uint64_t(((jd - 1) & 1) * 4);
#pragma unroll
                                for (int s = 0; s < 2; ++s) {
                                    asm volatile(
                                        "{\n\t.reg .pred p;\n\t"
                                        "setp.ne.b32 p, %4, 0;\n\t"
                                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                            tmem + buf * UBUF + uint32_t((tb - 2) * UNC)),
                                        "l"(ad + uint64_t(2 * s)), "l"(bd + uint64_t(2 * s)), "r"(idesc),
                                        "r"(acc)
                                        : "memory");
                                    acc = 1;
                                }
                            }
                        }
                        tc_commit(&mma_done[buf]);
                    }
                }
                __syncwarp();
            } else if (warp < UEW) {
                // ---- epilogue: thread = row, 8 columns; X is read while the
                // MMAs of the chunk run
                const uint32_t buf = nround & 1u;
                const int fl = rflag_s[row];
                const int Er = erow_s[row];
                const int nb0 = q * UNC + cq;
                double xv[8];
                if ((fl & 1) && nb0 < P.ncols) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        xv[u] = (nb0 + u < P.ncols) ? P.X[i + int64_t(P.c1 + P.n0 + nb0 + u) * P.ldx]
                                                    : 0.0;
                }
                const bool ok = mbar_wait(&mma_done[buf], (nround >> 1) & 1u, &abort_flag);
                if (!ok) abort_flag = 1;
                tc_fence_after();
                if (ok) {
                    if (nb0 < P.ncols) {
                        uint32_t bv[NDIG][8];
#pragma unroll
                        for (int tb = 0; tb < NDIG; ++tb)
                            tmem_ld8(tmem + (uint32_t((warp & 3) * 32) << 16) + buf * UBUF +
                                         uint32_t(tb * UNC + cq),
                                     bv[tb]);
                        tmem_wait_ld();
                        if (fl & 1) {
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int n = nb0 + u;
                                if (n >= P.ncols) continue;
                                const int Fc = fex_s[n];
                                double y;
                                if ((fl & 2) || Fc >= 2047) {
                                    y = __longlong_as_double(0x7FF8000000000000LL);
                                } else {
                                    float bb[NDIG];
#pragma unroll
                                    for (int tb = 0; tb < NDIG; ++tb) bb[tb] = __uint_as_float(bv[tb][u]);
                                    y = sub_bands(bb, xv[u], Er + Fc - E_BIAS);
                                }
                                P.X[i + int64_t(P.c1 + P.n0 + n) * P.ldx] = y;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_free[buf]);
            }
            ++nround;
        }
        __syncthreads();
        if (abort_flag) break;
    }
    __syncthreads();
    if (abort_flag) {
        if (t == 0) atomicCAS(P.status, DEV_OK, DEV_TIMEOUT);
        if (warp == COPY_WARP && lane == 0) mbar_wait_drain(&b_full, 0);
        if (warp == MMA_WARP && lane == 0) {
            tc_commit(&drain_bar);
            mbar_wait_drain(&drain_bar, 0);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tcols)
                     : "memory");
    }
}

struct TcluLayout {
    size_t head, keys, recs, ubuf, pos, piv, bimg, fexp, total;
};

TcluLayout tclu_layout(int64_t rows, int cols) {
    TcluLayout L{};
    size_t off = 0;
    auto add = [&](size_t bytes) {
        const size_t o = (off + 255) & ~size_t(255);
        off = o + bytes;
        return o;
    };
    const int64_t steps = rows < cols ? rows : cols;
    L.head = add(panel_head_bytes());
    L.keys = add(size_t(2) * LMAXG * sizeof(unsigned long long));
    L.recs = add(size_t(2) * LMAXG * RECW * sizeof(uint4));
    L.ubuf = add(size_t(steps) * size_t(cols) * sizeof(double));
    L.pos = add(size_t(rows) * sizeof(int));
    L.piv = add(size_t(rows) * sizeof(int));
    const int nmax = cols > LW ? cols - LW : 0;
    const int chunks = (nmax + UNC - 1) / UNC;
    L.bimg = add(size_t(chunks) * B_CHUNK + 1024);
    L.fexp = add(size_t(chunks) * UNC * sizeof(int) + 256);
    L.total = off + 256;
    return L;
}

int leaf_grid(int64_t rows, int num_sms, int* per_out) {
    int64_t nb = (rows + 31) / 32;
    if (nb > num_sms) nb = num_sms;
    if (nb > LMAXG) nb = LMAXG;
    if (nb < 1) nb = 1;
    const int64_t per = (rows + nb - 1) / nb;
    nb = (rows + per - 1) / per;
    *per_out = int(per);
    return int(nb);
}

size_t leaf_smem(int per) {
    return size_t(LW) * per * 8 + size_t(2) * LW * LW * 8 + size_t(2) * per * 4 + LW * 4 + 64;
}

size_t update_smem(int nchunks) {
    // at least ~116 KB so that one CTA (with its 512 TMEM columns) runs per SM
    size_t b = size_t(A_IMG) + size_t(nchunks) * B_CHUNK + 1024;
    return b < 118 * 1024 ? 118 * 1024 : b;
}

}  // namespace

bool tclu_supported(int64_t rows, int cols, int num_sms) {
    if (cols < 1 || rows < cols || cols > 2048 || rows > (int64_t(1) << 31) - 1) return false;
    int per = 0;
    leaf_grid(rows, num_sms, &per);
    return leaf_smem(per) <= 200 * 1024;
}

size_t tclu_scratch_bytes(int64_t rows, int cols) { return tclu_layout(rows, cols).total; }

cudaError_t launch_panel_lu_tc(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                               int32_t* perm, double* L, int64_t ldL, int l_trans, double* U,
                               int64_t ldU, int u_trans, int32_t* info, void* scratch,
                               int* dev_status, int64_t spin_budget, int num_sms, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (!tclu_supported(rows, cols, num_sms)) return cudaErrorInvalidValue;
    const TcluLayout Ly = tclu_layout(rows, cols);
    char* base = static_cast<char*>(scratch);
    PanelHead* head = reinterpret_cast<PanelHead*>(base + Ly.head);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + Ly.keys);
    uint4* recs = reinterpret_cast<uint4*>(base + Ly.recs);
    double* Ubuf = reinterpret_cast<double*>(base + Ly.ubuf);
    int* pos = reinterpret_cast<int*>(base + Ly.pos);
    int* pivstep = reinterpret_cast<int*>(base + Ly.piv);
    unsigned char* bimg = reinterpret_cast<unsigned char*>(base + Ly.bimg);
    int* fexp = reinterpret_cast<int*>(base + Ly.fexp);
    int per = 0;
    const int nb = leaf_grid(rows, num_sms, &per);
    cudaError_t e = cudaMemsetAsync(head, 0, panel_head_bytes(), s);
    if (e != cudaSuccess) return e;
    // step tags start below every step number
    e = cudaMemsetAsync(keys, 0, size_t(2) * LMAXG * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(recs, 0, size_t(2) * LMAXG * RECW * sizeof(uint4), s);
    if (e != cudaSuccess) return e;
    const size_t lsm = leaf_smem(per);
    e = cudaFuncSetAttribute(k_lu_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lsm));
    if (e != cudaSuccess) return e;
    const int steps = int(rows < int64_t(cols) ? rows : int64_t(cols));
    const int64_t ntiles = (rows + UM - 1) / UM;
    const int ugrid = int(ntiles < num_sms ? ntiles : num_sms);
    // grid barriers the leaves have passed on head->barrier: one per leaf
    // that has later columns (the column steps themselves synchronise on the
    // step-tagged keys)
    unsigned bar = 0;
    for (int c0 = 0; c0 < steps; c0 += LW) {
        const int w = steps - c0 < LW ? steps - c0 : LW;
        int64_t rows_ = rows;
        int cols_ = cols, c0_ = c0, w_ = w, steps_ = steps, per_ = per;
        int first = c0 == 0 ? 1 : 0;
        int64_t ldx_ = ldx, budget = spin_budget;
        unsigned bar_ = bar;
        void* args[] = {&rows_, &cols_, &X, &ldx_, &c0_, &w_, &head, &keys, &recs, &Ubuf, &steps_,
                        &pos, &pivstep, &dev_status, &budget, &per_, &bar_, &first, &bimg, &fexp};
        count_launch();
        e = cudaLaunchCooperativeKernel((const void*)k_lu_leaf, dim3(unsigned(nb)), dim3(LT), args,
                                        lsm, s);
        if (e != cudaSuccess) return e;
        const int c1 = c0 + w;
        if (c1 >= cols) continue;
        bar += 1;
        const int N = cols - c1;
        for (int n0 = 0; n0 < N; n0 += UMAXC * UNC) {
            UpdParams up;
            up.rows = rows;
            up.X = X;
            up.ldx = ldx;
            up.c0 = c0;
            up.w = w;
            up.c1 = c1;
            up.n0 = n0;
            up.ncols = N - n0 < UMAXC * UNC ? N - n0 : UMAXC * UNC;
            up.nchunks = (up.ncols + UNC - 1) / UNC;
            up.piv = pivstep;
            up.bimg = bimg + size_t(n0 / UNC) * B_CHUNK;
            up.fexp = fexp + n0;
            up.status = dev_status;
            const size_t usm = update_smem(up.nchunks);
            e = cudaFuncSetAttribute(k_lu_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(usm));
            if (e != cudaSuccess) return e;
            count_launch();
            k_lu_update<<<ugrid, UT, usm, s>>>(up);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return launch_panel_finish(rows, cols, X, ldx, mode, perm, L, ldL, l_trans, U, ldU, u_trans,
                               info, head, pos, pivstep, Ubuf, dev_status, num_sms, s);
}

}  // namespace plu
