// Split-precision tensor-core passes (3xTF32) over an FP32 A: the products
// that enter PowerLU's result to first order (the last pass Y = A V(:, 1:k)
// of Alg. bpowerlu step 3, RandLU's B^T = A^T W, and the G, H passes of
// Alg. singlepasslu in PLU_TF32X3 mode), FP32-accurate on the tensor cores.
//
// A = A_hi + A_lo with A_hi the TF32 rounding of A (its top 11 significant
// bits) and A_lo the TF32 rounding of the exact remainder A - A_hi; the same
// for X (rounded to FP32 first).  Then
//   Y = A_hi X_hi + A_lo X_hi + A_hi X_lo
// drops A_lo X_lo (<= 2^-22 |A||X|) and the remainders' own rounding
// (<= 2^-22 each), so every product is accurate to a few FP32 units.  The
// sums accumulate in FP32 in TMEM over segments of at most 32 K steps (see
// plan_split: the accumulator adds shrink long sums) and in FP64 across
// segments and CTAs (k_split_reduce).
//
// The structure follows the TF32 pass (plu_tc.cu): one CTA per SM walks an
// equal share of the (128-row output block, 32-wide K step) space with all
// output columns in TMEM, so A is read from HBM once.  Three things differ.
// (1) The A tile is split in shared memory: for Y = A^T X the splitter warps
// rewrite the TMA-loaded K-major tile as A_hi in place and write A_lo beside
// it; for Y = A X the transposer warps write the K-major A_hi and A_lo tiles
// from the MN-major staging tile.  (2) The small operand's two images (hi
// and lo, pre-tiled by k_split_operand) stream through their own ring, one
// entry per image and column chunk (at most 256 columns, one MMA wide):
// head x head and remainder x head off the hi entry, head x remainder off the
// lo entry.  (3) The remainder products accumulate in TMEM columns of their
// own when there is room (up to 256 output columns), so the main sum takes
// one accumulator add per 8-wide K slice.
//
// Every mbarrier wait is bounded; on timeout the CTA raises the device error
// word, lets its in-flight copies land, waits for its MMAs and frees TMEM.
#include "plu_internal.h"
#include "plu_ptx.cuh"

namespace plu {
namespace {

constexpr int BM = 128;            // output rows per block (MMA M)
constexpr int BK = 32;             // FP32 K elements per stage (128 bytes)
constexpr int A_TILE = BM * 128;   // 16 KB
constexpr int NTHR = 384;          // 12 warps
constexpr int MAXR = 8;            // ring depths
constexpr int CHMAX = 256;         // small-operand rows per chunk (MMA N)

// warps: 0-1 A producers, 2 B producer, 3 MMA, 4-7 epilogue, 8-11 splitter
// (Y = A^T X) or transposer (Y = A X)
constexpr int APW = 2, BPW = 2, MMAW = 3, EPIW = 4, SPW = 8;

struct SplitParams {
    int64_t M, K;
    int npad;            // output columns padded: nch x chn
    int nch, chn;        // column chunks, rows per chunk (multiple of 16)
    int sseg;            // K steps per accumulation segment
    int nkc;             // K chunks (segments) per 128-row block: nkc x sseg K steps
    int sep;             // the remainder products accumulate in their own TMEM columns
    int64_t total, per;
    int max_segs;
    int sa, sk, sb;      // A ring, K-major ring (A X), small-operand ring
    int e_bytes;         // one ring entry: the hi or the lo image of a chunk, chn x 128 bytes
    uint32_t tmem_cols;
    float* part;         // [grid][max_segs][npad][128]
    double* norm_parts;  // nullable: per-CTA sums of squares of the A tiles
    int* status;
};

// v = hi + lo + r: hi the TF32 rounding (to nearest, ties away) of v, lo the
// TF32 rounding of the exact FP32 remainder v - hi, |r| <= 2^-22 |v|.
__device__ __forceinline__ void split_tf32(uint32_t v, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(__uint_as_float(v)));
    const float r = __fsub_rn(__uint_as_float(v), __uint_as_float(hi));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

template <bool XPOSE>
__global__ void __launch_bounds__(NTHR, 1)
k_tc_split(const __grid_constant__ CUtensorMap mapA, const unsigned char* __restrict__ Bimg,
           const SplitParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[MAXR];
    __shared__ __align__(8) uint64_t a_empty[MAXR];
    __shared__ __align__(8) uint64_t k_full[MAXR];     // split A operand ready
    __shared__ __align__(8) uint64_t k_empty[MAXR];
    __shared__ __align__(8) uint64_t b_full[MAXR];
    __shared__ __align__(8) uint64_t b_empty[MAXR];
    __shared__ __align__(8) uint64_t acc_full;
    __shared__ __align__(8) uint64_t acc_empty;
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // Y = A^T X: [A ring sa x 16 KB (A_hi in place)][A_lo ring sa x 16 KB][B ring]
    // Y = A X:   [staging sa x 16 KB][A_hi ring sk x 16 KB][A_lo ring sk x 16 KB][B ring]
    unsigned char* a_ring = smem;
    unsigned char* hi_ring = XPOSE ? a_ring + P.sa * A_TILE : a_ring;
    const int nk = XPOSE ? P.sk : P.sa;                 // slots of the split operand
    unsigned char* lo_ring = hi_ring + nk * A_TILE;
    unsigned char* b_ring = lo_ring + nk * A_TILE;

    const int64_t s0 = int64_t(blockIdx.x) * P.per;
    const int64_t s1 = min(P.total, s0 + P.per);
    const int nst = int(s1 > s0 ? s1 - s0 : 0);         // this CTA's stages

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int i = 0; i < P.sa; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], XPOSE ? 4 : 1);      // transposer warps / MMA commit
        }
        for (int i = 0; i < nk; ++i) {
            mbar_init(&k_full[i], 4);                   // splitter / transposer warps
            mbar_init(&k_empty[i], 1);                  // MMA commit
        }
        for (int i = 0; i < P.sb; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&b_empty[i], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 4);
        mbar_init(&drain_bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(P.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    int a_issued = 0, b_issued = 0;
    SqSum32 nsq;                     // splitter / transposer: this thread's share of ||A||^2
    const bool want_norm = P.norm_parts != nullptr;
    if (nst > 0) {
        if (warp < APW) {
            // -------------------------------------------- A producers
            if (lane == 0) {
                const uint64_t pol = policy_evict_first();
                for (int g = warp; g < nst; g += APW) {
                    const int slot = g % P.sa;
                    if (g >= P.sa &&
                        !mbar_wait(&a_empty[slot], uint32_t(g / P.sa - 1) & 1u, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const int64_t s = s0 + g;
                    const int64_t vb = s / P.sseg;           // (row block, K chunk)
                    const int64_t blk = vb / P.nkc;
                    const int kk = (int(vb % P.nkc) * P.sseg + int(s % P.sseg)) * BK;
                    unsigned char* dst = a_ring + slot * A_TILE;
                    mbar_arrive_expect_tx(&a_full[slot], uint32_t(A_TILE));
                    if (XPOSE) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            tma_load_2d(dst + q * (32 * 128), &mapA, &a_full[slot],
                                        int(blk * BM + 32 * q), kk, pol);
                    } else {
                        tma_load_2d(dst, &mapA, &a_full[slot], kk, int(blk * BM), pol);
                    }
                    a_issued = g + 1;
                }
            }
        } else if (warp == BPW) {
            // ------------------------------------ small-operand producer
            if (lane == 0) {
                const uint64_t pol = policy_evict_last();
                int h = 0;
                for (int g = 0; g < nst; ++g) {
                    const int64_t s = s0 + g;
                    const int kpos = int((s / P.sseg) % P.nkc) * P.sseg + int(s % P.sseg);
                    // entries (chunk c, hi), (chunk c, lo), in image order
                    for (int e = 0; e < 2 * P.nch; ++e, ++h) {
                        const int slot = h % P.sb;
                        if (h >= P.sb &&
                            !mbar_wait(&b_empty[slot], uint32_t(h / P.sb - 1) & 1u, &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        mbar_arrive_expect_tx(&b_full[slot], uint32_t(P.e_bytes));
                        bulk_load(b_ring + slot * P.e_bytes,
                                  Bimg + (int64_t(kpos) * 2 * P.nch + e) * P.e_bytes,
                                  uint32_t(P.e_bytes), &b_full[slot], pol);
                        b_issued = h + 1;
                    }
                    if (abort_flag) break;
                }
            }
        } else if (warp == MMAW) {
            // ------------------------------------------------------ MMA
            if (lane == 0) {
                const uint32_t idesc = idesc_make(2 /* TF32 */, BM, P.chn);
                int seg = 0, h = 0;
                int kpos = int(s0 % P.sseg);
                for (int g = 0; g < nst; ++g) {
                    const int64_t s = s0 + g;
                    const bool seg_first = (g == 0) || (kpos == 0);
                    const bool seg_last = (s + 1 == s1) || (kpos + 1 == P.sseg);
                    if (seg_first && seg > 0) {
                        if (!mbar_wait(&acc_empty, uint32_t(seg - 1) & 1u, &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                    }
                    const int ks = g % nk;
                    if (!mbar_wait(&k_full[ks], uint32_t(g / nk) & 1u, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ahi = smem_desc(smem_u32(hi_ring + ks * A_TILE), 16, 1024);
                    const uint64_t alo = smem_desc(smem_u32(lo_ring + ks * A_TILE), 16, 1024);
                    bool ok = true;
                    // per chunk: head x head into the main columns and the
                    // remainder x head into the remainder columns (their own
                    // when TMEM has room, so the main sum takes one
                    // accumulator add per 8-wide slice, not three) off the hi
                    // entry, then head x remainder off the lo entry
                    for (int c = 0; c < P.nch && ok; ++c) {
                        const uint32_t d = tmem + uint32_t(c * P.chn);
                        const uint32_t dl = P.sep ? d + uint32_t(P.npad) : d;
                        for (int part = 0; part < 2; ++part, ++h) {
                            const int bs = h % P.sb;
                            if (!mbar_wait(&b_full[bs], uint32_t(h / P.sb) & 1u, &abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t bd = smem_desc(smem_u32(b_ring + bs * P.e_bytes), 16, 1024);
                            if (part == 0) {
#pragma unroll
                                for (int sub = 0; sub < 4; ++sub) {
                                    const uint64_t o = uint64_t(2 * sub);
                                    const uint32_t acc0 = (seg_first && sub == 0) ? 0u : 1u;
                                    const uint32_t acc1 = P.sep ? acc0 : 1u;
                                    asm volatile(
                                        "{\n\t.reg .pred p, r;\n\t"
                                        "setp.ne.b32 p, %4, 0;\n\t"
                                        "setp.ne.b32 r, %7, 0;\n\t"
                                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t"
                                        "tcgen05.mma.cta_group::1.kind::tf32 [%6], %5, %2, %3, r;\n\t}\n"
                                        ::"r"(d), "l"(ahi + o), "l"(bd + o), "r"(idesc), "r"(acc0),
                                        "l"(alo + o), "r"(dl), "r"(acc1)
                                        : "memory");
                                }
                            } else {
#pragma unroll
                                for (int sub = 0; sub < 4; ++sub) {
                                    const uint64_t o = uint64_t(2 * sub);
                                    asm volatile(
                                        "{\n\t.reg .pred q;\n\t"
                                        "setp.eq.b32 q, %3, %3;\n\t"
                                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}\n"
                                        ::"r"(dl), "l"(ahi + o), "l"(bd + o), "r"(idesc)
                                        : "memory");
                                }
                            }
                            tc_commit(&b_empty[bs]);
                        }
                    }
                    if (!ok) {
                        abort_flag = 1;
                        break;
                    }
                    tc_commit(&k_empty[ks]);
                    if (!XPOSE) tc_commit(&a_empty[g % P.sa]);     // the same slot index
                    if (seg_last) {
                        tc_commit(&acc_full);
                        ++seg;
                    }
                    if (++kpos == P.sseg) kpos = 0;
                }
            }
        } else if (warp >= SPW && warp < SPW + 4) {
            const int m = threadIdx.x - 32 * SPW;     // 0..127
            if (!XPOSE) {
                // ------------------------------------------- splitter
                // 16-byte word m + 128 q of the K-major tile: the same word
                // of the hi (in place) and lo tiles
                for (int g = 0; g < nst; ++g) {
                    const int slot = g % P.sa;
                    if (!mbar_wait(&a_full[slot], uint32_t(g / P.sa) & 1u, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    uint4* hi = reinterpret_cast<uint4*>(a_ring + slot * A_TILE);
                    uint4* lo = reinterpret_cast<uint4*>(lo_ring + slot * A_TILE);
#pragma unroll
                    for (int q = 0; q < A_TILE / 16 / 128; ++q) {
                        uint4 v = hi[m + 128 * q];
                        uint4 l;
                        uint32_t* vv = reinterpret_cast<uint32_t*>(&v);
                        uint32_t* ll = reinterpret_cast<uint32_t*>(&l);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            uint32_t h;
                            if (want_norm) nsq.add(__uint_as_float(vv[e]));
                            split_tf32(vv[e], h, ll[e]);
                            vv[e] = h;
                        }
                        hi[m + 128 * q] = v;
                        lo[m + 128 * q] = l;
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&k_full[slot]);
                }
            } else {
                // ----------------------------------------- transposer
                // thread m owns row m of the tile: staging box q = m / 32
                // holds A(32 q.., k) as 32 K-rows of 128 bytes (swizzled);
                // the K-major tiles hold row m as 128 bytes, 16-byte chunk c
                // (K = 4c .. 4c + 3) at chunk c ^ (m % 8)
                const int q = m / 32, mm = m % 32;
                for (int g = 0; g < nst; ++g) {
                    const int sa_ = g % P.sa, sk_ = g % P.sk;
                    if (!mbar_wait(&a_full[sa_], uint32_t(g / P.sa) & 1u, &abort_flag) ||
                        (g >= P.sk &&
                         !mbar_wait(&k_empty[sk_], uint32_t(g / P.sk - 1) & 1u, &abort_flag))) {
                        abort_flag = 1;
                        break;
                    }
                    const unsigned char* raw = a_ring + sa_ * A_TILE + q * (32 * 128);
                    unsigned char* th = hi_ring + sk_ * A_TILE;
                    unsigned char* tl = lo_ring + sk_ * A_TILE;
                    const int in_chunk = (mm % 4) * 4;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        uint32_t wh[4], wl[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int kr = c * 4 + e;
                            const uint32_t v = *reinterpret_cast<const uint32_t*>(
                                raw + kr * 128 + (((mm / 4) ^ (kr & 7)) << 4) + in_chunk);
                            if (want_norm) nsq.add(__uint_as_float(v));
                            split_tf32(v, wh[e], wl[e]);
                        }
                        const int off = m * 128 + ((c ^ (m & 7)) << 4);
                        *reinterpret_cast<uint4*>(th + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                        *reinterpret_cast<uint4*>(tl + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&k_full[sk_]);
                        mbar_arrive(&a_empty[sa_]);     // the staging slot may be refilled
                    }
                }
            }
        } else if (warp >= EPIW && warp < EPIW + 4) {
            // -------------------------------------------------- epilogue
            const int quarter = warp & 3;
            const int row = quarter * 32 + lane;
            int seg = 0;
            for (int64_t s = s0; s < s1;) {
                const int64_t vb = s / P.sseg;
                const int64_t next = min(s1, (vb + 1) * int64_t(P.sseg));
                if (!mbar_wait(&acc_full, uint32_t(seg) & 1u, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                float* dst = P.part + (int64_t(blockIdx.x) * P.max_segs + seg) *
                                          int64_t(P.npad) * BM;
                const uint32_t lane_base = tmem + (uint32_t(quarter * 32) << 16);
                for (int c0 = 0; c0 < P.npad; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(lane_base + uint32_t(c0), r);
                    if (P.sep) {
                        uint32_t rl[32];
                        tmem_ld32(lane_base + uint32_t(P.npad + c0), rl);
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            r[j] = __float_as_uint(__fadd_rn(__uint_as_float(r[j]),
                                                             __uint_as_float(rl[j])));
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < P.npad) dst[int64_t(c0 + j) * BM + row] = __uint_as_float(r[j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty);
                ++seg;
                s = next;
            }
        }
    }
    if (want_norm) {
        // every A entry is split by exactly one thread of one CTA (the
        // stream-K stages partition the tiles; padding reads as zero)
        const double tot = cta_sum(nsq.value());
        if (threadIdx.x == 0) P.norm_parts[blockIdx.x] = tot;
    }
    __syncthreads();
    if (abort_flag) {
        if (threadIdx.x == 0) atomicCAS(P.status, DEV_OK, DEV_TIMEOUT);
        // let the issued copies land before shared memory goes away
        if (warp < APW && lane == 0) {
            for (int g = a_issued - 1; g >= 0 && g > a_issued - 1 - P.sa; g -= APW)
                mbar_wait_drain(&a_full[g % P.sa], uint32_t(g / P.sa) & 1u);
        }
        if (warp == BPW && lane == 0) {
            for (int h = b_issued - 1; h >= 0 && h > b_issued - 1 - P.sb; --h)
                mbar_wait_drain(&b_full[h % P.sb], uint32_t(h / P.sb) & 1u);
        }
        if (warp == MMAW && lane == 0) {
            tc_commit(&drain_bar);
            mbar_wait_drain(&drain_bar, 0);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(P.tmem_cols)
                     : "memory");
    }
}

// The small operand X (FP64, K x cols) as the split pass reads it: for each
// K step t and column chunk c, the hi image (chn rows of 128 bytes: row j =
// column c chn + j, TF32 rounding of X) followed by the lo image (TF32
// rounding of X - X_hi), both in the 128-byte-swizzled K-major layout
// (16-byte chunk u of row j at chunk u ^ (j % 8)).  Zero beyond cols and K.
__global__ void k_split_operand(int64_t K, int cols, int nch, int chn, int ksteps,
                                const double* __restrict__ X, int64_t ldx,
                                unsigned char* __restrict__ out) {
    const int col = blockIdx.y;                       // 0 .. nch chn - 1
    const int c = col / chn, j = col % chn;
    const int64_t kall = int64_t(ksteps) * BK;
    const int64_t blk_bytes = int64_t(chn) * 128;
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < kall;
         k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = k / BK;
        const int kk = int(k % BK);
        const bool live = col < cols && k < K;
        const double x = live ? X[k + int64_t(col) * ldx] : 0.0;
        uint32_t hi, lo;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(float(x)));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(float(x - double(__uint_as_float(hi)))));
        unsigned char* base = out + (t * nch + c) * 2 * blk_bytes + j * 128 +
                              (((kk / 4) ^ (j & 7)) << 4) + (kk % 4) * 4;
        *reinterpret_cast<uint32_t*>(base) = hi;
        *reinterpret_cast<uint32_t*>(base + blk_bytes) = lo;
    }
}

struct SplitPlan {
    int npad, nch, chn, ksteps, sseg, nkc, sep, sa, sk, sb, max_segs, grid, e_bytes;
    int64_t blocks, total, per;
    uint32_t tmem_cols;
    size_t smem;
    bool ok;
};

// Segment length.  The tensor cores' FP32 accumulator adds shrink the running
// sum (measured: a 32768-long K in one accumulator lost ~2e-4 relative, about
// 2^-24 per add times a third of the adds), so each accumulator covers at most
// kSegSep (remainders in their own columns: one main add per 8-wide slice) or
// kSegOne (all three products in one accumulator) K steps of 32, and the
// segments are summed in FP64.  The K steps are padded to nkc equal segments
// (the padding reads zeros).  Everything here depends on K and cols only, so
// an operand image made once serves every pass with the same K and cols.
constexpr int kSegSep = 32, kSegOne = 16, kMaxChunks = 128;

SplitPlan plan_split(int64_t M, int64_t K, int cols, int num_sms, bool xpose) {
    SplitPlan p{};
    const int n16 = (cols + 15) / 16 * 16;
    p.nch = (n16 + CHMAX - 1) / CHMAX;
    p.chn = ((n16 + p.nch - 1) / p.nch + 15) / 16 * 16;
    p.npad = p.nch * p.chn;
    const int n32 = (p.npad + 31) / 32 * 32;              // columns the epilogue reads
    p.sep = (p.npad + n32 <= 512) ? 1 : 0;
    const int64_t ks_real = (K + BK - 1) / BK;
    const int target = p.sep ? kSegSep : kSegOne;
    int64_t nkc = (ks_real + target - 1) / target;
    if (nkc > kMaxChunks) nkc = kMaxChunks;
    p.nkc = int(nkc);
    p.sseg = int((ks_real + nkc - 1) / nkc);
    p.ksteps = p.nkc * p.sseg;                             // padded K steps
    p.blocks = (M + BM - 1) / BM;
    p.total = p.blocks * p.ksteps;
    p.grid = num_sms;
    if (p.grid > p.total) p.grid = int(p.total);
    p.per = (p.total + p.grid - 1) / p.grid;
    p.grid = int((p.total + p.per - 1) / p.per);
    p.max_segs = int((p.per + p.sseg - 1) / p.sseg) + 1;
    p.e_bytes = p.chn * 128;
    // rings within 225 KB of dynamic shared memory (with the 1 KB alignment
    // pad; the static part is under 2 KB of the 227 KB): two split-operand
    // slots for Y = A X, small-operand entries for two K steps (at most eight),
    // and every remaining A slot (at least two, even, at most MAXR)
    const int budget = 225 * 1024 - 1024;
    p.sk = xpose ? 2 : 0;
    const int per_a = xpose ? A_TILE : 2 * A_TILE;          // A^T X: hi in place + lo
    int sb = 4 * p.nch;
    if (sb > MAXR) sb = MAXR;
    while (sb > 2 && budget - sb * p.e_bytes - 2 * p.sk * A_TILE < 2 * per_a) --sb;
    p.sb = sb;
    int sa = (budget - p.sb * p.e_bytes - 2 * p.sk * A_TILE) / per_a;
    if (sa > MAXR) sa = MAXR;
    sa = sa / APW * APW;                                     // slots alternate over the producers
    p.sa = sa;
    p.ok = p.sa >= APW && p.npad <= 512;
    p.smem = size_t(xpose ? p.sa + 2 * p.sk : 2 * p.sa) * A_TILE + size_t(p.sb) * p.e_bytes + 1024;
    uint32_t tc = 32;
    while (tc < uint32_t(p.sep ? p.npad + n32 : n32)) tc <<= 1;
    p.tmem_cols = tc;
    return p;
}

// Y(i, j) (+)= the FP64 sum over the K chunks of row block i / 128, and over
// the CTAs whose stage range touches each chunk, of their FP32 partial tiles,
// in chunk and CTA order.  CTA (blk, g): rows blk*128 + threadIdx.x, columns
// 8 g .. 8 g + 7.  Thread kc < nkc lists chunk kc's (CTA, segment) tiles in
// shared memory (at most nkc + grid + 1 of them: a chunk boundary or a CTA
// boundary starts each one).
constexpr int RJ = 8;
__global__ void __launch_bounds__(BM) k_split_reduce(const float* __restrict__ part, int64_t M,
                                                     int cols, int npad, int sseg, int nkc,
                                                     int64_t per, int max_segs, int grid,
                                                     double* __restrict__ Y, int64_t ldy,
                                                     int accum) {
    extern __shared__ int64_t src[];                 // part offsets of the tiles
    __shared__ int cnt[kMaxChunks + 1];
    // the column groups of a block adjacent in launch order (they read the
    // same partial tiles)
    const int ncg = (cols + RJ - 1) / RJ;
    const int64_t blk = blockIdx.x / ncg;
    const int r = threadIdx.x;
    int64_t c_lo = 0, c_hi = -1, vb = 0;
    if (r < nkc) {
        vb = blk * nkc + r;
        const int64_t first = vb * sseg, last = first + sseg - 1;
        c_lo = first / per;
        c_hi = last / per;
        if (c_hi >= grid) c_hi = grid - 1;
        cnt[r + 1] = int(c_hi - c_lo + 1);
    }
    __syncthreads();
    if (r == 0) {
        cnt[0] = 0;
        for (int t = 1; t <= nkc; ++t) cnt[t] += cnt[t - 1];
    }
    __syncthreads();
    if (r < nkc) {
        int o = cnt[r];
        for (int64_t c = c_lo; c <= c_hi; ++c) {
            const int64_t seg = vb - (c * per) / sseg;
            src[o++] = (c * max_segs + seg) * int64_t(npad) * BM;
        }
    }
    __syncthreads();
    const int nsrc = cnt[nkc];
    const int64_t i = blk * BM + r;
    if (i >= M) return;
    const int j0 = int(blockIdx.x % ncg) * RJ;
    const int nj = min(RJ, cols - j0);
    // compensated FP32 sums: as accurate as FP64 sums of the FP32 tiles, with
    // one FP64 addition per output instead of two FP64 operations per tile
    Sum2f acc[RJ];
    // four tiles' loads in flight before their additions (the kernel waits on
    // memory latency otherwise)
    constexpr int TU = 4;
    for (int t0 = 0; t0 < nsrc; t0 += TU) {
        float v[TU][RJ];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            const float* p = part + src[min(t0 + u, nsrc - 1)] + int64_t(j0) * BM + r;
#pragma unroll
            for (int q = 0; q < RJ; ++q) v[u][q] = (q < nj) ? p[int64_t(q) * BM] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < TU; ++u)
            if (t0 + u < nsrc) {
#pragma unroll
                for (int q = 0; q < RJ; ++q)
                    if (q < nj) acc[q].add(v[u][q]);
            }
    }
#pragma unroll
    for (int q = 0; q < RJ; ++q)
        if (q < nj) {
            double* y = Y + i + int64_t(j0 + q) * ldy;
            *y = accum ? *y + acc[q].value() : acc[q].value();
        }
}

// Y (rows x cols, ld ldy) = X rounded to FP32 (nearest even), X FP64 (ld ldx).
// CTA row blockIdx.y strides over the columns, x over the rows (no division
// per element).
__global__ void k_to_f32_ld(int64_t rows, int cols, const double* __restrict__ X, int64_t ldx,
                            float* __restrict__ Y, int64_t ldy) {
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
             i += int64_t(gridDim.x) * blockDim.x)
            Y[i + j * ldy] = f64_to_f32_rn(X[i + j * ldx]);
}

}  // namespace

size_t tcs_product_scratch_bytes(int64_t rows, int k, int num_sms) {
    const int64_t ld = (rows + 3) / 4 * 4;
    return ((size_t(ld) * k * sizeof(float) + 255) & ~size_t(255)) +
           tcs_scratch_bytes(rows, k, k, num_sms) + 256;
}

cudaError_t launch_tcs_product(int64_t rows, int k, const double* X, int64_t ldx, const double* T,
                               int64_t ldt, double* Y, int64_t ldy, void* scratch,
                               size_t scratch_cap, int* dev_status, int num_sms, cudaStream_t s) {
    if (rows < 1 || k < 1) return cudaSuccess;
    if (scratch_cap < tcs_product_scratch_bytes(rows, k, num_sms)) return cudaErrorInvalidValue;
    const int64_t ld = (rows + 3) / 4 * 4;
    const size_t xb = (size_t(ld) * k * sizeof(float) + 255) & ~size_t(255);
    char* base = static_cast<char*>(scratch);
    base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255));
    float* X32 = reinterpret_cast<float*>(base);
    if (!tcs_supported(rows, k, k, X32, ld, 0)) return cudaErrorInvalidValue;
    {
        // about 16 CTAs of 256 threads per SM over (row chunks) x (columns)
        const int64_t gy = k < 65535 ? k : 65535;
        int64_t gx = (rows + 255) / 256;
        const int64_t want = int64_t(num_sms) * 16;
        if (gx * gy > want) gx = (want + gy - 1) / gy;
        if (gx < 1) gx = 1;
        count_launch();
        k_to_f32_ld<<<dim3(unsigned(gx), unsigned(gy)), 256, 0, s>>>(rows, k, X, ldx, X32, ld);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_tc_split_pass(0, rows, k, X32, ld, T, ldt, k, Y, ldy, base + xb,
                                scratch_cap - xb - size_t(base - static_cast<char*>(scratch)),
                                dev_status, num_sms, s);
}

bool tcs_supported(int64_t M, int64_t K, int cols, const void* A, int64_t lda, int trans) {
    if (cols < 1 || cols > 512 || M < 1 || K < 1) return false;
    if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda % 4) != 0) return false;
    if (M > (int64_t(1) << 31) - 256 || K > (int64_t(1) << 31) - 256) return false;
    return plan_split(M, K, cols, 152, trans == 0).ok;
}

size_t tcs_operand_bytes(int64_t K, int cols) {
    const SplitPlan p = plan_split(128, K, cols, 1, false);
    return size_t(p.ksteps) * 2 * p.nch * p.e_bytes;
}

cudaError_t launch_tcs_operand(int64_t K, int cols, const double* X, int64_t ldx, void* out,
                               int num_sms, cudaStream_t s) {
    if (cols < 1 || cols > 512 || K < 1) return cudaErrorInvalidValue;
    const SplitPlan p = plan_split(128, K, cols, 1, false);
    int64_t b = (int64_t(p.ksteps) * BK + 255) / 256;
    const int64_t bcap = (int64_t(num_sms) * 16 + p.npad - 1) / p.npad;
    if (b > bcap) b = bcap;
    count_launch();
    k_split_operand<<<dim3(unsigned(b), unsigned(p.npad)), 256, 0, s>>>(
        K, cols, p.nch, p.chn, p.ksteps, X, ldx, static_cast<unsigned char*>(out));
    return cudaGetLastError();
}

size_t tcs_scratch_bytes(int64_t M, int64_t K, int cols, int num_sms) {
    size_t best = 0;
    for (int xp = 0; xp < 2; ++xp) {
        const SplitPlan p = plan_split(M, K, cols, num_sms, xp != 0);
        const size_t part = size_t(p.grid) * p.max_segs * p.npad * BM * sizeof(float);
        const size_t img = size_t(p.ksteps) * 2 * p.nch * p.e_bytes;
        const size_t b = part + 256 + img + 256;
        if (b > best) best = b;
    }
    return best;
}

cudaError_t launch_tc_split_pass(int trans, int64_t m, int64_t n, const float* A, int64_t lda,
                                 const double* X, int64_t ldx, int cols, double* Y, int64_t ldy,
                                 void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                                 cudaStream_t s, int accum, const void* ximg_pre,
                                 const NormOut* norm) {
    const int64_t M = trans ? n : m;
    const int64_t K = trans ? m : n;
    if (!tcs_supported(M, K, cols, A, lda, trans)) return cudaErrorInvalidValue;
    const SplitPlan p = plan_split(M, K, cols, num_sms, trans == 0);
    if (!p.ok || scratch_cap < tcs_scratch_bytes(M, K, cols, num_sms)) return cudaErrorInvalidValue;
    if (norm && (!norm->parts || !norm->out || p.grid > norm->cap)) return cudaErrorInvalidValue;
    Workspace w;
    w.base = static_cast<char*>(scratch);
    w.cap = scratch_cap;
    float* part = static_cast<float*>(w.take(size_t(p.grid) * p.max_segs * p.npad * BM * sizeof(float)));
    unsigned char* img =
        static_cast<unsigned char*>(w.take(size_t(p.ksteps) * 2 * p.nch * p.e_bytes));
    if (!part || !img) return cudaErrorInvalidValue;
    cudaError_t e;
    if (ximg_pre) {
        img = static_cast<unsigned char*>(const_cast<void*>(ximg_pre));
    } else if ((e = launch_tcs_operand(K, cols, X, ldx, img, num_sms, s)) != cudaSuccess) {
        return e;
    }
    CUtensorMap mapA;
    if (!tc_make_map_2d(&mapA, 4, A, uint64_t(m), uint64_t(n), uint64_t(lda) * 4, 32,
                        trans ? 128 : 32))
        return cudaErrorInvalidValue;
    SplitParams P;
    P.M = M;
    P.K = K;
    P.npad = p.npad;
    P.nch = p.nch;
    P.chn = p.chn;
    P.sseg = p.sseg;
    P.nkc = p.nkc;
    P.sep = p.sep;
    P.total = p.total;
    P.per = p.per;
    P.max_segs = p.max_segs;
    P.sa = p.sa;
    P.sk = p.sk;
    P.sb = p.sb;
    P.e_bytes = p.e_bytes;
    P.tmem_cols = p.tmem_cols;
    P.part = part;
    P.norm_parts = norm ? norm->parts : nullptr;
    P.status = dev_status;
    if (trans) {
        e = cudaFuncSetAttribute(k_tc_split<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(p.smem));
        if (e != cudaSuccess) return e;
        count_launch();
        k_tc_split<false><<<p.grid, NTHR, p.smem, s>>>(mapA, img, P);
    } else {
        e = cudaFuncSetAttribute(k_tc_split<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(p.smem));
        if (e != cudaSuccess) return e;
        count_launch();
        k_tc_split<true><<<p.grid, NTHR, p.smem, s>>>(mapA, img, P);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (norm && (e = launch_sum_partials(norm->parts, p.grid, norm->out, s)) != cudaSuccess)
        return e;
    count_launch();
    k_split_reduce<<<unsigned(p.blocks * ((cols + RJ - 1) / RJ)), BM,
                     size_t(p.nkc + p.grid) * sizeof(int64_t), s>>>(
        part, M, cols, p.npad, p.sseg, p.nkc, p.per, p.max_segs, p.grid, Y, ldy, accum);
    return cudaGetLastError();
}

}  // namespace plu
