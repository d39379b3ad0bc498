// Tensor-core passes over A on sm_103a: tcgen05.mma (kind::tf32, FP32
// accumulation in TMEM) fed by TMA, for the products Y = A X and Y = A^T X
// of Alg. gpowerlu / Alg. bpowerlu when A is stored in FP32.
//
// Shape of the problem: A is m x n (large), the other operand is K x l with
// l <= 512 (the sketch width).  One CTA per SM walks an equal share of the
// (128-row output block, 32-wide K step) iteration space ("stream-K"): each
// CTA's output rows x all l columns live in TMEM (<= 512 FP32 columns), so
// every byte of A is read from HBM exactly once, and the small operand is
// re-read from L2.  A CTA ends at most a few output blocks ("segments");
// their partial sums go to a scratch buffer and a second kernel adds the
// contributions of each block in CTA order in FP64 (deterministic).
//
// Operand layouts in shared memory are the canonical 128-byte-swizzled
// layouts written by TMA (SWIZZLE_128B) and read by the MMA through shared
// memory descriptors:
//   * Y = A^T X: the MMA's A operand is A^T, contiguous along K (= rows of
//     A): K-major, 128 rows x 128 bytes per 32-wide K step;
//   * Y = A X:   the MMA's A operand is A itself, contiguous along M (= rows
//     of A): four 32-row x 32-column TMA boxes per K step land in a staging
//     buffer and four transposer warps rewrite the 128 x 32 tile into the
//     same K-major swizzled layout (float4 stores, conflict-free), then
//     fence the generic-proxy writes for the tensor core;
//   * the small operand (converted to FP32, zero-padded to Npad columns) is
//     K-major in both cases.
// Warp roles: up to four warps issue the copies (A tiles and slices of the
// small operand), one thread issues the MMAs, four warps drain TMEM to the
// partial buffer and, for Y = A X, four warps transpose.  Every wait on an
// mbarrier is bounded; on timeout the CTA raises the device error word,
// lets its in-flight copies land, frees its TMEM and returns.
#include "plu_internal.h"
#include "plu_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace plu {
namespace {

constexpr int TC_THREADS = 320;   // Y = A^T X
constexpr int TC_THREADS_X = 448; // Y = A X (with transposer warps)
constexpr int NPA_MAX = 4;        // warps issuing the TMA loads of A
constexpr int BM = 128;           // rows of an output block (MMA M)
constexpr int BKB = 128;          // bytes of K per stage (one swizzle row)
constexpr int A_TILE = BM * BKB;  // 16 KB

// Operand kinds of the passes: element bytes E, K elements per 128-byte
// swizzle row = 128 / E, one MMA consumes 32 bytes of K (8, 16, 32 elements).
enum TcKind { KIND_TF32 = 0, KIND_BF16 = 1, KIND_FP8 = 2 };
template <int KIND> struct Kind;
template <> struct Kind<KIND_TF32> { static constexpr int E = 4; static constexpr uint32_t fmt = 2; };
template <> struct Kind<KIND_BF16> { static constexpr int E = 2; static constexpr uint32_t fmt = 1; };
template <> struct Kind<KIND_FP8>  { static constexpr int E = 1; static constexpr uint32_t fmt = 0; };

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accumulate) {
    if constexpr (KIND == KIND_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (KIND == KIND_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

struct TcParams {
    int64_t M;          // output rows
    int64_t K;          // reduction length
    int npad;           // padded output columns (multiple of 16, <= 512)
    int nchunk;         // columns per MMA (npad or npad / 2, <= 256)
    int ksteps;         // K steps (of 128 bytes) per output block
    int64_t total;      // blocks * ksteps
    int64_t per;        // steps per CTA
    int max_segs;       // partial tiles per CTA
    int sa;             // A ring depth (the MN-major staging ring for Y = A X)
    int sb;             // small-operand ring depth
    int sk;             // K-major A ring depth (Y = A X only)
    int npa;            // A producer warps (sa is a multiple of npa)
    int b_bytes;        // npad * 128
    uint32_t tmem_cols;
    float* part;        // [grid][max_segs][npad][128]
    double* norm_parts; // per-CTA sums of squares of the A tiles (NORM kernels)
    int* status;
};

constexpr int MAX_SA = 16, MAX_SK = 4;

// Ring structure.  Stage g (the g-th K step of this CTA's share) puts its A
// tile in A-ring slot g % sa and its slice of the small operand in B-ring
// slot g % sb; both copies complete on a_full[g % sa], so the MMA thread
// waits once per stage.  The copies of stage g are issued by producer warp
// g % npa, which owns the A slots congruent to it: one issuing thread
// sustains only about a third of the HBM bandwidth of an SM, several in
// parallel reach it.  A B slot is reused once the MMAs of stage g - sb have
// completed (sb <= sa, and sb <= sk for Y = A X, so a phase waited on
// cannot be overtaken).  For Y = A X the A tile arrives MN-major; four
// transposer warps rewrite it into a K-major ring of sk slots and release
// the staging slot at once, so staging slots recycle without waiting for
// the MMA.  The MMA thread (one thread issues every MMA of the CTA, so its
// loop carries no divisions and one commit per stage) releases the stage
// through a_empty (Y = A^T X) or k_empty (Y = A X).
//
// Parity waits on a ring of depth D are exact only while the waiter lags the
// barrier by less than D phases.  A producer checks the completion of stage
// g - sb after having checked that of stage g - npa - sb, so it never lags by
// a full ring: that needs npa <= sa for A^T X (a_empty, depth sa) and
// npa <= sb = sk for A X (k_empty, depth sk).
//
// NORM (TF32 only): the kernel also sums the squares of every entry of A it
// stages (each entry once over the grid: the stream-K shares partition the
// iteration space), for ||A||_F^2 of Alg. adaptivewithoutupdating step 1
// fused into the first pass.  For Y = A X the transposer threads add the
// entries they move; for Y = A^T X four more warps (10-13) read each A stage
// and release it together with the MMA commit.
template <bool XPOSE, int KIND, bool NORM = false>
__global__ void __launch_bounds__((XPOSE || NORM) ? TC_THREADS_X : TC_THREADS, 1)
k_tc_pass(const __grid_constant__ CUtensorMap mapA, const unsigned char* __restrict__ Bt,
          const TcParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[MAX_SA];
    __shared__ __align__(8) uint64_t a_empty[MAX_SA];
    __shared__ __align__(8) uint64_t k_full[MAX_SK];       // transposed tile ready (XPOSE)
    __shared__ __align__(8) uint64_t k_empty[MAX_SK];
    __shared__ __align__(8) uint64_t acc_full;
    __shared__ __align__(8) uint64_t acc_empty;
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;

    constexpr int E = Kind<KIND>::E;
    constexpr int BKE = 128 / E;                  // K elements per stage
    constexpr int MB = 128 / E;                   // M elements per staging box (A X)
    // warps: 0..npa-1 producers, 4-7 epilogue (TMEM lane quarter = warp % 4),
    // 8 MMA, 10-13 transposer (Y = A X)
    constexpr int EPI_WARP = 4, MMA_WARP = 8, XP_WARP = 10;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    SqSum32 nsq;                                  // NORM: this thread's share of ||A||^2
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // [A ring: sa x 16 KB][K-major ring: sk x 16 KB][B ring: sb x b_bytes]
    unsigned char* a_ring = smem;
    unsigned char* k_ring = a_ring + P.sa * A_TILE;
    unsigned char* b_ring = k_ring + P.sk * A_TILE;

    const int64_t s0 = int64_t(blockIdx.x) * P.per;
    const int64_t s1 = min(P.total, s0 + P.per);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int i = 0; i < P.sa; ++i) {
            mbar_init(&a_full[i], 1);
            // transposer warps, or the MMA commit (plus the norm warps)
            mbar_init(&a_empty[i], XPOSE ? 4 : (NORM ? 5 : 1));
        }
        for (int i = 0; i < P.sk; ++i) {
            mbar_init(&k_full[i], 4);                   // one arrival per transposer warp
            mbar_init(&k_empty[i], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 4);                       // one arrival per epilogue warp
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

    int issued = 0;          // one past the last stage this producer issued
    if (s0 < s1) {
        if (warp < P.npa) {
            // ------------------------------------------------------ producers
            if (lane == 0) {
                // stages warp, warp + npa, ...; slots and rounds kept incrementally
                const uint64_t pol_a = policy_evict_first(), pol_b = policy_evict_last();
                int g = warp, st = warp;
                uint32_t round = 0;
                int64_t blk = (s0 + warp) / P.ksteps;
                int kpos = int((s0 + warp) % P.ksteps);
                for (int64_t s = s0 + warp; s < s1; s += P.npa, g += P.npa) {
                    // the MMAs of stage g - sb have completed: B slot g % sb is free
                    // (and, for A^T X, A slot g % sa, since sb <= sa)
                    if (g >= P.sb) {
                        const int gp = g - P.sb;
                        const bool ok =
                            XPOSE ? mbar_wait(&k_empty[gp % P.sk], uint32_t(gp / P.sk) & 1u,
                                              &abort_flag)
                                  : mbar_wait(&a_empty[gp % P.sa], uint32_t(gp / P.sa) & 1u,
                                              &abort_flag);
                        if (!ok) {
                            abort_flag = 1;
                            break;
                        }
                    }
                    // A X: the transposer has released staging slot g % sa
                    if (XPOSE && round > 0 &&
                        !mbar_wait(&a_empty[st], (round - 1) & 1u, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const int kk = kpos * BKE;
                    unsigned char* dst = a_ring + st * A_TILE;
                    mbar_arrive_expect_tx(&a_full[st], uint32_t(A_TILE + P.b_bytes));
                    if (XPOSE) {
#pragma unroll
                        for (int q = 0; q < E; ++q)
                            tma_load_2d(dst + q * (128 * BKE), &mapA, &a_full[st],
                                        int(blk * BM + MB * q), kk, pol_a);
                    } else {
                        tma_load_2d(dst, &mapA, &a_full[st], kk, int(blk * BM), pol_a);
                    }
                    // the K step's slice of the small operand, pre-tiled as its
                    // shared-memory image
                    bulk_load(b_ring + (g % P.sb) * P.b_bytes, Bt + int64_t(kpos) * P.b_bytes,
                              uint32_t(P.b_bytes), &a_full[st], pol_b);
                    issued = g + 1;
                    st += P.npa;
                    if (st >= P.sa) { st -= P.sa; ++round; }
                    kpos += P.npa;
                    while (kpos >= P.ksteps) { kpos -= P.ksteps; ++blk; }
                }
            }
        } else if (warp == MMA_WARP) {
            // ------------------------------------------------------- MMA
            if (lane == 0) {
                const uint32_t idesc = idesc_make(Kind<KIND>::fmt, BM, P.nchunk);
                const int ra = XPOSE ? P.sk : P.sa;
                const int nch = P.npad > P.nchunk ? 2 : 1;
                const uint64_t chunk_off = uint64_t(P.nchunk * 128 / 16);
                int slot_a = 0, slot_b = 0, seg = 0;
                uint32_t ph_a = 0;
                int kpos = int(s0 % P.ksteps);
                for (int64_t s = s0; s < s1; ++s) {
                    const bool seg_first = (s == s0) || (kpos == 0);
                    const bool seg_last = (s + 1 == s1) || (kpos + 1 == P.ksteps);
                    if (seg_first && seg > 0) {
                        if (!mbar_wait(&acc_empty, (seg - 1) & 1u, &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                    }
                    if (!mbar_wait(XPOSE ? &k_full[slot_a] : &a_full[slot_a], ph_a, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of the stage's first K slice; the next 32-byte slices
                    // and the second column chunk only move the start address field
                    // (16-byte units), which stays below 2^14 in shared memory
                    const uint64_t ad0 =
                        smem_desc(smem_u32((XPOSE ? k_ring : a_ring) + slot_a * A_TILE), 16, 1024);
                    const uint64_t bd0 = smem_desc(smem_u32(b_ring + slot_b * P.b_bytes), 16, 1024);
                    const uint32_t acc0 = seg_first ? 0u : 1u;
#pragma unroll
                    for (int sub = 0; sub < 4; ++sub) {
                        umma<KIND>(tmem, ad0 + uint64_t(2 * sub), bd0 + uint64_t(2 * sub), idesc,
                                   sub == 0 ? acc0 : 1u);
                        if (nch == 2)
                            umma<KIND>(tmem + uint32_t(P.nchunk), ad0 + uint64_t(2 * sub),
                                       bd0 + uint64_t(2 * sub) + chunk_off, idesc,
                                       sub == 0 ? acc0 : 1u);
                    }
                    tc_commit(XPOSE ? &k_empty[slot_a] : &a_empty[slot_a]);
                    if (seg_last) {
                        tc_commit(&acc_full);
                        ++seg;
                    }
                    if (++slot_a == ra) { slot_a = 0; ph_a ^= 1u; }
                    if (++slot_b == P.sb) slot_b = 0;
                    if (++kpos == P.ksteps) kpos = 0;
                }
            }
        } else if (XPOSE && warp >= XP_WARP && warp < XP_WARP + 4) {
            // ------------------------------------------------ transposer
            // thread t owns row m = t of the 128-row tile; staging box q = m / MB
            // holds A(MB q.., k) as BKE K-rows of 128 bytes (128-byte swizzle);
            // the K-major tile holds row m as 128 bytes, 16-byte chunk c of
            // K = c T .. c T + T - 1 (T = 16 / E elements) at chunk c ^ (m % 8).
            constexpr int T = 16 / E;
            const int m = threadIdx.x - 32 * XP_WARP;
            const int q = m / MB, mm = m % MB;
            int sa_ = 0, sk_ = 0, kround = 0;
            uint32_t ph_a = 0;
            for (int64_t it = 0; it < s1 - s0; ++it) {
                if (!mbar_wait(&a_full[sa_], ph_a, &abort_flag) ||
                    (kround > 0 &&
                     !mbar_wait(&k_empty[sk_], uint32_t(kround - 1) & 1u, &abort_flag))) {
                    abort_flag = 1;
                    break;
                }
                unsigned char* kt = k_ring + sk_ * A_TILE;
                const unsigned char* raw = a_ring + sa_ * A_TILE + q * (128 * BKE);
                const int src_in_chunk = (mm % T) * E;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int e = 0; e < T; ++e) {
                        const int kr = c * T + e;
                        const unsigned char* src =
                            raw + kr * 128 + (((mm / T) ^ (kr & 7)) << 4) + src_in_chunk;
                        uint32_t v;
                        if constexpr (E == 4) v = *reinterpret_cast<const uint32_t*>(src);
                        else if constexpr (E == 2) v = *reinterpret_cast<const uint16_t*>(src);
                        else v = *src;
                        if constexpr (NORM && E == 4) nsq.add(__uint_as_float(v));
                        w[(e * E) >> 2] |= v << (((e * E) & 3) * 8);
                    }
                    *reinterpret_cast<uint4*>(kt + m * 128 + ((c ^ (m & 7)) << 4)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&k_full[sk_]);
                    mbar_arrive(&a_empty[sa_]);     // the staging slot may be refilled
                }
                if (++sa_ == P.sa) { sa_ = 0; ph_a ^= 1u; }
                if (++sk_ == P.sk) { sk_ = 0; ++kround; }
            }
        } else if (NORM && !XPOSE && warp >= XP_WARP && warp < XP_WARP + 4) {
            // ----------------------------------------- norm readers (A^T X)
            // thread tn reads 16-byte words tn, tn + 128, ... of each A stage
            const int tn = threadIdx.x - 32 * XP_WARP;
            int sa_ = 0;
            uint32_t ph_a = 0;
            for (int64_t it = 0; it < s1 - s0; ++it) {
                if (!mbar_wait(&a_full[sa_], ph_a, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                const uint4* tile = reinterpret_cast<const uint4*>(a_ring + sa_ * A_TILE);
#pragma unroll
                for (int q = 0; q < A_TILE / 16 / 128; ++q) {
                    const uint4 v = tile[tn + 128 * q];
                    nsq.add(__uint_as_float(v.x));
                    nsq.add(__uint_as_float(v.y));
                    nsq.add(__uint_as_float(v.z));
                    nsq.add(__uint_as_float(v.w));
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_empty[sa_]);   // with the MMA commit
                if (++sa_ == P.sa) { sa_ = 0; ph_a ^= 1u; }
            }
        } else if (warp >= EPI_WARP && warp < EPI_WARP + 4) {
            // -------------------------------------------------- epilogue
            const int quarter = warp & 3;                 // TMEM lanes 32*quarter..
            const int row = quarter * 32 + lane;
            int seg = 0;
            for (int64_t s = s0; s < s1;) {
                const int64_t blk = s / P.ksteps;
                const int64_t next = min(s1, (blk + 1) * int64_t(P.ksteps));
                if (!mbar_wait(&acc_full, uint32_t(seg) & 1u, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                float* dst = P.part + (int64_t(blockIdx.x) * P.max_segs + seg) *
                                          int64_t(P.npad) * BM;
                for (int c0 = 0; c0 < P.npad; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c0), r);
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
    if constexpr (NORM) {
        const double tot = cta_sum(nsq.value());     // threads without entries add 0
        if (threadIdx.x == 0) P.norm_parts[blockIdx.x] = tot;
    }
    __syncthreads();
    if (abort_flag) {
        if (threadIdx.x == 0) atomicCAS(P.status, DEV_OK, DEV_TIMEOUT);
        // let the copies already issued land before shared memory goes away:
        // both copies of a stage complete on its a_full phase
        if (warp < P.npa && lane == 0) {
            // this warp's stages among the last sa issued: g = issued-1, issued-1-npa, ...
            for (int g = issued - 1; g >= 0 && g > issued - 1 - P.sa; g -= P.npa)
                mbar_wait_drain(&a_full[g % P.sa], uint32_t(g / P.sa) & 1u);
        }
        if (warp == MMA_WARP && lane == 0) {
            // wait for every MMA this thread issued before TMEM is freed
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

// Y(i, j) = sum over the CTAs whose share touches block i/128 of their partial
// tile, in CTA order, in FP64 (many row blocks, few contributors each).  CTA
// (blk, g): rows blk*128 + threadIdx.x,
// columns g*RJT .. g*RJT + RJT - 1.  The segment index of CTA c in block blk
// is blk - floor(c per / ksteps), stepped from one CTA to the next without
// divisions; the loads of Y (accum) are issued before any store.
template <int RJT>
__global__ void __launch_bounds__(BM) k_tc_reduce_wide(const float* __restrict__ part, int64_t M,
                                                  int l, int npad, int ksteps, int64_t total,
                                                  int64_t per, int max_segs, int grid,
                                                  double* __restrict__ Y, int64_t ldy,
                                                  const float* __restrict__ rowblk_scale,
                                                  const float* __restrict__ col_scale, int accum) {
    // one CTA per (128-row block, RJT columns), the column groups of a block
    // adjacent in launch order, so the CTAs that read the same partial tiles
    // run together
    const int ncg = (l + RJT - 1) / RJT;
    const int64_t blk = blockIdx.x / ncg;
    const int r = threadIdx.x;
    const int64_t i = blk * BM + r;
    // the contributing CTAs of this row block, found once per CTA (64-bit
    // divisions are long instruction sequences)
    __shared__ int64_t sh[6];
    if (r == 0) {
        const int64_t first = blk * ksteps, last = min(total, first + ksteps) - 1;
        const int64_t lo = first / per;
        int64_t hi = last / per;
        if (hi >= grid) hi = grid - 1;
        sh[0] = lo;
        sh[1] = hi;
        sh[2] = per / ksteps;
        sh[3] = per % ksteps;
        sh[4] = (lo * per) / ksteps;
        sh[5] = (lo * per) % ksteps;
    }
    __syncthreads();
    if (i >= M) return;
    const int j0 = int(blockIdx.x % ncg) * RJT;
    const int nj = min(RJT, l - j0);
    const int64_t c_lo = sh[0], c_hi = sh[1], pq = sh[2], pr = sh[3];
    int64_t cb = sh[4], rem = sh[5];
    // compensated FP32 sums (Sum2f): the FP64 sum of the FP32 tiles without
    // an FP64 conversion and addition per tile (GB300's FP64 pipe would bound
    // this kernel); integer-valued tiles (the exact slice products) still
    // add up exactly
    Sum2f acc[RJT];
#pragma unroll 4
    for (int64_t c = c_lo; c <= c_hi; ++c) {
        const float* src = part + ((c * max_segs + (blk - cb)) * npad + j0) * BM + r;
#pragma unroll
        for (int q = 0; q < RJT; ++q)
            if (q < nj) acc[q].add(src[int64_t(q) * BM]);
        cb += pq;
        rem += pr;
        if (rem >= ksteps) {
            rem -= ksteps;
            ++cb;
        }
    }
    double yv[RJT];
#pragma unroll
    for (int q = 0; q < RJT; ++q)
        yv[q] = (accum && q < nj) ? Y[i + int64_t(j0 + q) * ldy] : 0.0;
    const double rs = rowblk_scale ? double(rowblk_scale[blk]) : 1.0;
#pragma unroll
    for (int q = 0; q < RJT; ++q) {
        if (q < nj) {
            double a = acc[q].value();
            if (rowblk_scale) a *= rs;
            if (col_scale) a *= double(col_scale[j0 + q]);
            Y[i + int64_t(j0 + q) * ldy] = accum ? yv[q] + a : a;
        }
    }
}

// Y(i, j) = sum over the CTAs whose share touches block i/128 of their partial
// tile, in CTA order, in FP64 (few row blocks, many contributors each: the
// Gram matrices, the single-pass sweep).  CTA (blk, g): rows blk*128 + (threadIdx.x %
// 128) of columns RRC RL g .. RRC RL (g + 1) - 1, RRC columns at a time (one
// output per thread), the contributing CTAs of block blk found once per CTA
// (64-bit divisions are long instruction sequences).  The segment index of
// CTA c in block blk is blk - floor(c per / ksteps), stepped from one CTA to
// the next without divisions.  The partial tiles of U contributors are
// loaded for all RL columns before any of them is added (the adds stay in
// CTA order), and Y (accum) before them.
constexpr int RRC = 2;      // columns at a time (BM threads each)

template <int RL, int U>
__global__ void __launch_bounds__(BM * RRC) k_tc_reduce(const float* __restrict__ part, int64_t M,
                                                        int l, int npad, int ksteps, int64_t total,
                                                        int64_t per, int max_segs, int grid,
                                                        double* __restrict__ Y, int64_t ldy,
                                                        const float* __restrict__ rowblk_scale,
                                                        const float* __restrict__ col_scale,
                                                        int accum) {
    // the column groups of a block adjacent in launch order, so the CTAs that
    // read the same partial tiles run together
    const int ncg = (l + RRC * RL - 1) / (RRC * RL);
    const int64_t blk = blockIdx.x / ncg;
    const int r = threadIdx.x % BM;
    const int jb = int(blockIdx.x % ncg) * RRC * RL + threadIdx.x / BM;
    const int64_t i = blk * BM + r;
    __shared__ int64_t sh[4];
    __shared__ int shi[3];
    if (threadIdx.x == 0) {
        const int64_t first = blk * ksteps, last = min(total, first + ksteps) - 1;
        const int64_t lo = first / per;
        int64_t hi = last / per;
        if (hi >= grid) hi = grid - 1;
        const int64_t cb0 = (lo * per) / ksteps;
        sh[0] = (lo * max_segs + (blk - cb0)) * npad * BM;   // tile of the first contributor
        sh[1] = int64_t(max_segs) * npad * BM;              // next CTA, same segment index
        sh[2] = int64_t(npad) * BM;                         // one segment
        sh[3] = hi - lo + 1;                                // contributors
        shi[0] = int((lo * per) % ksteps);
        shi[1] = int(per % ksteps);
        shi[2] = int(per / ksteps);
    }
    __syncthreads();
    if (i >= M) return;
    const int64_t base = sh[0], cstep = sh[1], sstep = sh[2];
    const int ncon = int(sh[3]);
    const int rem0 = shi[0], pr = shi[1], pq = shi[2];
    const double rs = rowblk_scale ? double(rowblk_scale[blk]) : 1.0;
    // the contributors' tile offsets do not depend on the column: U of them
    // at a time, then the RL columns' loads all issued before any add
    double yv[RL];
#pragma unroll
    for (int st = 0; st < RL; ++st) {
        const int j = jb + st * RRC;
        yv[st] = (accum && j < l) ? Y[i + int64_t(j) * ldy] : 0.0;
    }
    // compensated FP32 sums (Sum2f): the FP64 sum of the FP32 tiles without
    // an FP64 conversion and addition per tile (GB300's FP64 pipe would bound
    // this kernel); integer-valued tiles (the exact slice products) still add
    // up exactly
    Sum2f acc[RL];
    int64_t off = base;
    int rk = rem0;
    for (int c0 = 0; c0 < ncon; c0 += U) {
        int64_t coff[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            coff[u] = off;
            if (c0 + u < ncon) {
                rk += pr;
                int adv = pq;
                if (rk >= ksteps) {
                    rk -= ksteps;
                    ++adv;
                }
                off += cstep - int64_t(adv) * sstep;
            }
        }
        float v[RL][U];
#pragma unroll
        for (int st = 0; st < RL; ++st) {
            const int j = jb + st * RRC;
            const float* pj = part + int64_t(j) * BM + r;
#pragma unroll
            for (int u = 0; u < U; ++u) v[st][u] = (j < l && c0 + u < ncon) ? pj[coff[u]] : 0.f;
        }
#pragma unroll
        for (int st = 0; st < RL; ++st)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c0 + u < ncon) acc[st].add(v[st][u]);
    }
#pragma unroll
    for (int st = 0; st < RL; ++st) {
        const int j = jb + st * RRC;
        if (j >= l) break;
        double a = acc[st].value();
        if (rowblk_scale) a *= rs;
        if (col_scale) a *= double(col_scale[j]);
        Y[i + int64_t(j) * ldy] = accum ? yv[st] + a : a;
    }
}

// Y(i, j) = sum over bands b of (sum over the CTAs whose share touches block
// i/128 of band b's partial tile), the bands added in order, in FP64: the
// reduction of several passes into one Y with one write.  The partial tiles
// hold integers (exact sums of slice products), so each band's sum over its
// CTAs is exact in any order.  CTA (blk, g): rows blk*128 + (threadIdx.x %
// 128) of columns RBC RBL g .. RBC RBL (g + 1) - 1, RBC columns at a time (one
// output per thread), the CTA's setup (every band's contributors of block
// blk) done once for all of them.  Per output the first RBU partial tiles of
// RBG bands are loaded before any is added, so a thread keeps up to RBG x RBU
// loads in flight.
struct TcBands {
    TcPartials b[kMaxBands];
    int n;
};

constexpr int RBC = 2;      // columns at a time (BM threads each)
constexpr int RBL = 8;      // column steps per CTA
constexpr int RBG = 8;      // bands per group of loads
constexpr int RBU = 3;      // partial tiles per band loaded up front

__global__ void __launch_bounds__(BM * RBC) k_tc_reduce_bands(TcBands bands, int64_t M, int l,
                                                              double* __restrict__ Y, int64_t ldy) {
    const int ncg = (l + RBC * RBL - 1) / (RBC * RBL);   // column groups of a block adjacent
    const int64_t blk = blockIdx.x / ncg;
    const int r = threadIdx.x % BM;
    const int jb = int(blockIdx.x % ncg) * RBC * RBL + threadIdx.x / BM;
    const int64_t i = blk * BM + r;
    // per band: the float offset of the first contributing CTA's tile of
    // block blk and of its column 0, row 0; how many CTAs contribute; and the
    // offset steps between consecutive contributors (their first blocks
    // advance by per / ksteps or one more)
    __shared__ int64_t base[kMaxBands];
    __shared__ int ncon[kMaxBands];
    __shared__ int64_t cstep[kMaxBands][2];
    __shared__ int pinfo[kMaxBands][3];      // (lo per) % ksteps, per % ksteps, per / ksteps
    if (threadIdx.x < bands.n) {
        const TcPartials& B = bands.b[threadIdx.x];
        const int64_t first = blk * B.ksteps, last = min(B.total, first + B.ksteps) - 1;
        const int64_t lo = first / B.per;
        int64_t hi = last / B.per;
        if (hi >= B.grid) hi = B.grid - 1;
        const int64_t cb0 = (lo * B.per) / B.ksteps;
        base[threadIdx.x] = (lo * B.max_segs + (blk - cb0)) * B.npad * BM;
        ncon[threadIdx.x] = int(hi - lo + 1);
        cstep[threadIdx.x][0] = int64_t(B.max_segs) * B.npad * BM;   // next CTA, same segment
        cstep[threadIdx.x][1] = int64_t(B.npad) * BM;                // one segment
        pinfo[threadIdx.x][0] = int((lo * B.per) % B.ksteps);
        pinfo[threadIdx.x][1] = int(B.per % B.ksteps);
        pinfo[threadIdx.x][2] = int(B.per / B.ksteps);
    }
    __syncthreads();
    if (i >= M) return;
    const int nb = bands.n;
    // contributor w + 1 of a band is the next CTA: its stage range starts per
    // steps later, so its segment index for block blk is lower by the blocks
    // it starts later
    for (int step = 0; step < RBL; ++step) {
        const int j = jb + step * RBC;
        if (j >= l) break;
        const int64_t colo = int64_t(j) * BM + r;
        double tot = 0.0;
        for (int b0 = 0; b0 < nb; b0 += RBG) {
            float v[RBG][RBU];
#pragma unroll
            for (int u = 0; u < RBG; ++u) {
                const int bi = b0 + u;
#pragma unroll
                for (int w = 0; w < RBU; ++w) v[u][w] = 0.f;
                if (bi >= nb) continue;
                const float* part = bands.b[bi].part;
                const int ks = bands.b[bi].ksteps;
                int64_t off = base[bi] + colo;
                int rk = pinfo[bi][0];
#pragma unroll
                for (int w = 0; w < RBU; ++w) {
                    if (w >= ncon[bi]) break;
                    v[u][w] = part[off];
                    // the next contributor: CTA + 1, its segment of block blk
                    rk += pinfo[bi][1];
                    int adv = pinfo[bi][2];
                    if (rk >= ks) {
                        rk -= ks;
                        ++adv;
                    }
                    off += cstep[bi][0] - int64_t(adv) * cstep[bi][1];
                }
            }
#pragma unroll
            for (int u = 0; u < RBG; ++u) {
                const int bi = b0 + u;
                if (bi >= nb) break;
                Sum2f acc;                          // exact for the integer-valued tiles
#pragma unroll
                for (int w = 0; w < RBU; ++w) acc.add(v[u][w]);
                if (ncon[bi] > RBU) {
                    // contributors beyond the first RBU (a share shorter than
                    // a third of a block's K steps)
                    const float* part = bands.b[bi].part;
                    const int ks = bands.b[bi].ksteps;
                    int64_t off = base[bi] + colo;
                    int rk = pinfo[bi][0];
                    for (int w = 0; w < ncon[bi]; ++w) {
                        if (w >= RBU) acc.add(part[off]);
                        rk += pinfo[bi][1];
                        int adv = pinfo[bi][2];
                        if (rk >= ks) {
                            rk -= ks;
                            ++adv;
                        }
                        off += cstep[bi][0] - int64_t(adv) * cstep[bi][1];
                    }
                }
                tot = bi == 0 ? acc.value() : tot + acc.value();
            }
        }
        Y[i + int64_t(j) * ldy] = tot;
    }
}

// Small operand X (FP64, K x cols, ldx) -> operand type, written as the
// shared-memory image of each K step: step t holds rows j < npad of 128 bytes
// (K = t BKE .. t BKE + BKE - 1), 16-byte chunk c of row j stored at chunk
// c ^ (j % 8) (the 128-byte swizzle), so one bulk copy moves a whole step.
// Entries beyond cols or K are zero.  TF32: rounded to nearest (ties away),
// as FP32 bits; BF16: rounded to nearest even; FP8-E4M3: X(k, j) *
// fold[k / 128] / col_scale[j], saturated.
template <int KIND>
__global__ void k_to_operand(int64_t K, int cols, int npad, int ksteps, const double* __restrict__ X,
                             int64_t ldx, const float* __restrict__ fold,
                             const float* __restrict__ col_scale, unsigned char* __restrict__ out) {
    constexpr int E = Kind<KIND>::E;
    constexpr int BKE = 128 / E;
    constexpr int T = 16 / E;
    // CTA row blockIdx.y = operand row j; x strides over the reduction index k
    const int j = blockIdx.y;
    const int64_t kall = int64_t(ksteps) * BKE;
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < kall;
         k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = k / BKE;
        const int kk = int(k % BKE);
        unsigned char* dst = out + t * int64_t(npad) * 128 + j * 128 +
                             (((kk / T) ^ (j & 7)) << 4) + (kk % T) * E;
        const bool live = j < cols && k < K;
        const double x = live ? X[k + int64_t(j) * ldx] : 0.0;
        if constexpr (KIND == KIND_TF32) {
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(float(x)));
            *reinterpret_cast<uint32_t*>(dst) = u;
        } else if constexpr (KIND == KIND_BF16) {
            *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(float(x));
        } else {
            float v = 0.f;
            if (live) v = float(x * double(fold[k / 128]) / double(col_scale[j]));
            *reinterpret_cast<__nv_fp8_storage_t*>(dst) =
                __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// col_scale[j] = max_k |X(k, j) fold[k/128]| / 448 (1 when the column is zero).
__global__ void k_fp8_colscale(int64_t K, int cols, const double* __restrict__ X, int64_t ldx,
                               const float* __restrict__ fold, float* __restrict__ col_scale) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < K; i += 256)
        mx = fmax(mx, fabs(X[i + int64_t(j) * ldx] * double(fold[i / 128])));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s2]);
        __syncthreads();
    }
    if (threadIdx.x == 0) col_scale[j] = red[0] > 0.0 ? float(red[0] / 448.0) : 1.f;
}

// FP32 A -> BF16 copy (column-major, ld ldq), round to nearest even.
// norm_parts (nullable): the CTA's sum of squares of the entries it reads
// (the quantisation reads every entry once: ||A||_F^2 comes with it).
__global__ void k_quant_bf16(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                             __nv_bfloat16* __restrict__ Aq, int64_t ldq,
                             double* __restrict__ norm_parts) {
    SqSum32 nsq;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y)
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
             i += int64_t(gridDim.x) * blockDim.x) {
            const float a = A[i + j * lda];
            if (norm_parts) nsq.add(a);
            Aq[i + j * ldq] = __float2bfloat16_rn(a);
        }
    if (norm_parts) {
        const double tot = cta_sum(nsq.value());
        if (threadIdx.x == 0) norm_parts[blockIdx.x + int64_t(gridDim.x) * blockIdx.y] = tot;
    }
}

// amax of every 128 x 128 tile of A (tile (rb, cb) at amax[rb + cb * RB]).
__global__ void k_tile_amax(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                            int RB, float* __restrict__ amax) {
    __shared__ float red[256];
    const int64_t rb = blockIdx.x, cb = blockIdx.y;
    float mx = 0.f;
    for (int e = threadIdx.x; e < 128 * 128; e += 256) {
        const int64_t i = rb * 128 + (e & 127), j = cb * 128 + (e >> 7);
        if (i < m && j < n) mx = fmaxf(mx, fabsf(A[i + j * lda]));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s2]);
        __syncthreads();
    }
    if (threadIdx.x == 0) amax[rb + cb * RB] = red[0];
}

// Rank-1 tile scales: s_r[rb] = max_cb amax, s_c[cb] = max_rb amax / s_r[rb] / 448,
// so |A(i, j)| / (s_r[rb] s_c[cb]) <= 448 in every tile.
__global__ void k_tile_scales(const float* __restrict__ amax, int RB, int CB,
                              float* __restrict__ s_r, float* __restrict__ s_c) {
    for (int rb = threadIdx.x; rb < RB; rb += blockDim.x) {
        float mx = 0.f;
        for (int cb = 0; cb < CB; ++cb) mx = fmaxf(mx, amax[rb + cb * RB]);
        s_r[rb] = mx > 0.f ? mx : 1.f;
    }
    __syncthreads();
    for (int cb = threadIdx.x; cb < CB; cb += blockDim.x) {
        float mx = 0.f;
        for (int rb = 0; rb < RB; ++rb) mx = fmaxf(mx, amax[rb + cb * RB] / s_r[rb]);
        s_c[cb] = mx > 0.f ? mx / 448.f : 1.f;
    }
}

// FP32 A -> FP8-E4M3 copy A(i, j) / (s_r[i/128] s_c[j/128]), saturated.
// norm_parts (nullable): as in k_quant_bf16.
__global__ void k_quant_fp8(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                            const float* __restrict__ s_r, const float* __restrict__ s_c,
                            __nv_fp8_storage_t* __restrict__ Aq, int64_t ldq,
                            double* __restrict__ norm_parts) {
    SqSum32 nsq;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const float cs = s_c[j / 128];
        for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
             i += int64_t(gridDim.x) * blockDim.x) {
            const float a = A[i + j * lda];
            if (norm_parts) nsq.add(a);
            Aq[i + j * ldq] = __nv_cvt_float_to_fp8(a / (s_r[i / 128] * cs), __NV_SATFINITE,
                                                    __NV_E4M3);
        }
    }
    if (norm_parts) {
        const double tot = cta_sum(nsq.value());
        if (threadIdx.x == 0) norm_parts[blockIdx.x + int64_t(gridDim.x) * blockIdx.y] = tot;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t dim0,
                 uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {dim0, dim1};
    cuuint64_t strides[1] = {stride1_bytes};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct TcPlan {
    int npad, nchunk, ksteps, sa, sb, sk, npa, max_segs, grid;
    bool ok;
    int64_t blocks, total, per;
    uint32_t tmem_cols;
    size_t smem;
    int64_t ldx32;
};

TcPlan plan_tc(int64_t M, int64_t K, int cols, int num_sms, bool xpose, int E = 4) {
    TcPlan p{};
    p.npad = cols <= 256 ? (cols + 15) / 16 * 16 : (cols + 31) / 32 * 32;
    p.nchunk = p.npad <= 256 ? p.npad : p.npad / 2;
    const int bke = 128 / E;
    p.ksteps = int((K + bke - 1) / bke);
    p.blocks = (M + BM - 1) / BM;
    p.total = p.blocks * p.ksteps;
    p.grid = num_sms;
    if (p.grid > p.total) p.grid = int(p.total);
    p.per = (p.total + p.grid - 1) / p.grid;
    p.grid = int((p.total + p.per - 1) / p.per);
    p.max_segs = int((p.per + p.ksteps - 1) / p.ksteps) + 1;
    // ring depths within ~224 KB of dynamic shared memory: three small-operand
    // slots when they fit in 112 KB (two otherwise), as many K-major slots for
    // Y = A X, and every remaining 16 KB slot for A
    const int b_bytes = p.npad * 128;
    const int budget = 224 * 1024 - 1024;
    p.sb = 3 * b_bytes <= 112 * 1024 ? 3 : 2;
    p.sk = xpose ? p.sb : 0;                          // sb <= sk (see the kernel)
    int sa = (budget - p.sb * b_bytes - p.sk * A_TILE) / A_TILE;
    if (sa > MAX_SA) sa = MAX_SA;
    // producers: four with at least eight slots, three with six or seven, else
    // one per slot up to four; every slot belongs to exactly one producer
    if (sa >= 2 * NPA_MAX) p.npa = NPA_MAX;
    else if (sa >= 6) p.npa = 3;
    else p.npa = sa < NPA_MAX ? sa : NPA_MAX;
    if (xpose && p.npa > p.sb) p.npa = p.sb;          // producers never lag a full k_empty ring
    if (p.npa > 0) sa = sa / p.npa * p.npa;
    p.sa = sa;
    p.ok = p.sa >= 2 && p.npa >= 1 && (xpose || p.sa >= p.sb);
    p.smem = size_t(p.sa + p.sk) * A_TILE + size_t(p.sb) * b_bytes + 1024;
    uint32_t tc = 32;
    while (tc < uint32_t(p.npad)) tc <<= 1;
    p.tmem_cols = tc;
    p.ldx32 = (K + 15) / 16 * 16;                 // 16-byte strides for every element size
    return p;
}

}  // namespace

bool tc_make_map_2d(CUtensorMap* map, int dtype_code, const void* base, uint64_t dim0,
                    uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1) {
    const CUtensorMapDataType dt = dtype_code == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype_code == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    return make_map_2d(map, dt, base, dim0, dim1, stride1_bytes, box0, box1);
}

namespace {

// The reduction of a pass's partial tiles: eight columns per thread when the
// blocks are many (few contributors each), else one column per thread with
// sixteen contributors' tiles in flight (many contributors each).
cudaError_t tc_reduce_launch(const float* part, int64_t M, int cols, const TcPlan& p, double* Y,
                             int64_t ldy, const float* rowblk, const float* colsc, int accum,
                             int num_sms, cudaStream_t s) {
    const int64_t nblk = (M + BM - 1) / BM;
    const bool wide = nblk * ((cols + 7) / 8) >= 2 * int64_t(num_sms);
    count_launch();
    if (!wide) {
        k_tc_reduce<1, 16><<<unsigned(nblk * ((cols + RRC - 1) / RRC)), BM * RRC, 0, s>>>(
            part, M, cols, p.npad, p.ksteps, p.total, p.per, p.max_segs, p.grid, Y, ldy, rowblk,
            colsc, accum);
        return cudaGetLastError();
    }
    k_tc_reduce_wide<8><<<unsigned(nblk * ((cols + 7) / 8)), BM, 0, s>>>(
        part, M, cols, p.npad, p.ksteps, p.total, p.per, p.max_segs, p.grid, Y, ldy, rowblk,
        colsc, accum);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_reduce(const TcPartials& P, int64_t M, int cols, double* Y, int64_t ldy,
                             int accum, int num_sms, cudaStream_t s) {
    TcPlan p{};
    p.npad = P.npad;
    p.ksteps = P.ksteps;
    p.total = P.total;
    p.per = P.per;
    p.max_segs = P.max_segs;
    p.grid = P.grid;
    return tc_reduce_launch(P.part, M, cols, p, Y, ldy, nullptr, nullptr, accum, num_sms, s);
}

bool tc_supported(int64_t M, int64_t K, int cols, const void* A, int64_t lda, int trans) {
    if (cols < 1 || cols > 512 || M < 1 || K < 1) return false;
    if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda % 4) != 0) return false;
    if (M > (int64_t(1) << 31) - 256 || K > (int64_t(1) << 31) - 256) return false;
    const TcPlan p = plan_tc(M, K, cols, 152, trans == 0, 4);
    return p.ok && get_encode() != nullptr;
}

size_t tc_scratch_bytes(int64_t M, int64_t K, int cols, int num_sms) {
    size_t part = 0;
    for (int E = 1; E <= 4; E *= 2) {                  // the largest over the element sizes
        const TcPlan p = plan_tc(M, K, cols, num_sms, false, E);
        const size_t b = size_t(p.grid) * p.max_segs * p.npad * BM * sizeof(float);
        if (b > part) part = b;
    }
    size_t bt = 0;
    for (int E = 1; E <= 4; E *= 2) {
        const TcPlan p = plan_tc(M, K, cols, num_sms, false, E);
        const size_t b = size_t(p.ksteps) * p.npad * 128;
        if (b > bt) bt = b;
    }
    const TcPlan p = plan_tc(M, K, cols, num_sms, false, 4);
    return part + 256 + bt + 256 + size_t(p.npad) * sizeof(float) + 256;
}

size_t tc_quant_bytes(int64_t m, int64_t n, int prec) {
    const int E = prec == PLU_BF16 ? 2 : 1;
    const int64_t ldq = (m + 15) / 16 * 16;
    const int64_t RB = (m + 127) / 128, CB = (n + 127) / 128;
    return size_t(ldq) * size_t(n) * E + 256 + size_t(RB * CB + RB + CB) * sizeof(float) + 768;
}

cudaError_t launch_tc_quantize(int prec, const float* A, int64_t m, int64_t n, int64_t lda,
                               void* qbuf, QuantA* out, int num_sms, cudaStream_t s,
                               const NormOut* norm) {
    const int E = prec == PLU_BF16 ? 2 : 1;
    const int64_t ldq = (m + 15) / 16 * 16;
    const int64_t RB = (m + 127) / 128, CB = (n + 127) / 128;
    Workspace w;
    w.base = static_cast<char*>(qbuf);
    w.cap = tc_quant_bytes(m, n, prec);
    void* Aq = w.take(size_t(ldq) * size_t(n) * E);
    float* amax = static_cast<float*>(w.take(size_t(RB * CB) * sizeof(float)));
    float* s_r = static_cast<float*>(w.take(size_t(RB) * sizeof(float)));
    float* s_c = static_cast<float*>(w.take(size_t(CB) * sizeof(float)));
    if (!Aq || !amax || !s_r || !s_c) return cudaErrorInvalidValue;
    unsigned gy = unsigned(n < 65535 ? n : 65535);
    unsigned gx = unsigned((m + 255) / 256 < 64 ? (m + 255) / 256 : 64);
    double* nparts = nullptr;
    if (norm) {
        // one partial per CTA: at most 8 x 152-ish CTAs
        if (gx > 8) gx = 8;
        if (gy > unsigned(num_sms)) gy = unsigned(num_sms);
        if (!norm->parts || !norm->out || int64_t(gx) * gy > norm->cap) return cudaErrorInvalidValue;
        nparts = norm->parts;
    }
    cudaError_t e;
    if (prec == PLU_BF16) {
        count_launch();
        k_quant_bf16<<<dim3(gx, gy), 256, 0, s>>>(A, m, n, lda, static_cast<__nv_bfloat16*>(Aq), ldq,
                                                  nparts);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        out->s_r = nullptr;
        out->s_c = nullptr;
    } else {
        count_launch();
        k_tile_amax<<<dim3(unsigned(RB), unsigned(CB)), 256, 0, s>>>(A, m, n, lda, int(RB), amax);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count_launch();
        k_tile_scales<<<1, 256, 0, s>>>(amax, int(RB), int(CB), s_r, s_c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count_launch();
        k_quant_fp8<<<dim3(gx, gy), 256, 0, s>>>(A, m, n, lda, s_r, s_c,
                                                 static_cast<__nv_fp8_storage_t*>(Aq), ldq, nparts);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        out->s_r = s_r;
        out->s_c = s_c;
    }
    if (norm && (e = launch_sum_partials(nparts, int(gx * gy), norm->out, s)) != cudaSuccess)
        return e;
    out->data = Aq;
    out->ld = ldq;
    out->prec = prec;
    out->m = m;
    out->n = n;
    return cudaSuccess;
}

namespace {

template <int KIND>
cudaError_t tc_pass_kind(int trans, int64_t m, int64_t n, const void* A, int64_t lda,
                         const float* s_r, const float* s_c, const double* X, int64_t ldx,
                         int cols, double* Y, int64_t ldy, void* scratch, size_t scratch_cap,
                         int* dev_status, int num_sms, cudaStream_t s, int accum,
                         const void* xq_pre = nullptr, TcPartials* keep = nullptr,
                         const NormOut* norm = nullptr) {
    constexpr int E = Kind<KIND>::E;
    constexpr int BKE = 128 / E;
    const int64_t M = trans ? n : m;
    const int64_t K = trans ? m : n;
    const TcPlan p = plan_tc(M, K, cols, num_sms, trans == 0, E);
    if (!p.ok) return cudaErrorInvalidValue;
    if (scratch_cap < tc_scratch_bytes(M, K, cols, num_sms)) return cudaErrorInvalidValue;
    Workspace w;
    w.base = static_cast<char*>(scratch);
    w.cap = scratch_cap;
    float* part = static_cast<float*>(w.take(size_t(p.grid) * p.max_segs * p.npad * BM * sizeof(float)));
    unsigned char* xq = static_cast<unsigned char*>(w.take(size_t(p.ksteps) * p.npad * 128));
    float* colsc = static_cast<float*>(w.take(size_t(p.npad) * sizeof(float)));
    if (!part || !xq || !colsc) return cudaErrorInvalidValue;
    // fold: scales of A along the reduction index (A X: s_c by column block of
    // A; A^T X: s_r by row block); rowblk: scales along the output rows
    const float* fold = trans ? s_r : s_c;
    const float* rowblk = trans ? s_c : s_r;
    cudaError_t e;
    if (xq_pre && KIND == KIND_FP8) return cudaErrorInvalidValue;   // FP8 folds scales into X
    if (!xq_pre) {
        int64_t b = (int64_t(p.ksteps) * BKE + 255) / 256;
        const int64_t bcap = (int64_t(num_sms) * 16 + p.npad - 1) / p.npad;
        if (b > bcap) b = bcap;
        if (KIND == KIND_FP8) {
            count_launch();
            k_fp8_colscale<<<cols, 256, 0, s>>>(K, cols, X, ldx, fold, colsc);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        count_launch();
        k_to_operand<KIND><<<dim3(unsigned(b), unsigned(p.npad)), 256, 0, s>>>(K, cols, p.npad, p.ksteps, X, ldx, fold,
                                                        colsc, xq);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const CUtensorMapDataType dt = KIND == KIND_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : KIND == KIND_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUtensorMap mapA;
    // A as stored: dim0 = rows (m, contiguous), dim1 = columns (n)
    if (!make_map_2d(&mapA, dt, A, uint64_t(m), uint64_t(n), uint64_t(lda) * E, BKE,
                     trans ? 128 : BKE))
        return cudaErrorInvalidValue;
    TcParams P;
    P.M = M;
    P.K = K;
    P.npad = p.npad;
    P.nchunk = p.nchunk;
    P.ksteps = p.ksteps;
    P.total = p.total;
    P.per = p.per;
    P.max_segs = p.max_segs;
    P.sa = p.sa;
    P.sb = p.sb;
    P.sk = p.sk;
    P.npa = p.npa;
    P.b_bytes = p.npad * 128;
    P.tmem_cols = p.tmem_cols;
    P.part = part;
    P.status = dev_status;
    P.norm_parts = nullptr;
    if (norm) {
        if (KIND != KIND_TF32 || !norm->parts || !norm->out || p.grid > norm->cap)
            return cudaErrorInvalidValue;
        P.norm_parts = norm->parts;
        const unsigned char* op = xq_pre ? static_cast<const unsigned char*>(xq_pre) : xq;
        if (trans) {
            e = cudaFuncSetAttribute(k_tc_pass<false, KIND, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(p.smem));
            if (e != cudaSuccess) return e;
            count_launch();
            k_tc_pass<false, KIND, true><<<p.grid, TC_THREADS_X, p.smem, s>>>(mapA, op, P);
        } else {
            e = cudaFuncSetAttribute(k_tc_pass<true, KIND, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(p.smem));
            if (e != cudaSuccess) return e;
            count_launch();
            k_tc_pass<true, KIND, true><<<p.grid, TC_THREADS_X, p.smem, s>>>(mapA, op, P);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_sum_partials(norm->parts, p.grid, norm->out, s)) != cudaSuccess) return e;
    } else if (trans) {
        e = cudaFuncSetAttribute(k_tc_pass<false, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(p.smem));
        if (e != cudaSuccess) return e;
        count_launch();
        k_tc_pass<false, KIND><<<p.grid, TC_THREADS, p.smem, s>>>(
            mapA, xq_pre ? static_cast<const unsigned char*>(xq_pre) : xq, P);
    } else {
        e = cudaFuncSetAttribute(k_tc_pass<true, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(p.smem));
        if (e != cudaSuccess) return e;
        count_launch();
        k_tc_pass<true, KIND><<<p.grid, TC_THREADS_X, p.smem, s>>>(
            mapA, xq_pre ? static_cast<const unsigned char*>(xq_pre) : xq, P);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (keep) {              // the caller reduces later (launch_tc_reduce_bands)
        keep->part = part;
        keep->npad = p.npad;
        keep->ksteps = p.ksteps;
        keep->max_segs = p.max_segs;
        keep->grid = p.grid;
        keep->total = p.total;
        keep->per = p.per;
        return cudaSuccess;
    }
    return tc_reduce_launch(part, M, cols, p, Y, ldy, rowblk, KIND == KIND_FP8 ? colsc : nullptr,
                            accum, num_sms, s);
}

}  // namespace

cudaError_t launch_tc_pass(int trans, int64_t m, int64_t n, const float* A, int64_t lda,
                           const double* X, int64_t ldx, int cols, double* Y, int64_t ldy,
                           void* scratch, size_t scratch_cap, int* dev_status, int num_sms,
                           cudaStream_t s, int accum, const void* xq_pre, const NormOut* norm) {
    return tc_pass_kind<KIND_TF32>(trans, m, n, A, lda, nullptr, nullptr, X, ldx, cols, Y, ldy,
                                   scratch, scratch_cap, dev_status, num_sms, s, accum, xq_pre,
                                   nullptr, norm);
}

int quant_norm_parts(int num_sms) { return num_sms * 8; }

cudaError_t launch_tc_reduce_bands(const TcPartials* bands, int nbands, int64_t M, int cols,
                                  double* Y, int64_t ldy, cudaStream_t s) {
    if (nbands < 1 || nbands > kMaxBands || M < 1 || cols < 1) return cudaErrorInvalidValue;
    TcBands tb;
    tb.n = nbands;
    for (int b = 0; b < nbands; ++b) tb.b[b] = bands[b];
    count_launch();
    k_tc_reduce_bands<<<unsigned((M + BM - 1) / BM * ((cols + RBC * RBL - 1) / (RBC * RBL))),
                        BM * RBC, 0, s>>>(tb, M, cols, Y, ldy);
    return cudaGetLastError();
}

size_t tc_operand_bytes(int64_t K, int cols) {
    const TcPlan p = plan_tc(BM, K, cols, 1, false, 4);
    return size_t(p.ksteps) * p.npad * 128;
}

cudaError_t launch_tc_operand(int64_t K, int cols, const double* X, int64_t ldx, void* out,
                              int num_sms, cudaStream_t s) {
    if (K < 1 || cols < 1 || cols > 512 || !X || !out) return cudaErrorInvalidValue;
    const TcPlan p = plan_tc(BM, K, cols, num_sms, false, 4);
    constexpr int BKE = 128 / Kind<KIND_TF32>::E;
    int64_t b = (int64_t(p.ksteps) * BKE + 255) / 256;
    const int64_t bcap = (int64_t(num_sms) * 16 + p.npad - 1) / p.npad;
    if (b > bcap) b = bcap;
    count_launch();
    k_to_operand<KIND_TF32><<<dim3(unsigned(b), unsigned(p.npad)), 256, 0, s>>>(
        K, cols, p.npad, p.ksteps, X, ldx, nullptr, nullptr, static_cast<unsigned char*>(out));
    return cudaGetLastError();
}

cudaError_t launch_tc_pass_q(int trans, const QuantA& q, const double* X, int64_t ldx, int cols,
                             double* Y, int64_t ldy, void* scratch, size_t scratch_cap,
                             int* dev_status, int num_sms, cudaStream_t s, int accum,
                             const void* xq_pre, TcPartials* keep) {
    if (q.prec == PLU_BF16)
        return tc_pass_kind<KIND_BF16>(trans, q.m, q.n, q.data, q.ld, nullptr, nullptr, X, ldx,
                                       cols, Y, ldy, scratch, scratch_cap, dev_status, num_sms, s,
                                       accum, xq_pre, keep);
    if (xq_pre || keep) return cudaErrorInvalidValue;
    return tc_pass_kind<KIND_FP8>(trans, q.m, q.n, q.data, q.ld, q.s_r, q.s_c, X, ldx, cols, Y,
                                  ldy, scratch, scratch_cap, dev_status, num_sms, s, accum);
}

}  // namespace plu
