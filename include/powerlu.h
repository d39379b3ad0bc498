/*
 * powerlu.h -- C ABI of a GB300 (sm_103a) implementation of the hot path of
 * PowerLU, the pass-efficient randomized LU of Zhang & Mascagni,
 * "Pass-Efficient Randomized LU Algorithms for Computing Low-Rank Matrix
 * Approximation" (arXiv 2002.07138).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major: entry (i, j) of an R x C matrix M with
 *    leading dimension ld >= max(R, 1) lives at M[i + j * ld].
 *  - Every matrix and index pointer is DEVICE memory owned by the caller,
 *    unless the argument says "host".  The library never frees or keeps a
 *    caller pointer beyond the call.
 *  - Work is enqueued on the context's CUDA stream.  Entry points that
 *    produce factors end with one stream synchronisation and return the
 *    device status of the call (PLU_ETIMEOUT, PLU_ENUMERIC, ...), unless
 *    plu_set_async(ctx, 1) was called; then they return after enqueueing
 *    and plu_check() reports the device status later.
 *  - Arguments are validated on the host before anything is launched; a
 *    violation returns PLU_EINVAL and launches nothing.
 *  - plu_last_error() describes the last non-PLU_OK status of a context.
 *  - A context is used by one host thread at a time.
 *
 * Index vectors are 0-based int32: p (length m) and q (length n) encode
 * P and Q by  (P A Q^T)(i, j) = A(p[i], q[j]).
 */
#ifndef POWERLU_H
#define POWERLU_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of the passes over A (Sec. 3.3 counts them; v passes).
 * PLU_FP64: FP64 FMA.  PLU_FP32: FP32 FMA, FP32 accumulation.
 * PLU_TF32, PLU_BF16, PLU_FP8_E4M3: tensor-core products with FP32
 * accumulation.  TF32 reads the FP32 A directly; BF16 and FP8 read a
 * quantised copy made once per call (FP8 with per-tile scales).
 * PLU_TF32X3: split-precision tensor-core products, FP32-accurate: A and the
 * small operand are each split into a TF32 head and a TF32 remainder and
 * three TF32 products (head x head, remainder x head, head x remainder) are
 * summed in FP32 (about 3x the tensor work of PLU_TF32, same HBM traffic).
 * In the TF32, BF16 and FP8 modes the products that enter the result to first
 * order run as PLU_TF32X3 on the FP32 A: the last pass Y = A V_k of PowerLU
 * and RandLU's pass B^T = A^T W.  The fixed-precision pass G = A V, whose
 * column norms decide the rank, runs with FP32 FMAs in every mode but FP64
 * (the tensor cores' accumulation shrinks sums by ~1e-6 relative even when
 * split, which would bias the rank indicator).  Everything between the passes
 * (LU, QR, rank, tail) is FP64 in every mode.  The tensor-core modes need A
 * stored in FP32. */
typedef enum {
    PLU_FP64 = 0,
    PLU_TF32 = 1,
    PLU_BF16 = 2,
    PLU_FP8_E4M3 = 3,
    PLU_FP32 = 4,
    PLU_TF32X3 = 5
} plu_prec;

/* Element type of A. */
typedef enum { PLU_F64 = 0, PLU_F32 = 1 } plu_dtype;

typedef enum {
    PLU_OK = 0,
    PLU_EINVAL = 1,        /* bad argument (host check, nothing launched)       */
    PLU_ENOMEM = 2,        /* workspace allocation failed                        */
    PLU_ECUDA = 3,         /* a CUDA runtime call failed                         */
    PLU_ENUMERIC = 4,      /* non-finite value or zero pivot in a final LU       */
    PLU_ETIMEOUT = 5,      /* a device-side wait ran out of its iteration budget */
    PLU_TOL_NOT_MET = 6,   /* fixed precision: l columns did not reach eps       */
    PLU_EUNSUPPORTED = 7,  /* combination not built (e.g. precision for dtype)   */
    PLU_EINDEX = 8         /* a sparse index or row pointer out of range (device) */
} plu_status;

/* Dense input matrix A (m x n), column-major, device memory, not owned. */
typedef struct {
    int64_t m, n, ld;
    int32_t dtype;          /* plu_dtype */
    const void* data;
} plu_matrix;

/* Sparse input matrix A (m x n) in compressed sparse rows, device memory,
 * not owned (the sparse experiment of Sec. 6 uses MATLAB sprand matrices).
 * Row i holds the nonzeros row_ptr[i] .. row_ptr[i+1]-1: column col_idx[t]
 * (0-based) and value val[t].  row_ptr has m + 1 entries, row_ptr[0] = 0,
 * row_ptr[m] = nnz, non-decreasing; column indices need not be sorted, and
 * each position (i, j) is stored at most once (plu_powerlu_fp_csr takes
 * ||A||_F^2 as the sum of val^2).  The passes read A^T through its own CSR (t_*: the
 * CSR of the n x m matrix A^T, i.e. the compressed columns of A), which must
 * hold the same entries.  A row pointer outside [0, nnz] or a column index
 * outside its range is detected on the device: the entry is skipped and the
 * call returns PLU_EINDEX. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t* row_ptr;     /* m + 1 */
    const int32_t* col_idx;     /* nnz, in [0, n) */
    const double* val;          /* nnz */
    const int64_t* t_row_ptr;   /* n + 1 */
    const int32_t* t_col_idx;   /* nnz, in [0, m) */
    const double* t_val;        /* nnz */
} plu_csr;

/* Phases of a call, for plu_report.ms_phase: the Gaussian sketch (and the
 * quantised copy of A in the BF16 / FP8 modes); the passes of the power
 * iteration (Alg. gpowerlu); the re-orthogonalising LUs between them; the
 * final QR; the last pass (Y = A V_k or G = A V); the rank determination
 * (||A||_F^2, column norms, rank scan, restart copies); the two getrf of the
 * tail; the tail's two m x k x k products. */
enum {
    PLU_PHASE_SKETCH = 0,
    PLU_PHASE_POWER_PASSES = 1,
    PLU_PHASE_REORTH = 2,
    PLU_PHASE_QR = 3,
    PLU_PHASE_LAST_PASS = 4,
    PLU_PHASE_RANK = 5,
    PLU_PHASE_TAIL_LU = 6,
    PLU_PHASE_TAIL_PRODUCTS = 7,
    PLU_NPHASES = 8
};

/* Per-call report (host struct, filled when a non-NULL pointer is given). */
typedef struct {
    double ms_total;        /* device time of the call (CUDA events)             */
    double ms_passes;       /* device time of the kernels that read A            */
    int32_t passes;         /* number of passes over A launched                  */
    int32_t rank;           /* k used for the factors                            */
    double indicator;       /* fixed precision: sqrt(max(E,0))/||A||_F, else -1  */
    double normA2;          /* fixed precision: ||A||_F^2, else -1               */
    int32_t info1, info2;   /* first zero pivot (1-based) of lu(Y), lu(B^T)      */
    double flops_passes;    /* algorithmic flops of the passes, 2 m n cols each   */
    double bytes_passes;    /* algorithmic bytes of the passes (A + operands)    */
    int32_t launches;       /* library kernels launched by the call              */
    int32_t rounds;         /* fixed precision: rounds of the rank determination */
    double ms_phase[PLU_NPHASES];  /* device time per phase (CUDA events between the
                                      phase boundaries; plu_powerlu, plu_powerlu_fp
                                      and their sparse forms; 0 elsewhere)        */
} plu_report;

typedef struct plu_ctx plu_ctx;

/* Create a context bound to `device` and the CUDA stream `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The context owns a
 * device workspace that grows on demand and is freed by plu_destroy. */
plu_status plu_create(plu_ctx** ctx, int device, void* cuda_stream);
void plu_destroy(plu_ctx* ctx);
const char* plu_last_error(const plu_ctx* ctx);
plu_status plu_set_stream(plu_ctx* ctx, void* cuda_stream);
/* async != 0: factor calls return after enqueueing (no synchronisation). */
plu_status plu_set_async(plu_ctx* ctx, int async);
/* Synchronise the stream and return (then clear) the device status. */
plu_status plu_check(plu_ctx* ctx);
/* Iteration budget of every device-side wait (grid barriers); <= 0 restores
 * the default (about a second).  A tiny budget makes the waits give up and
 * the call return PLU_ETIMEOUT, with the context still usable. */
plu_status plu_set_wait_budget(plu_ctx* ctx, int64_t spins);
/* How every panel LU of the context (the re-orthogonalising lu of
 * Alg. gpowerlu, the getrf steps of Alg. bpowerlu / powerlufp / rlu /
 * singlepasslu, plu_lu_reorth, plu_getrf) forms its trailing updates between
 * 32-column blocks: mode 0 with FP64 FMAs; mode 1 on the tensor cores, as
 * sums of exact FP16 digit products rounded once to FP64 (FP64-accurate: the
 * error stays below an FP64 dot product's rounding bound); mode -1 (the
 * default) mode 1 for the mixed-precision modes and the sparse path, mode 0
 * for the FP64 path.  The pivot rule (largest |x|, ties to the first row in
 * the current order) and the outputs are the same in both modes; shapes the
 * tensor-core kernels do not take (more than 2048 columns, or too many rows
 * per SM for shared memory) use mode 0.  PLU_EINVAL for another mode. */
plu_status plu_set_lu_updates(plu_ctx* ctx, int mode);

/* ---------------------------------------------------------------------
 * Steps of the hot path, one entry point each (Sec. 3, Alg. gpowerlu).
 * ------------------------------------------------------------------- */

/* a1. Gaussian test matrix Omega (Alg. bpowerlu step 1; Alg. gpowerlu):
 * out (rows x cols, ld) receives i.i.d. N(0,1) values, entry (i, j) being the
 * Box-Muller output number t = i + j*rows of the Philox4x32-10 stream
 * (key = seed, counter = (t/2, stream_id)), computed in correctly rounded
 * float32 steps (the values are float32 numbers, exact in the FP64 output).
 * The same (seed, stream_id, rows, cols) gives bit-identical values on every
 * call. */
plu_status plu_gaussian(plu_ctx* ctx, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t stream_id, double* out, int64_t ld);

/* a2/a4/a6. One pass over A (the products of Alg. gpowerlu and Alg.
 * bpowerlu step 3): Y = A X (trans = 0; X n x cols, Y m x cols) or
 * Y = A^T X (trans = 1; X m x cols, Y n x cols), in arithmetic `prec`.
 * X and Y are FP64 and must not overlap. */
plu_status plu_pass(plu_ctx* ctx, const plu_matrix* A, int trans, const double* X,
                    int64_t ldx, int cols, plu_prec prec, double* Y, int64_t ldy);

/* a2/a4/a6 on a sparse A: Y = A X (trans = 0; X n x cols, Y m x cols) or
 * Y = A^T X (trans = 1, through the CSR of A^T; X m x cols, Y n x cols),
 * FP64.  Each entry of Y sums the nonzeros of its row of S (A or A^T) in a
 * fixed order (alternate nonzeros, in CSR order, into two partial sums that
 * are then added), so the result does not depend on the launch.  X and Y
 * must not overlap.  PLU_EINDEX: see plu_csr. */
plu_status plu_spmm(plu_ctx* ctx, const plu_csr* A, int trans, const double* X, int64_t ldx,
                    int cols, double* Y, int64_t ldy);

/* a3. [X, ~] = lu(X) in place (Alg. gpowerlu, the LU re-orthogonalisation):
 * X (rows x cols, rows >= cols) is overwritten by the permuted unit lower
 * factor P^T L of the partial-pivoting LU P X = L U (ties: first row in the
 * LAPACK swap order).  U is discarded. */
plu_status plu_lu_reorth(plu_ctx* ctx, int64_t rows, int cols, double* X, int64_t ldx);

/* a3/a8. [L, U, P] = lu(X) (Alg. bpowerlu steps 4 and 6): X (rows x cols,
 * rows >= cols) is read; perm (rows) receives P as perm[i] = source row of
 * row i of P X; L (rows x cols, ldL) the unit lower trapezoidal factor in
 * pivoted order; U (cols x cols, ldU) the upper triangular factor.  X is
 * used as scratch and destroyed.  info (device int32, nullable) receives the
 * first zero-pivot column (1-based) or 0. */
plu_status plu_getrf(plu_ctx* ctx, int64_t rows, int cols, double* X, int64_t ldx,
                     int32_t* perm, double* L, int64_t ldL, double* U, int64_t ldU,
                     int32_t* info);

/* a5. [V, ~] = qr(X) (Alg. gpowerlu, last step): X (rows x cols) is
 * overwritten by Q with orthonormal columns, X = Q R, R_ii > 0.  R (cols x
 * cols, ldR) receives R when non-NULL.  FP64 CholeskyQR2. */
plu_status plu_qr(plu_ctx* ctx, int64_t rows, int cols, double* X, int64_t ldx,
                  double* R, int64_t ldR);

/* a5 as the mixed modes run it: one CholeskyQR round, X (rows x cols) <- X
 * R^{-1} with R^T R = X^T X (Alg. gpowerlu, last step; R, when non-NULL,
 * receives R, ldR >= cols).  tc != 0: the two FP64 products X^T X and
 * X R^{-1} run on the BF16 tensor cores as sums of exact products of 7-bit
 * slices of the operands (FP64-accurate; needs cols <= 512, else
 * PLU_EUNSUPPORTED); tc = 0: FP64 FMAs.  Orthogonality of one round degrades
 * with cond(X)^2; plu_qr runs two. */
plu_status plu_cholqr1(plu_ctx* ctx, int64_t rows, int cols, double* X, int64_t ldx,
                       double* R, int64_t ldR, int tc);

/* a7. Blocked rank determination (Alg. adaptivewithoutupdating; precise != 0
 * adds the per-column loop of Sec. 6.4): from G = A V (rows x cols) and
 * normA2 = ||A||_F^2 (host value), find the first block of b columns (or
 * column) with E <= eps^2 ||A||_F^2, E = ||A||_F^2 - sum ||G(:, j)||^2
 * (Thm. errorerror, FP64).  k_out and E_out are host pointers.  Returns
 * PLU_TOL_NOT_MET (k = cols) when the tolerance is not met. */
plu_status plu_rank(plu_ctx* ctx, int64_t rows, int cols, const double* G, int64_t ldg,
                    double normA2, double eps, int b, int precise, int* k_out,
                    double* E_out);

/* ||A||_F^2 in FP64 (Alg. adaptivewithoutupdating step 1); out is a host
 * pointer.  One pass over A. */
plu_status plu_norm2(plu_ctx* ctx, const plu_matrix* A, double* out);

/* ---------------------------------------------------------------------
 * Whole algorithms.
 * ------------------------------------------------------------------- */

/* Fixed rank (Def. lowrank): Alg. bpowerlu with steps 1-2 replaced by
 * Alg. gpowerlu.  1 <= k <= l < min(m, n), v >= 2.  Outputs: p (m), q (n),
 * L (m x k, ldL >= m), U (k x n, ldU >= k) with P A Q^T ~= L U.
 * Exactly v passes over A. */
plu_status plu_powerlu(plu_ctx* ctx, const plu_matrix* A, int k, int l, int v,
                       uint64_t seed, plu_prec prec, int32_t* p, int32_t* q,
                       double* L, int64_t ldL, double* U, int64_t ldU,
                       plu_report* rep);

/* Fixed precision: Alg. powerlufp on Alg. adaptivewithoutupdating
 * (precise != 0: the per-column refinement of Sec. 6.4).  0 < eps < 1,
 * 1 <= b <= l < min(m, n), v >= 2.  *k_out (host) receives the rank;
 * L must hold m x l (ldL >= m) and U l x n (ldU >= l); the first k columns
 * of L and rows of U are the factors.  Returns PLU_TOL_NOT_MET with k = l
 * and valid factors when l columns do not reach eps.  One stream
 * synchronisation to read k.  v + 1 passes over A (one for ||A||_F). */
plu_status plu_powerlu_fp(plu_ctx* ctx, const plu_matrix* A, double eps, int b, int l,
                          int v, int precise, uint64_t seed, plu_prec prec, int* k_out,
                          int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                          int64_t ldU, plu_report* rep);

/* Fixed precision with the restart of the Remark after Alg.
 * adaptivewithoutupdating: when the l columns of a round leave
 * E > eps^2 ||A||_F^2, the next round reruns Alg. adaptivewithoutupdating on
 * the remainder A - A W W^T (W: every basis column so far, applied as
 * A X - (A W)(W^T X)) with a fresh Gaussian matrix (the Philox streams of
 * round r are those of round 0 plus 16 r), the indicator E carrying over; at
 * most max_rounds rounds (max_rounds * l <= 2048 and < min(m, n)).  The rank k
 * is the number of columns consumed over all rounds; Alg. powerlufp's tail
 * runs on the union of the rounds' bases.  L must hold m x (l max_rounds)
 * (ldL >= m) and U (l max_rounds) x n (ldU >= l max_rounds).  Returns
 * PLU_TOL_NOT_MET with valid factors of rank l max_rounds when eps is not
 * reached.  rep->rounds receives the rounds used.  One stream synchronisation
 * per round; v passes over A per round plus one for ||A||_F.  The paper's
 * interface is this one with max_rounds = 1 (plu_powerlu_fp). */
plu_status plu_powerlu_fp_restart(plu_ctx* ctx, const plu_matrix* A, double eps, int b, int l,
                                  int v, int precise, int max_rounds, uint64_t seed,
                                  plu_prec prec, int* k_out, int32_t* p, int32_t* q, double* L,
                                  int64_t ldL, double* U, int64_t ldU, plu_report* rep);

/* Single pass (Alg. singlepasslu, Sec. 5): Omega m x k, G = A^T Omega and
 * H = A G from one read of A, then two LUs.  1 <= k < min(m, n).
 * Outputs as plu_powerlu. */
plu_status plu_singlepass(plu_ctx* ctx, const plu_matrix* A, int k, uint64_t seed,
                          plu_prec prec, int32_t* p, int32_t* q, double* L, int64_t ldL,
                          double* U, int64_t ldU, plu_report* rep);

/* RandLU with power iteration (Alg. rlu, steps 1-3 replaced by
 * Alg. basicpoweriteration): the randomized LU the paper compares PowerLU
 * with.  Omega is n x l (the stream plu_powerlu uses for odd v); Y = A Omega,
 * then `piter` >= 0 rounds of A^T / A products, each re-orthogonalised by the
 * permuted L of an LU; the last product's full LU gives P and L_y (first k
 * columns); B = L_y^+ P A (Eq. pseudoinverse) is formed as
 * B^T = A^T Q R^{-T} with W = P^T L_y = Q R (CholeskyQR2), and
 * Q B^T = L' U' gives L = L_y U'^T, U = L'^T.  The call reads A 2 piter + 2
 * times.  1 <= k <= l < min(m, n), l <= 2048.  Outputs as plu_powerlu:
 * A[p[i], q[j]] ~= (L U)(i, j). */
plu_status plu_randlu(plu_ctx* ctx, const plu_matrix* A, int k, int l, int piter,
                      uint64_t seed, plu_prec prec, int32_t* p, int32_t* q, double* L,
                      int64_t ldL, double* U, int64_t ldU, plu_report* rep);

/* plu_powerlu on a sparse A: every pass over A (v of them) is an FP64 sparse
 * product (plu_spmm), everything else as plu_powerlu in PLU_FP64, except
 * that the dense products between the passes (CholeskyQR's X^T X and
 * X R^{-1}, the tail's B^T = V_k U_1^T and L = L_1 U_2^T) run as
 * FP64-accurate sums of exact BF16 slice products on the tensor cores (as
 * plu_cholqr1 with tc) when k, l <= 512.  The result is that of plu_powerlu
 * on the dense A in FP64 up to rounding.  rep->flops_passes counts 2 nnz
 * flops per column of a pass and rep->bytes_passes the CSR arrays plus the
 * operands. */
plu_status plu_powerlu_csr(plu_ctx* ctx, const plu_csr* A, int k, int l, int v, uint64_t seed,
                           int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                           int64_t ldU, plu_report* rep);

/* plu_powerlu_fp_restart on a sparse A, with FP64 sparse passes and the
 * products between them as in plu_powerlu_csr (max_rounds = 1 is
 * plu_powerlu_fp); ||A||_F^2 is the sum of val^2. */
plu_status plu_powerlu_fp_csr(plu_ctx* ctx, const plu_csr* A, double eps, int b, int l, int v,
                              int precise, int max_rounds, uint64_t seed, int* k_out,
                              int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                              int64_t ldU, plu_report* rep);

/* One problem of a batch (plu_batched).  A is m x n, column-major, device
 * memory, element type `dtype` (plu_dtype).  algo 0: PowerLU (Alg. bpowerlu
 * with Alg. gpowerlu), 1 <= k <= l < min(m, n), v >= 2; algo 1: single pass
 * (Alg. singlepasslu), 1 <= k < min(m, n), l and v ignored.  Outputs as in
 * plu_powerlu (device): p (m), q (n), L (m x k, ldL >= m), U (k x n, ldU >= k).
 * The Gaussian sketch of a problem is the one plu_powerlu / plu_singlepass
 * would draw from the same seed. */
typedef struct {
    int64_t m, n, ld;
    int32_t dtype;
    const void* A;
    int32_t k, l, v, algo;
    uint64_t seed;
    int32_t* p;
    int32_t* q;
    double* L;
    int64_t ldL;
    double* U;
    int64_t ldU;
} plu_batch_problem;

/* Batched factorisation of `count` independent problems of uneven size
 * (host array `problems`).  Every step of every problem runs in grouped
 * launches (one per kind of step and phase, each covering all problems), all
 * captured into one CUDA graph that is launched once on the context's stream.
 * prec: PLU_FP64 or PLU_FP32 (passes in FP32 FMA); tensor-core precisions are
 * not taken here.  Synchronises before returning.  rep (nullable) reports
 * the graph's device time, the passes and the kernels in the graph. */
plu_status plu_batched(plu_ctx* ctx, const plu_batch_problem* problems, int count, plu_prec prec,
                       plu_report* rep);

/* The tile shapes (rows bm[i] x columns bn[i] per CTA) of the grouped GEMM
 * launches of the last plu_batched call on ctx, in launch order.  The first
 * call for a batch signature (the problems' m, n, k, l, v, algo, dtype, ld and
 * the precision) times every launch in each shape the library has and keeps
 * the fastest; later calls with the same signature reuse that choice.  *count
 * receives the number of launches; at most cap entries are written. */
plu_status plu_batched_tiles(plu_ctx* ctx, int* bm, int* bn, int cap, int* count);

/* Every grouped GEMM of later plu_batched calls on ctx takes the tile shape
 * bm x bn (64 x 32, 64 x 64 or 128 x 32; PLU_EINVAL otherwise), without
 * split-K, instead of the autotuner's choice; bm = bn = 0 restores the
 * autotuner. */
plu_status plu_set_batched_tile(plu_ctx* ctx, int bm, int bn);

/* The split-K choice of each grouped GEMM launch of the last plu_batched call
 * on ctx, in launch order: kchunk[i] = the length of the K chunks its jobs
 * with few output tiles (at most 8) and a longer K were cut into, 0 for no
 * split.  The partial sums of the chunks are added in FP64 in chunk order
 * by a second grouped launch.  The autotuner picks the split-K length (none,
 * 1024, 256) together with the tile shape. */
plu_status plu_batched_splitk(plu_ctx* ctx, int* kchunk, int cap, int* count);

/* Persist the batched autotuner's choices in the text file at path (NULL or
 * "" turns it off).  A batch signature met for the first time in ctx is
 * looked up in the file before any timing, and a signature the autotuner
 * times is appended to it, so a later process skips the timing.  The file
 * must be openable for appending (PLU_EINVAL otherwise); its lines read
 * "plu-batched-tune 1 <signature> <launches> <choice>...", the last line of a
 * signature wins and malformed lines are ignored.  Processes that share the
 * file may append at once; a line is written with one call. */
plu_status plu_set_batched_tune_file(plu_ctx* ctx, const char* path);

/* ---------------------------------------------------------------------
 * Allocation-free variant (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory, such as code running
 * under a framework that owns all GPU memory through its own pool, plug-ins
 * that may not allocate, and latency-critical loops that cannot afford
 * cudaMalloc's device-wide synchronisation).
 *
 * Same result as plu_lu_reorth (X overwritten by P^T L, in place), with no
 * context and no allocation: the kernels' scratch is a fixed 2 MiB device
 * array inside the library, held by every GPU that loads the library until
 * the process exits.  Limits: rows <= 65536, cols <= 256; larger panels are
 * rejected with PLU_EINVAL and a message.  The work is enqueued on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream) of the current
 * device; the call then synchronises that stream and returns the device
 * status (PLU_ETIMEOUT, PLU_ENUMERIC).  The first call in each CUDA context
 * of a device (so the first call on the device, and the first one after a
 * device reset) looks up the array's device address: make that call before
 * any stream capture begins.  All calls
 * share the array, so calls whose GPU work overlaps race; each call clears
 * what must start at zero.  err (host buffer of err_len bytes, nullable)
 * receives a message on failure.
 * ------------------------------------------------------------------- */
plu_status plu_lu_reorth_static(void* cuda_stream, int64_t rows, int cols, double* X,
                                int64_t ldx, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* POWERLU_H */
