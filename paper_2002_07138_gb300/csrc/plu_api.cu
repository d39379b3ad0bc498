// C ABI entry points (include/powerlu.h): argument checks, workspace
// layout and the order of the steps of PowerLU (Alg. bpowerlu with
// Alg. gpowerlu), PowerLU_FP (Alg. powerlufp on Alg. adaptivewithoutupdating)
// on one CUDA stream.
#include "plu_internal.h"

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace plu;

thread_local long long plu::g_launches = 0;

struct plu_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    char* ws = nullptr;
    size_t ws_cap = 0;
    int* d_status = nullptr;   // device status word (DevStatus)
    int* h_status = nullptr;   // pinned mirror
    int* d_kmet = nullptr;     // rank scan results (k, met)
    double* d_scal = nullptr;  // device scalars: [0] ||A||_F^2, [1] E
    int* h_kmet = nullptr;
    double* h_scal = nullptr;
    int async = 0;
    int64_t spin_budget = kDefaultSpin;
    char err[512] = {0};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaStream_t capture = nullptr;   // private stream for graph capture (batched)
    // batched: the autotuner's tile shapes per batch signature, and those of
    // the last call
    std::map<uint64_t, std::vector<int>> batch_tiles;
    std::vector<int> last_tiles;
    int forced_tile = -1;             // a fixed tile shape instead of the autotuner
    double* bpart = nullptr;          // batched split-K partials (grown on demand)
    size_t bpart_cap = 0;
    std::string tune_file;            // autotuner choices persisted here (empty: off)
    // panel LU trailing updates: -1 default (tensor cores in the mixed modes and
    // on the sparse path, FP64 FMAs in the FP64 path), 0 FP64 FMAs, 1 tensor cores
    int lu_tc = -1;
    // set while a sparse driver runs: every pass over A is then a sparse product
    const plu_csr* csr = nullptr;
    static constexpr int64_t kDefaultSpin = 16LL << 20;
};

namespace {

constexpr uint32_t kStreamOmegaN = 1;   // n x l (odd v)
constexpr uint32_t kStreamOmegaM = 2;   // m x l (even v)
constexpr uint32_t kStreamOmegaSP = 3;  // m x k (single pass)
constexpr uint32_t kStreamRestartStride = 16;   // restart round r: streams + 16 r

plu_status fail(plu_ctx* c, plu_status st, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define PLU_CUDA(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess)                                                               \
            return fail(ctx, PLU_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                        __FILE__, __LINE__);                                                 \
    } while (0)

#define PLU_TRY(expr)                      \
    do {                                   \
        plu_status _s = (expr);            \
        if (_s != PLU_OK) return _s;       \
    } while (0)

plu_status ensure_ws(plu_ctx* c, size_t bytes) {
    if (bytes <= c->ws_cap) return PLU_OK;
    size_t want = bytes + (bytes >> 3) + (1 << 20);
    if (c->ws) {
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_cap = 0;
    }
    if (cudaMalloc(&c->ws, want) != cudaSuccess) {
        cudaGetLastError();
        c->ws = nullptr;
        return fail(c, PLU_ENOMEM, "workspace allocation of %zu bytes failed", want);
    }
    c->ws_cap = want;
    return PLU_OK;
}

// Two-phase layout: first count, then carve.
struct Layout {
    size_t total = 0;
    size_t add(size_t bytes) {
        size_t off = (total + 255) & ~size_t(255);
        total = off + bytes;
        return off;
    }
};

plu_status bind(plu_ctx* c) {
    if (!c) return PLU_EINVAL;
    PLU_CUDA(c, cudaSetDevice(c->device));
    return PLU_OK;
}

plu_status check_matrix(plu_ctx* c, const plu_matrix* A) {
    if (!A || !A->data) return fail(c, PLU_EINVAL, "A is NULL");
    if (A->m < 1 || A->n < 1) return fail(c, PLU_EINVAL, "A must be at least 1 x 1");
    if (A->ld < A->m) return fail(c, PLU_EINVAL, "ld (%lld) < m (%lld)", (long long)A->ld, (long long)A->m);
    if (A->dtype != PLU_F32 && A->dtype != PLU_F64) return fail(c, PLU_EINVAL, "bad dtype %d", A->dtype);
    if (A->m > (int64_t(1) << 31) - 1 || A->n > (int64_t(1) << 31) - 1)
        return fail(c, PLU_EINVAL, "dimensions must fit int32");
    return PLU_OK;
}

plu_status check_prec(plu_ctx* c, int prec, const plu_matrix* A) {
    if (prec == PLU_FP64 || prec == PLU_FP32) return PLU_OK;
    if (prec == PLU_TF32 || prec == PLU_BF16 || prec == PLU_FP8_E4M3 || prec == PLU_TF32X3) {
        if (A && A->dtype != PLU_F32)
            return fail(c, PLU_EUNSUPPORTED, "tensor-core passes need A stored in FP32");
        return PLU_OK;
    }
    return fail(c, PLU_EINVAL, "bad precision %d", prec);
}

// Finish a call: read the device status word unless asynchronous.
plu_status finish(plu_ctx* c) {
    if (c->async) return PLU_OK;
    return plu_check(c);
}

plu_status dev_status_to_plu(plu_ctx* c, int st) {
    if (st == DEV_OK) return PLU_OK;
    if (st == DEV_TIMEOUT) return fail(c, PLU_ETIMEOUT, "a device-side wait ran out of its budget");
    if (st == DEV_BADINDEX)
        return fail(c, PLU_EINDEX, "a sparse row pointer or column index is out of range");
    return fail(c, PLU_ENUMERIC, "non-finite value or breakdown in an FP64 factorisation");
}

// ---- workspace needs of the steps
bool is_tc(int prec) { return prec == PLU_TF32 || prec == PLU_BF16 || prec == PLU_FP8_E4M3; }

// FP32-accurate split products on the tensor cores (3xTF32, plu_tcsplit.cu)
// over an FP32 A, FP32 SIMT FMAs where the split kernel does not take the
// shape.  The mixed modes take it for the products that enter the result to
// first order: PowerLU's last pass and RandLU's B pass.
constexpr int kPrecSplit = PLU_TF32X3;

// Scratch of a panel LU of either kind (FP64 FMA updates or tensor-core updates).
size_t lu_scratch_bytes(int64_t rows, int cols) {
    const size_t a = panel_scratch_bytes(rows, cols), b = tclu_scratch_bytes(rows, cols);
    return a > b ? a : b;
}

// The panel LU of a step: trailing updates on the tensor cores (FP64-accurate
// exact digit products, plu_tclu.cu) when the context asks for them, and by
// default in the mixed-precision modes and on the sparse path (which already
// takes its other FP64 products that way); FP64 FMAs otherwise.  Both give
// the same pivot rule and outputs.
cudaError_t launch_lu(const plu_ctx* c, int prec, int64_t rows, int cols, double* X, int64_t ldx,
                      int mode, int32_t* perm, double* L, int64_t ldL, int l_trans, double* U,
                      int64_t ldU, int u_trans, int32_t* info, void* scratch, int* dev_status,
                      int64_t spin_budget, int num_sms, cudaStream_t s) {
    const bool want = c->lu_tc == 1 || (c->lu_tc < 0 && (prec != PLU_FP64 || c->csr != nullptr));
    if (want && tclu_supported(rows, cols, num_sms))
        return launch_panel_lu_tc(rows, cols, X, ldx, mode, perm, L, ldL, l_trans, U, ldU, u_trans,
                                  info, scratch, dev_status, spin_budget, num_sms, s);
    return launch_panel_lu(rows, cols, X, ldx, mode, perm, L, ldL, l_trans, U, ldU, u_trans, info,
                           scratch, dev_status, spin_budget, num_sms, s);
}

size_t pass_ws(int64_t M, int64_t N, int64_t K, int prec, int sms) {
    const int sprec = (is_tc(prec) || prec == kPrecSplit) ? PLU_FP32 : prec;
    size_t b = gemm_partials_bytes(M, N, K, sprec, sms) + 256;
    if (sprec == PLU_FP32) b += size_t(K) * N * sizeof(float) + 256;
    if (is_tc(prec)) {
        const size_t t = tc_scratch_bytes(M, K, int(N), sms);
        if (t > b) b = t;
    }
    if (is_tc(prec) || prec == kPrecSplit) {
        const size_t t = tcs_scratch_bytes(M, K, int(N), sms);
        if (t > b) b = t;
    }
    return b;
}

// One pass over A.  BF16 / FP8 passes read the quantized copy q (made once
// per call); TF32 reads the FP32 A directly; shapes the tensor-core kernel
// does not take (more than 512 columns, unaligned A) use the FP32 SIMT kernel.
// ws holds ws_cap bytes; a shape that needs more is an error, never an overrun.
// norm (nullable): ||A||_F^2 summed by the pass kernel from the entries it
// reads (not for the passes over a quantised copy: its quantisation does it).
plu_status do_pass(plu_ctx* c, const plu_matrix* A, int trans, const double* X, int64_t ldx,
                   int cols, int prec, double* Y, int64_t ldy, char* ws, size_t ws_cap,
                   const QuantA* q = nullptr, int accum = 0, const void* xq_pre = nullptr,
                   const NormOut* norm = nullptr) {
    const int64_t M = trans ? A->n : A->m;
    const int64_t K = trans ? A->m : A->n;
    if (c->csr) {
        const plu_csr* S = c->csr;
        PLU_CUDA(c, launch_spmm_csr(M, K, S->nnz, trans ? S->t_row_ptr : S->row_ptr,
                                    trans ? S->t_col_idx : S->col_idx, trans ? S->t_val : S->val,
                                    X, ldx, cols, Y, ldy, ws, ws_cap, c->d_status, c->num_sms,
                                    c->stream, norm));
        return PLU_OK;
    }
    if ((prec == PLU_BF16 || prec == PLU_FP8_E4M3) && q && cols <= 512) {
        if (norm) return fail(c, PLU_EINVAL, "a pass over a quantised copy cannot sum ||A||^2");
        PLU_CUDA(c, launch_tc_pass_q(trans, *q, X, ldx, cols, Y, ldy, ws, ws_cap, c->d_status,
                                     c->num_sms, c->stream, accum));
        return PLU_OK;
    }
    if (is_tc(prec) && A->dtype == PLU_F32 && tc_supported(M, K, cols, A->data, A->ld, trans)) {
        PLU_CUDA(c, launch_tc_pass(trans, A->m, A->n, static_cast<const float*>(A->data), A->ld, X,
                                   ldx, cols, Y, ldy, ws, ws_cap, c->d_status, c->num_sms,
                                   c->stream, accum, xq_pre, norm));
        return PLU_OK;
    }
    if (prec == kPrecSplit && A->dtype == PLU_F32 &&
        tcs_supported(M, K, cols, A->data, A->ld, trans)) {
        // xq_pre: X already in the split operand form (launch_tcs_operand)
        PLU_CUDA(c, launch_tc_split_pass(trans, A->m, A->n, static_cast<const float*>(A->data),
                                         A->ld, X, ldx, cols, Y, ldy, ws, ws_cap, c->d_status,
                                         c->num_sms, c->stream, accum, xq_pre, norm));
        return PLU_OK;
    }
    if (is_tc(prec) || prec == kPrecSplit) prec = PLU_FP32;
    Workspace w;
    w.base = ws;
    w.cap = ws_cap;
    float* b32 = nullptr;
    if (prec == PLU_FP32) {
        b32 = static_cast<float*>(w.take(size_t(K) * cols * sizeof(float)));
        if (!b32) return fail(c, PLU_ENOMEM, "pass scratch too small");
    }
    // the rest holds the split-K partial sums
    const size_t off = (w.used + 255) & ~size_t(255);
    const size_t part_cap = ws_cap > off ? ws_cap - off : 0;
    void* part = w.take(part_cap);
    PLU_CUDA(c, launch_gemm_simt(trans, M, cols, K, A->data, A->dtype, A->ld, X, ldx, Y, ldy, prec,
                                 part, part_cap, b32, c->num_sms, c->stream, accum, norm));
    return PLU_OK;
}

// Room for the per-CTA partials of ||A||_F^2 in whichever kernel runs the
// first pass (tensor-core pass, quantisation, SIMT GEMM or sparse pass).
int norm_parts_needed(int64_t m, int64_t n, int l, int sms) {
    int p = quant_norm_parts(sms);
    for (const int64_t M : {m, n}) {
        const int64_t K = M == m ? n : m;
        const int g = gemm_norm_parts(M, l, K, sms);
        if (g > p) p = g;
        const int sp = spmm_norm_parts(M, sms);
        if (sp > p) p = sp;
    }
    return p;
}

// Largest scratch over every rank 1..kmax the tail (and, on the sparse path,
// its slice products) may run at.  Neither size is monotone in the rank (the
// split count of a product changes with its shape), so every rank is
// evaluated; the result is kept per shape, so a driver pays the scan once.
struct TailScratchKey {
    int64_t m, n;
    int kmax, sms;
    bool oz;
    bool operator<(const TailScratchKey& o) const {
        if (m != o.m) return m < o.m;
        if (n != o.n) return n < o.n;
        if (kmax != o.kmax) return kmax < o.kmax;
        if (sms != o.sms) return sms < o.sms;
        return oz < o.oz;
    }
};

size_t tail_scratch_max(int64_t m, int64_t n, int kmax, int sms, bool oz) {
    static std::mutex mu;
    static std::map<TailScratchKey, size_t> memo;
    const TailScratchKey key{m, n, kmax, sms, oz};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
    }
    size_t best = 0;
    for (int kk = 1; kk <= kmax; ++kk)
        for (const int64_t rows : {m, n}) {
            size_t t;
            if (oz) t = oz_supported(rows, kk, sms) ? oz_scratch_bytes(rows, kk, sms) : 0;
            else t = gemm_f64_partials_bytes(rows, kk, kk, sms);
            if (t > best) best = t;
        }
    std::lock_guard<std::mutex> lock(mu);
    if (memo.size() > 256) memo.clear();
    memo[key] = best;
    return best;
}

struct PowerLUPlan {
    // offsets into the workspace
    size_t V, Z, step, L1, U1T, BT, U2T, tailpart, cn, normparts, quant, total;
    int normparts_cap;
    size_t step_bytes, tailpart_bytes;
};

// Shared by the fixed-rank and fixed-precision drivers: workspace for
// Alg. gpowerlu (basis V n x l, products Z m x l, step scratch) and the tail
// (Alg. bpowerlu steps 4-8) at rank kmax.
PowerLUPlan plan_powerlu(int64_t m, int64_t n, int l, int kmax, int prec, int sms,
                         bool sparse = false) {
    Layout lay;
    PowerLUPlan p{};
    p.V = lay.add(size_t(n) * l * sizeof(double));
    p.Z = lay.add(size_t(m) * l * sizeof(double));
    size_t step = pass_ws(m, l, n, prec, sms);
    size_t t = pass_ws(n, l, m, prec, sms);
    if (t > step) step = t;
    t = lu_scratch_bytes(m > n ? m : n, l);
    if (t > step) step = t;
    t = qr_scratch_bytes(n, l, sms);
    if (t > step) step = t;
    if (sparse) {
        t = spmm_scratch_bytes(m > n ? m : n, l);
        if (t > step) step = t;
        // the tail's slice products at any rank up to kmax
        t = tail_scratch_max(m, n, kmax, sms, true);
        if (t > step) step = t;
    }
    // the mixed modes' tail products as split-precision tensor-core products
    if (prec != PLU_FP64 && !sparse && kmax <= 512) {
        const int64_t mx = m > n ? m : n;
        t = tcs_product_scratch_bytes(mx, kmax, sms);
        if (t > step) step = t;
    }
    // the mixed modes and the sparse path orthonormalise with tensor-core
    // products (the kmax leading columns at fixed rank, all l columns at
    // fixed precision)
    if (prec != PLU_FP64 || sparse) {
        t = qr_scratch_bytes(n, kmax, sms, 1);
        if (t > step) step = t;
        t = qr_scratch_bytes(n, l, sms, 1);
        if (t > step) step = t;
    }
    p.step = lay.add(step);
    p.step_bytes = step;
    p.L1 = lay.add(size_t(m) * kmax * sizeof(double));
    p.U1T = lay.add(size_t(kmax) * kmax * sizeof(double));
    p.BT = lay.add(size_t(n) * kmax * sizeof(double));
    p.U2T = lay.add(size_t(kmax) * kmax * sizeof(double));
    // the tail runs at any rank k <= kmax (fixed precision): the largest
    // preferred partial-sum size over those ranks
    const size_t tp = tail_scratch_max(m, n, kmax, sms, false);
    p.tailpart = lay.add(tp);
    p.tailpart_bytes = tp;
    p.cn = lay.add(size_t(l) * sizeof(double) + norm2_scratch_bytes(sms));
    p.normparts_cap = norm_parts_needed(m, n, l, sms);
    p.normparts = lay.add(size_t(p.normparts_cap) * sizeof(double));
    p.quant = (prec == PLU_BF16 || prec == PLU_FP8_E4M3) ? lay.add(tc_quant_bytes(m, n, prec)) : 0;
    p.total = lay.total + 256;
    return p;
}

// CUDA events of a call (only when a report is requested): pairs around the
// passes, and phase boundaries (each phase lasts until the next boundary).
struct PassTimer {
    plu_ctx* c;
    bool on;
    cudaEvent_t ev[64];
    int n = 0;
    static constexpr int kMaxPhaseMarks = 128;
    cudaEvent_t pev[kMaxPhaseMarks];
    int pid[kMaxPhaseMarks];
    int np = 0;
    explicit PassTimer(plu_ctx* ctx, bool enable) : c(ctx), on(enable) {}
    ~PassTimer() {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
        for (int i = 0; i < np; ++i) cudaEventDestroy(pev[i]);
    }
    // start of phase id (PLU_PHASE_*; -1 ends the last one)
    void phase(int id) {
        if (!on || np >= kMaxPhaseMarks) return;
        cudaEventCreate(&pev[np]);
        cudaEventRecord(pev[np], c->stream);
        pid[np++] = id;
    }
    void phases_ms(double* out) {
        for (int i = 0; i < PLU_NPHASES; ++i) out[i] = 0.0;
        for (int i = 0; i + 1 < np; ++i) {
            if (pid[i] < 0 || pid[i] >= PLU_NPHASES) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pev[i], pev[i + 1]) == cudaSuccess) out[pid[i]] += ms;
        }
    }
    void mark() {
        if (!on || n >= 64) return;
        cudaEventCreate(&ev[n]);
        cudaEventRecord(ev[n], c->stream);
        ++n;
    }
    // sum of the (start, stop) pairs
    double pairs_ms() {
        double s = 0.0;
        for (int i = 0; i + 1 < n; i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) s += ms;
        }
        return s;
    }
};

// The remainder A_r = A - A W W^T of a restart round (the Remark after
// Alg. adaptivewithoutupdating), applied through G = A W:
// A_r X = A X - G (W^T X), A_r^T Z = A^T Z - W (G^T Z).  W (n x kw) and G
// (m x kw) are FP64, T (kw x cols) is scratch.
struct Remainder {
    const double* W = nullptr;
    const double* G = nullptr;
    int kw = 0;
    double* T = nullptr;
};

// Y -= the remainder's correction of a pass Y = op(A) X (cols columns).
plu_status remainder_correct(plu_ctx* c, const plu_matrix* A, const Remainder& r, int trans,
                             const double* X, int64_t ldx, int cols, double* Y, int64_t ldy,
                             char* step, size_t step_cap) {
    if (!r.W || r.kw < 1) return PLU_OK;
    const int64_t m = A->m, n = A->n;
    // T = W^T X (A X) or G^T X (A^T X); then Y -= G T or W T, in FP64
    PLU_CUDA(c, launch_gemm_f64(1, 0, r.kw, cols, trans ? m : n, trans ? r.G : r.W, trans ? m : n,
                                X, ldx, r.T, r.kw, step, step_cap, c->num_sms, c->stream));
    PLU_CUDA(c, launch_gemm_simt(0, trans ? n : m, cols, r.kw, trans ? r.W : r.G, PLU_F64,
                                 trans ? n : m, r.T, r.kw, Y, ldy, PLU_FP64, step, step_cap,
                                 nullptr, c->num_sms, c->stream, -1));
    return PLU_OK;
}

// Alg. gpowerlu into V (n x l).  Returns the number of passes launched.
// The final QR orthonormalises only the leading qr_cols columns of the
// n x l product: Q(:, 1:j) depends on X(:, 1:j) alone, and the fixed-rank
// path reads only V(:, 1:k) (Alg. bpowerlu step 3 and the tail).  With a
// remainder (restart round r), every pass is over A_r and Omega comes from
// the streams shifted by 16 r.
// first_norm (nullable): the first pass also sums ||A||_F^2 into it.
plu_status run_gpowerlu(plu_ctx* c, const plu_matrix* A, int l, int v, uint64_t seed, int prec,
                        double* V, double* Z, char* step, size_t step_cap, PassTimer& pt,
                        int* passes, const QuantA* q, int qr_cols, int adaptive_qr,
                        int tc_qr, const Remainder& rem = Remainder(), int round = 0,
                        const NormOut* first_norm = nullptr) {
    const int64_t m = A->m, n = A->n;
    const int p = (v - 1) / 2;
    const uint32_t shift = kStreamRestartStride * uint32_t(round);
    int np = 0;
    auto pass = [&](int trans, const double* X, int64_t ldx, double* Y, int64_t ldy) -> plu_status {
        pt.phase(PLU_PHASE_POWER_PASSES);
        pt.mark();
        PLU_TRY(do_pass(c, A, trans, X, ldx, l, prec, Y, ldy, step, step_cap, q, 0, nullptr,
                        np == 0 ? first_norm : nullptr));
        pt.mark();
        PLU_TRY(remainder_correct(c, A, rem, trans, X, ldx, l, Y, ldy, step, step_cap));
        ++np;
        return PLU_OK;
    };
    auto reorth = [&](int64_t rows, double* X) -> plu_status {
        pt.phase(PLU_PHASE_REORTH);
        PLU_CUDA(c, launch_lu(c, prec, rows, l, X, rows, 0, nullptr, nullptr, 0, 0, nullptr, 0, 0,
                                    nullptr, step, c->d_status, c->spin_budget, c->num_sms,
                                    c->stream));
        return PLU_OK;
    };
    auto qr = [&](double* X) -> plu_status {
        pt.phase(PLU_PHASE_QR);
        const cudaError_t e = launch_cholqr2(n, qr_cols, X, n, nullptr, 0, step, step_cap,
                                             c->d_status, c->num_sms, c->stream, adaptive_qr, 2,
                                             tc_qr);
        if (e != cudaSuccess)
            return fail(c, PLU_ECUDA, "CholeskyQR (%s): %s", cholqr_failed_step(),
                        cudaGetErrorString(e));
        return PLU_OK;
    };
    pt.phase(PLU_PHASE_SKETCH);
    if (v % 2 == 0) {
        PLU_CUDA(c, launch_gaussian(m, l, seed, kStreamOmegaM + shift, Z, m, c->stream));
        PLU_TRY(pass(1, Z, m, V, n));                 // A^T Omega
        if (v > 2) PLU_TRY(reorth(n, V));
        else PLU_TRY(qr(V));
    } else {
        PLU_CUDA(c, launch_gaussian(n, l, seed, kStreamOmegaN + shift, V, n, c->stream));
    }
    for (int i = 1; i <= p; ++i) {
        PLU_TRY(pass(0, V, n, Z, m));                 // A V
        PLU_TRY(reorth(m, Z));
        PLU_TRY(pass(1, Z, m, V, n));                 // A^T V
        if (i == p) PLU_TRY(qr(V));
        else PLU_TRY(reorth(n, V));
    }
    *passes = np;
    return PLU_OK;
}

// Alg. bpowerlu steps 4-8 on Y (m x k, ld m, destroyed) and Vk (n x k, ld n).
plu_status run_tail(plu_ctx* c, int64_t m, int64_t n, int k, double* Y, const double* Vk,
                    char* ws, const PowerLUPlan& pl, char* step, int32_t* p, int32_t* q,
                    double* L, int64_t ldL, double* U, int64_t ldU, int32_t* info2dev,
                    int prec, bool oz, PassTimer& pt) {
    double* L1 = reinterpret_cast<double*>(ws + pl.L1);
    double* U1T = reinterpret_cast<double*>(ws + pl.U1T);
    double* BT = reinterpret_cast<double*>(ws + pl.BT);
    double* U2T = reinterpret_cast<double*>(ws + pl.U2T);
    void* tp = ws + pl.tailpart;
    // [L1, U1, P] = lu(Y)
    pt.phase(PLU_PHASE_TAIL_LU);
    PLU_CUDA(c, launch_lu(c, prec, m, k, Y, m, 1, p, L1, m, 0, U1T, k, 1, info2dev, step, c->d_status,
                                c->spin_budget, c->num_sms, c->stream));
    // The two m x k x k products are FP32-accurate when the passes are not
    // FP64: Y itself then carries the pass precision's rounding (2^-11
    // relative for TF32), far above the few 1e-7 these products add.  They
    // run as split-precision tensor-core products (3xTF32 on an FP32 copy of
    // the left operand) when the step scratch holds them, else with FP32
    // FMAs.  The getrf steps stay FP64.
    const bool f32 = prec != PLU_FP64;
    const bool tcs_bt = f32 && k <= 512 &&
                        tcs_product_scratch_bytes(n, k, c->num_sms) <= pl.step_bytes;
    const bool tcs_l = f32 && k <= 512 &&
                       tcs_product_scratch_bytes(m, k, c->num_sms) <= pl.step_bytes;
    // oz: the FP64 products as FP64-accurate sums of exact BF16 slice
    // products on the tensor cores (U1^T and U2^T are stored whole, zeros
    // above the diagonal, so the dense slice product applies)
    const bool oz_bt = oz && !f32 && oz_supported(n, k, c->num_sms) &&
                       oz_scratch_bytes(n, k, c->num_sms) <= pl.step_bytes;
    const bool oz_l = oz && !f32 && oz_supported(m, k, c->num_sms) &&
                      oz_scratch_bytes(m, k, c->num_sms) <= pl.step_bytes;
    // B^T = Vk U1^T (U1^T lower triangular)
    pt.phase(PLU_PHASE_TAIL_PRODUCTS);
    if (oz_bt)
        PLU_CUDA(c, launch_oz_xrinv(n, k, Vk, n, U1T, BT, n, step, pl.step_bytes, c->d_status,
                                    c->num_sms, c->stream));
    else if (tcs_bt)
        PLU_CUDA(c, launch_tcs_product(n, k, Vk, n, U1T, k, BT, n, step, pl.step_bytes,
                                       c->d_status, c->num_sms, c->stream));
    else if (f32)
        PLU_CUDA(c, launch_gemm_f32_tri(3, n, k, k, Vk, n, U1T, k, BT, n, tp, pl.tailpart_bytes,
                                        c->num_sms, c->stream));
    else
        PLU_CUDA(c, launch_gemm_f64_tri(0, 3, n, k, k, Vk, n, U1T, k, BT, n, tp,
                                        pl.tailpart_bytes, c->num_sms, c->stream));
    // [L2, U2, Q] = lu(B^T); U = L2^T written straight into U
    pt.phase(PLU_PHASE_TAIL_LU);
    PLU_CUDA(c, launch_lu(c, prec, n, k, BT, n, 1, q, U, ldU, 1, U2T, k, 1, info2dev + 1, step,
                                c->d_status, c->spin_budget, c->num_sms, c->stream));
    // L = L1 U2^T (U2^T lower triangular)
    pt.phase(PLU_PHASE_TAIL_PRODUCTS);
    if (oz_l)
        PLU_CUDA(c, launch_oz_xrinv(m, k, L1, m, U2T, L, ldL, step, pl.step_bytes, c->d_status,
                                    c->num_sms, c->stream));
    else if (tcs_l)
        PLU_CUDA(c, launch_tcs_product(m, k, L1, m, U2T, k, L, ldL, step, pl.step_bytes,
                                       c->d_status, c->num_sms, c->stream));
    else if (f32)
        PLU_CUDA(c, launch_gemm_f32_tri(3, m, k, k, L1, m, U2T, k, L, ldL, tp, pl.tailpart_bytes,
                                        c->num_sms, c->stream));
    else
        PLU_CUDA(c, launch_gemm_f64_tri(0, 3, m, k, k, L1, m, U2T, k, L, ldL, tp,
                                        pl.tailpart_bytes, c->num_sms, c->stream));
    return PLU_OK;
}

void fill_pass_report(plu_report* rep, const plu_matrix* A, int passes_l, int l, int k_last,
                      int prec, bool final_pass, const plu_csr* sp = nullptr) {
    // a sparse pass does 2 flops per nonzero and column and reads the CSR
    // arrays of A or A^T (the larger row-pointer array counted)
    const double mn = sp ? double(sp->nnz) : double(A->m) * double(A->n);
    const double abytes =
        sp ? double(sp->nnz) * 12.0 + double((A->m > A->n ? A->m : A->n) + 1) * 8.0
           : mn * (A->dtype == PLU_F32 ? 4.0 : 8.0);
    double fl = 2.0 * mn * l * passes_l;
    double by = (abytes + double(A->m + A->n) * l * 8.0) * passes_l;
    if (final_pass) {
        fl += 2.0 * mn * k_last;
        by += abytes + double(A->m + A->n) * k_last * 8.0;
    }
    (void)prec;
    rep->flops_passes = fl;
    rep->bytes_passes = by;
}

}  // namespace

// ---- sparse A
namespace {

plu_status check_csr(plu_ctx* c, const plu_csr* A) {
    if (!A) return fail(c, PLU_EINVAL, "A is NULL");
    if (A->m < 1 || A->n < 1) return fail(c, PLU_EINVAL, "A must be at least 1 x 1");
    if (A->m > (int64_t(1) << 31) - 1 || A->n > (int64_t(1) << 31) - 1)
        return fail(c, PLU_EINVAL, "dimensions must fit int32");
    if (A->nnz < 0) return fail(c, PLU_EINVAL, "nnz < 0");
    if (!A->row_ptr || !A->t_row_ptr) return fail(c, PLU_EINVAL, "row pointers are NULL");
    if (A->nnz > 0 && (!A->col_idx || !A->val || !A->t_col_idx || !A->t_val))
        return fail(c, PLU_EINVAL, "index or value arrays are NULL");
    return PLU_OK;
}

// The dense drivers run on A's shape with every pass routed to the sparse
// product while the guard lives.
struct CsrScope {
    plu_ctx* c;
    plu_matrix shape;
    CsrScope(plu_ctx* ctx, const plu_csr* A) : c(ctx) {
        c->csr = A;
        shape.m = A->m;
        shape.n = A->n;
        shape.ld = A->m;
        shape.dtype = PLU_F64;
        shape.data = A->row_ptr;
    }
    ~CsrScope() { c->csr = nullptr; }
};

}  // namespace

// ======================================================================
extern "C" {

plu_status plu_create(plu_ctx** out, int device, void* cuda_stream) {
    if (!out) return PLU_EINVAL;
    *out = nullptr;
    plu_ctx* c = new (std::nothrow) plu_ctx();
    if (!c) return PLU_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete c;
        return PLU_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->d_status, 64) != cudaSuccess ||
        cudaMallocHost(&c->h_status, 64) != cudaSuccess) {
        cudaGetLastError();
        plu_destroy(c);
        return PLU_ECUDA;
    }
    c->d_kmet = c->d_status + 4;
    c->d_scal = reinterpret_cast<double*>(c->d_status + 8);
    c->h_kmet = c->h_status + 4;
    c->h_scal = reinterpret_cast<double*>(c->h_status + 8);
    if (cudaMemset(c->d_status, 0, 64) != cudaSuccess ||
        cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        plu_destroy(c);
        return PLU_ECUDA;
    }
    *out = c;
    return PLU_OK;
}

void plu_destroy(plu_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->ws) cudaFree(c->ws);
    if (c->d_status) cudaFree(c->d_status);
    if (c->h_status) cudaFreeHost(c->h_status);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->bpart) cudaFree(c->bpart);
    delete c;
}

const char* plu_last_error(const plu_ctx* c) { return c ? c->err : "NULL context"; }

plu_status plu_set_stream(plu_ctx* c, void* s) {
    if (!c) return PLU_EINVAL;
    c->stream = static_cast<cudaStream_t>(s);
    return PLU_OK;
}

plu_status plu_set_async(plu_ctx* c, int async) {
    if (!c) return PLU_EINVAL;
    c->async = async ? 1 : 0;
    return PLU_OK;
}

plu_status plu_set_wait_budget(plu_ctx* c, int64_t spins) {
    if (!c) return PLU_EINVAL;
    c->spin_budget = spins > 0 ? spins : plu_ctx::kDefaultSpin;
    return PLU_OK;
}

plu_status plu_set_lu_updates(plu_ctx* c, int mode) {
    if (!c) return PLU_EINVAL;
    if (mode < -1 || mode > 1) return fail(c, PLU_EINVAL, "lu update mode must be -1, 0 or 1");
    c->lu_tc = mode;
    return PLU_OK;
}

plu_status plu_check(plu_ctx* c) {
    PLU_TRY(bind(c));
    PLU_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PLU_CUDA(c, cudaStreamSynchronize(c->stream));
    const int st = c->h_status[0];
    if (st != DEV_OK) {
        PLU_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return dev_status_to_plu(c, st);
}

plu_status plu_gaussian(plu_ctx* c, int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                        double* out, int64_t ld) {
    PLU_TRY(bind(c));
    if (rows < 0 || cols < 0 || (rows * cols > 0 && !out) || ld < (rows > 1 ? rows : 1))
        return fail(c, PLU_EINVAL, "bad gaussian arguments");
    PLU_CUDA(c, launch_gaussian(rows, cols, seed, stream_id, out, ld, c->stream));
    return finish(c);
}

plu_status plu_pass(plu_ctx* c, const plu_matrix* A, int trans, const double* X, int64_t ldx,
                    int cols, plu_prec prec, double* Y, int64_t ldy) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    PLU_TRY(check_prec(c, prec, A));
    const int64_t M = trans ? A->n : A->m;
    const int64_t K = trans ? A->m : A->n;
    if (cols < 1 || !X || !Y || ldx < K || ldy < M) return fail(c, PLU_EINVAL, "bad pass operands");
    const bool quant = (prec == PLU_BF16 || prec == PLU_FP8_E4M3) && cols <= 512;
    const size_t qb = quant ? ((tc_quant_bytes(A->m, A->n, prec) + 255) & ~size_t(255)) : 0;
    const size_t pw = pass_ws(M, cols, K, prec, c->num_sms);
    PLU_TRY(ensure_ws(c, qb + pw));
    QuantA q;
    if (quant)
        PLU_CUDA(c, launch_tc_quantize(prec, static_cast<const float*>(A->data), A->m, A->n, A->ld,
                                       c->ws, &q, c->num_sms, c->stream));
    PLU_TRY(do_pass(c, A, trans, X, ldx, cols, prec, Y, ldy, c->ws + qb, pw, quant ? &q : nullptr));
    return finish(c);
}

plu_status plu_lu_reorth(plu_ctx* c, int64_t rows, int cols, double* X, int64_t ldx) {
    PLU_TRY(bind(c));
    if (cols < 1 || rows < cols || !X || ldx < rows || cols > 2048)
        return fail(c, PLU_EINVAL, "lu_reorth needs rows >= cols >= 1, cols <= 2048, ldx >= rows");
    PLU_TRY(ensure_ws(c, lu_scratch_bytes(rows, cols)));
    PLU_CUDA(c, launch_lu(c, PLU_FP64, rows, cols, X, ldx, 0, nullptr, nullptr, 0, 0, nullptr, 0, 0, nullptr,
                                c->ws, c->d_status, c->spin_budget, c->num_sms, c->stream));
    return finish(c);
}

plu_status plu_getrf(plu_ctx* c, int64_t rows, int cols, double* X, int64_t ldx, int32_t* perm,
                     double* L, int64_t ldL, double* U, int64_t ldU, int32_t* info) {
    PLU_TRY(bind(c));
    if (cols < 1 || rows < cols || !X || ldx < rows || cols > 2048 || !perm || !L || !U ||
        ldL < rows || ldU < cols)
        return fail(c, PLU_EINVAL, "getrf needs rows >= cols >= 1, cols <= 2048 and valid outputs");
    PLU_TRY(ensure_ws(c, lu_scratch_bytes(rows, cols)));
    PLU_CUDA(c, launch_lu(c, PLU_FP64, rows, cols, X, ldx, 1, perm, L, ldL, 0, U, ldU, 0, info, c->ws,
                                c->d_status, c->spin_budget, c->num_sms, c->stream));
    return finish(c);
}

plu_status plu_qr(plu_ctx* c, int64_t rows, int cols, double* X, int64_t ldx, double* R, int64_t ldR) {
    PLU_TRY(bind(c));
    if (cols < 1 || rows < cols || !X || ldx < rows || (R && ldR < cols))
        return fail(c, PLU_EINVAL, "qr needs rows >= cols >= 1");
    const size_t qw = qr_scratch_bytes(rows, cols, c->num_sms);
    PLU_TRY(ensure_ws(c, qw));
    PLU_CUDA(c, launch_cholqr2(rows, cols, X, ldx, R, ldR, c->ws, qw, c->d_status, c->num_sms,
                               c->stream));
    return finish(c);
}

plu_status plu_cholqr1(plu_ctx* c, int64_t rows, int cols, double* X, int64_t ldx, double* R,
                       int64_t ldR, int tc) {
    PLU_TRY(bind(c));
    if (cols < 1 || rows < cols || !X || ldx < rows || (R && ldR < cols))
        return fail(c, PLU_EINVAL, "cholqr1 needs rows >= cols >= 1");
    if (tc && !oz_supported(rows, cols, c->num_sms))
        return fail(c, PLU_EUNSUPPORTED, "tensor-core products need cols <= 512 and a shorter X");
    const size_t qw = qr_scratch_bytes(rows, cols, c->num_sms, tc ? 1 : 0);
    PLU_TRY(ensure_ws(c, qw));
    PLU_CUDA(c, launch_cholqr2(rows, cols, X, ldx, R, ldR, c->ws, qw, c->d_status, c->num_sms,
                               c->stream, 0, 1, tc ? 1 : 0));
    return finish(c);
}

plu_status plu_norm2(plu_ctx* c, const plu_matrix* A, double* out) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    if (!out) return fail(c, PLU_EINVAL, "out is NULL");
    PLU_TRY(ensure_ws(c, norm2_scratch_bytes(c->num_sms)));
    PLU_CUDA(c, launch_norm2(A->data, A->dtype, A->m, A->n, A->ld, c->d_scal, c->ws, c->num_sms,
                             c->stream));
    PLU_CUDA(c, cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PLU_TRY(plu_check(c));
    *out = c->h_scal[0];
    return PLU_OK;
}

plu_status plu_rank(plu_ctx* c, int64_t rows, int cols, const double* G, int64_t ldg, double normA2,
                    double eps, int b, int precise, int* k_out, double* E_out) {
    PLU_TRY(bind(c));
    if (rows < 1 || cols < 1 || !G || ldg < rows || !(eps > 0.0 && eps < 1.0) || b < 1 || !k_out)
        return fail(c, PLU_EINVAL, "bad rank arguments");
    PLU_TRY(ensure_ws(c, size_t(cols) * sizeof(double) + 256));
    double* cn = reinterpret_cast<double*>(c->ws);
    c->h_scal[0] = normA2;
    PLU_CUDA(c, cudaMemcpyAsync(c->d_scal, c->h_scal, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PLU_CUDA(c, launch_colnorm2(rows, cols, G, ldg, cn, c->stream));
    PLU_CUDA(c, launch_rank_scan(cn, cols, c->d_scal, eps, b, precise, c->d_kmet, c->d_scal + 1,
                                 c->stream));
    PLU_CUDA(c, cudaMemcpyAsync(c->h_kmet, c->d_kmet, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PLU_CUDA(c, cudaMemcpyAsync(c->h_scal + 1, c->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    PLU_TRY(plu_check(c));
    *k_out = c->h_kmet[0];
    if (E_out) *E_out = c->h_scal[1];
    return c->h_kmet[1] ? PLU_OK : fail(c, PLU_TOL_NOT_MET, "tolerance not met within %d columns", cols);
}

plu_status plu_powerlu(plu_ctx* c, const plu_matrix* A, int k, int l, int v, uint64_t seed,
                       plu_prec prec, int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                       int64_t ldU, plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    PLU_TRY(check_prec(c, prec, A));
    const int64_t m = A->m, n = A->n;
    const int64_t mn = m < n ? m : n;
    if (k < 1 || l < k || l >= mn) return fail(c, PLU_EINVAL, "need 1 <= k <= l < min(m, n)");
    if (v < 2) return fail(c, PLU_EINVAL, "need v >= 2 passes");
    if (l > 2048) return fail(c, PLU_EINVAL, "l > 2048 is not supported");
    if (!p || !q || !L || !U || ldL < m || ldU < k) return fail(c, PLU_EINVAL, "bad outputs");
    const PowerLUPlan pl = plan_powerlu(m, n, l, k, prec, c->num_sms, c->csr != nullptr);
    PLU_TRY(ensure_ws(c, pl.total));
    char* ws = c->ws;
    double* V = reinterpret_cast<double*>(ws + pl.V);
    double* Z = reinterpret_cast<double*>(ws + pl.Z);
    char* step = ws + pl.step;
    PassTimer pt(c, rep != nullptr);
    const long long launches0 = g_launches;
    if (rep) PLU_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    int np = 0;
    QuantA qa;
    const bool quant = prec == PLU_BF16 || prec == PLU_FP8_E4M3;
    pt.phase(PLU_PHASE_SKETCH);
    if (quant)
        PLU_CUDA(c, launch_tc_quantize(prec, static_cast<const float*>(A->data), m, n, A->ld,
                                       ws + pl.quant, &qa, c->num_sms, c->stream));
    // mixed modes: one CholeskyQR round when it is orthogonal enough (see
    // launch_cholqr2); the FP64 path keeps both rounds.  The sparse path (FP64
    // passes) takes CholeskyQR's products, and the tail's, as FP64-accurate
    // slice products on the tensor cores: at GB300's FP64 FMA rate they would
    // outlast the sparse passes.
    PLU_TRY(run_gpowerlu(c, A, l, v, seed, prec, V, Z, step, pl.step_bytes, pt, &np,
                         quant ? &qa : nullptr, k, prec != PLU_FP64 ? 1 : 0,
                         prec != PLU_FP64 || c->csr ? 1 : 0));
    // Y = A V(:, 1:k) (Alg. bpowerlu step 3), the v-th pass; in the mixed
    // modes it reads the FP32 A with FP32-accurate split products (3xTF32):
    // it enters the result to first order
    pt.phase(PLU_PHASE_LAST_PASS);
    pt.mark();
    PLU_TRY(do_pass(c, A, 0, V, n, k, is_tc(prec) ? kPrecSplit : int(prec), Z, m, step,
                    pl.step_bytes));
    pt.mark();
    ++np;
    int32_t* info = reinterpret_cast<int32_t*>(ws + pl.cn);
    PLU_TRY(run_tail(c, m, n, k, Z, V, ws, pl, step, p, q, L, ldL, U, ldU, info, prec,
                     c->csr != nullptr, pt));
    pt.phase(-1);
    if (rep) {
        PLU_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
        int32_t hinfo[2] = {0, 0};
        PLU_CUDA(c, cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        memset(rep, 0, sizeof(*rep));
        rep->ms_total = ms;
        rep->ms_passes = pt.pairs_ms();
        rep->passes = np;
        rep->rank = k;
        rep->indicator = -1.0;
        rep->normA2 = -1.0;
        rep->info1 = hinfo[0];
        rep->info2 = hinfo[1];
        fill_pass_report(rep, A, np - 1, l, k, prec, true, c->csr);
        rep->launches = int32_t(g_launches - launches0);
        pt.phases_ms(rep->ms_phase);
    }
    return finish(c);
}

// Alg. powerlufp with up to max_rounds rounds of Alg. adaptivewithoutupdating
// (the restart of its Remark: round r runs on the remainder A - A W W^T of the
// earlier rounds' bases W, with Omega from streams shifted by 16 r, and the
// indicator E carries over).  One round is Alg. powerlufp as printed.
plu_status powerlu_fp_rounds(plu_ctx* c, const plu_matrix* A, double eps, int b, int l, int v,
                             int precise, int max_rounds, uint64_t seed, plu_prec prec,
                             int* k_out, int32_t* p, int32_t* q, double* L, int64_t ldL,
                             double* U, int64_t ldU, plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    PLU_TRY(check_prec(c, prec, A));
    const int64_t m = A->m, n = A->n;
    const int64_t mn = m < n ? m : n;
    if (!(eps > 0.0 && eps < 1.0)) return fail(c, PLU_EINVAL, "need 0 < eps < 1");
    if (b < 1 || l < b || l >= mn) return fail(c, PLU_EINVAL, "need 1 <= b <= l < min(m, n)");
    if (v < 2) return fail(c, PLU_EINVAL, "need v >= 2 passes");
    if (l > 2048) return fail(c, PLU_EINVAL, "l > 2048 is not supported");
    if (max_rounds < 1 || int64_t(max_rounds) * l > 2048 || int64_t(max_rounds) * l >= mn)
        return fail(c, PLU_EINVAL, "need max_rounds >= 1 and max_rounds * l <= 2048, < min(m, n)");
    const int K = l * max_rounds;                       // largest possible rank
    if (!k_out || !p || !q || !L || !U || ldL < m || ldU < K)
        return fail(c, PLU_EINVAL, "bad outputs (L needs m x %d, U %d x n)", K, K);
    const PowerLUPlan pl = plan_powerlu(m, n, l, K, prec, c->num_sms, c->csr != nullptr);
    // restart rounds: the union of the bases W (n x K), G = A W (m x K), and
    // the corrections' scratch T (K x l)
    Layout lay;
    lay.total = pl.total;
    const bool multi = max_rounds > 1;
    const size_t oW = multi ? lay.add(size_t(n) * K * sizeof(double)) : 0;
    const size_t oG = multi ? lay.add(size_t(m) * K * sizeof(double)) : 0;
    const size_t oT = multi ? lay.add(size_t(K) * l * sizeof(double)) : 0;
    PLU_TRY(ensure_ws(c, lay.total + 256));
    char* ws = c->ws;
    double* V = reinterpret_cast<double*>(ws + pl.V);
    double* Z = reinterpret_cast<double*>(ws + pl.Z);
    double* Wu = multi ? reinterpret_cast<double*>(ws + oW) : nullptr;
    double* Gu = multi ? reinterpret_cast<double*>(ws + oG) : nullptr;
    double* T = multi ? reinterpret_cast<double*>(ws + oT) : nullptr;
    char* step = ws + pl.step;
    double* cn = reinterpret_cast<double*>(ws + pl.cn);
    PassTimer pt(c, rep != nullptr);
    const long long launches0 = g_launches;
    if (rep) PLU_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    // E = ||A||_F^2 (Alg. adaptivewithoutupdating step 1) is summed from the
    // entries of A that the first read of A stages: the first pass of
    // Alg. gpowerlu, or the quantisation in the BF16 / FP8 modes (itself a
    // read of A).  So A is read v times, as the algorithm counts passes.
    NormOut norm;
    norm.parts = reinterpret_cast<double*>(ws + pl.normparts);
    norm.cap = pl.normparts_cap;
    norm.out = c->d_scal;
    int np = 0;
    QuantA qa;
    const bool quant = prec == PLU_BF16 || prec == PLU_FP8_E4M3;
    pt.phase(PLU_PHASE_SKETCH);
    if (quant)
        PLU_CUDA(c, launch_tc_quantize(prec, static_cast<const float*>(A->data), m, n, A->ld,
                                       ws + pl.quant, &qa, c->num_sms, c->stream, &norm));
    int kw = 0, met = 0, rounds = 0;
    for (int r = 0; r < max_rounds; ++r) {
        Remainder rem;
        if (r > 0) {
            rem.W = Wu;
            rem.G = Gu;
            rem.kw = kw;
            rem.T = T;
        }
        int npr = 0;
        PLU_TRY(run_gpowerlu(c, A, l, v, seed, prec, V, Z, step, pl.step_bytes, pt, &npr,
                             quant ? &qa : nullptr, l, 0, prec != PLU_FP64 || c->csr ? 1 : 0,
                             rem, r, (r == 0 && !quant) ? &norm : nullptr));
        np += npr;
        // G = A V (step 3), the v-th pass.  Its column norms decide the rank:
        // E = ||A||_F^2 - sum ||G(:, j)||^2 must resolve eps^2 ||A||_F^2 without
        // bias.  The tensor cores' accumulator adds shrink every sum toward
        // zero (measured at 32768^2: -4e-4 relative for TF32 and -2e-6 for the
        // split products even with FP64 sums of 1024-long segments), which
        // biases sum ||G(:, j)||^2 by more than eps^2 = 1e-6; so every mode but
        // FP64 takes this pass with FP32 FMAs and FP64 partial sums (unbiased).
        pt.phase(PLU_PHASE_LAST_PASS);
        pt.mark();
        PLU_TRY(do_pass(c, A, 0, V, n, l, prec == PLU_FP64 ? int(prec) : int(PLU_FP32), Z, m,
                        step, pl.step_bytes));
        pt.mark();
        PLU_TRY(remainder_correct(c, A, rem, 0, V, n, l, Z, m, step, pl.step_bytes));
        ++np;
        pt.phase(PLU_PHASE_RANK);
        PLU_CUDA(c, launch_colnorm2(m, l, Z, m, cn, c->stream));
        PLU_CUDA(c, launch_rank_scan(cn, l, c->d_scal, eps, b, precise, c->d_kmet, c->d_scal + 1,
                                     c->stream, r > 0 ? c->d_scal + 1 : nullptr));
        PLU_CUDA(c, cudaMemcpyAsync(c->h_kmet, c->d_kmet, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
        PLU_CUDA(c, cudaMemcpyAsync(c->h_scal, c->d_scal, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        const int kr = c->h_kmet[0];
        met = c->h_kmet[1];
        if (kr < 1 || kr > l) return fail(c, PLU_ECUDA, "rank scan returned k = %d", kr);
        rounds = r + 1;
        if (!multi) {
            kw = kr;
            break;
        }
        PLU_CUDA(c, launch_copy_cols(n, kr, V, n, Wu + size_t(kw) * n, n, c->stream));
        PLU_CUDA(c, launch_copy_cols(m, kr, Z, m, Gu + size_t(kw) * m, m, c->stream));
        kw += kr;
        if (met) break;
    }
    const int k = kw;
    int32_t* info = reinterpret_cast<int32_t*>(c->d_kmet + 2);
    PLU_TRY(run_tail(c, m, n, k, multi ? Gu : Z, multi ? Wu : V, ws, pl, step, p, q, L, ldL, U,
                     ldU, info, prec, c->csr != nullptr, pt));
    pt.phase(-1);
    *k_out = k;
    if (rep) {
        PLU_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
        int32_t hinfo[2] = {0, 0};
        PLU_CUDA(c, cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        memset(rep, 0, sizeof(*rep));
        rep->ms_total = ms;
        rep->ms_passes = pt.pairs_ms();
        rep->passes = np;
        rep->rank = k;
        const double nA2 = c->h_scal[0], E = c->h_scal[1];
        rep->normA2 = nA2;
        rep->indicator = nA2 > 0 ? sqrt((E > 0 ? E : 0.0) / nA2) : 0.0;
        rep->info1 = hinfo[0];
        rep->info2 = hinfo[1];
        rep->rounds = rounds;
        fill_pass_report(rep, A, np, l, 0, prec, false, c->csr);
        rep->launches = int32_t(g_launches - launches0);
        pt.phases_ms(rep->ms_phase);
    }
    plu_status st = finish(c);
    if (st != PLU_OK) return st;
    return met ? PLU_OK
               : fail(c, PLU_TOL_NOT_MET, "tolerance not met within %d round(s) of l = %d columns",
                      rounds, l);
}

plu_status plu_powerlu_fp(plu_ctx* c, const plu_matrix* A, double eps, int b, int l, int v,
                          int precise, uint64_t seed, plu_prec prec, int* k_out, int32_t* p,
                          int32_t* q, double* L, int64_t ldL, double* U, int64_t ldU,
                          plu_report* rep) {
    return powerlu_fp_rounds(c, A, eps, b, l, v, precise, 1, seed, prec, k_out, p, q, L, ldL, U,
                             ldU, rep);
}

plu_status plu_powerlu_fp_restart(plu_ctx* c, const plu_matrix* A, double eps, int b, int l,
                                  int v, int precise, int max_rounds, uint64_t seed,
                                  plu_prec prec, int* k_out, int32_t* p, int32_t* q, double* L,
                                  int64_t ldL, double* U, int64_t ldU, plu_report* rep) {
    return powerlu_fp_rounds(c, A, eps, b, l, v, precise, max_rounds, seed, prec, k_out, p, q, L,
                             ldL, U, ldU, rep);
}

plu_status plu_singlepass(plu_ctx* c, const plu_matrix* A, int k, uint64_t seed, plu_prec prec,
                          int32_t* p, int32_t* q, double* L, int64_t ldL, double* U, int64_t ldU,
                          plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    PLU_TRY(check_prec(c, prec, A));
    if (prec == PLU_BF16 || prec == PLU_FP8_E4M3)
        return fail(c, PLU_EUNSUPPORTED,
                    "single pass: a quantized copy would need its own read of A; use TF32");
    const int64_t m = A->m, n = A->n;
    const int64_t mn = m < n ? m : n;
    if (k < 1 || k >= mn) return fail(c, PLU_EINVAL, "need 1 <= k < min(m, n)");
    if (k > 2048) return fail(c, PLU_EINVAL, "k > 2048 is not supported");
    if (!p || !q || !L || !U || ldL < m || ldU < k) return fail(c, PLU_EINVAL, "bad outputs");
    const int64_t es = A->dtype == PLU_F32 ? 4 : 8;
    // column panels small enough to stay in L2 between their two products
    int64_t wc = (int64_t(48) << 20) / (m * es) / 128 * 128;
    if (wc < 128) wc = 128;
    if (wc > n) wc = n;
    const size_t dk = size_t(k) * sizeof(double);
    Layout lay;
    const size_t oOm = lay.add(size_t(m) * dk), oH = lay.add(size_t(m) * dk);
    const size_t oG = lay.add(size_t(n) * dk), oW = lay.add(size_t(n) * dk);
    const size_t oL1 = lay.add(size_t(m) * dk);
    const size_t oR = lay.add(size_t(k) * dk), oRi = lay.add(size_t(k) * dk);
    const size_t oS = lay.add(size_t(k) * dk);
    const size_t oU1T = lay.add(size_t(k) * dk), oU2T = lay.add(size_t(k) * dk);
    size_t step = 0, t = 0;
    for (int64_t w : {wc, n % wc}) {                // full panels and the last one
        if (w == 0) continue;
        t = pass_ws(w, k, m, prec, c->num_sms);
        if (t > step) step = t;
        t = pass_ws(m, k, w, prec, c->num_sms);
        if (t > step) step = t;
    }
    t = lu_scratch_bytes(m > n ? m : n, k);
    if (t > step) step = t;
    t = qr_scratch_bytes(n, k, c->num_sms, prec != PLU_FP64 ? 1 : 0);
    if (t > step) step = t;
    const size_t oStep = lay.add(step);
    size_t tp = gemm_f64_partials_bytes(n, k, k, c->num_sms);
    t = gemm_f64_partials_bytes(m, k, k, c->num_sms);
    if (t > tp) tp = t;
    t = gemm_f64_partials_bytes(k, k, k, c->num_sms);
    if (t > tp) tp = t;
    const size_t oTp = lay.add(tp);
    const size_t oInfo = lay.add(2 * sizeof(int32_t));
    // Omega in the tensor-core operand form, converted once for all panels
    const bool hoist = (is_tc(prec) || prec == kPrecSplit) && A->dtype == PLU_F32 && k <= 512;
    const size_t oXq =
        hoist ? lay.add(prec == kPrecSplit ? tcs_operand_bytes(m, k) : tc_operand_bytes(m, k)) : 0;
    PLU_TRY(ensure_ws(c, lay.total + 256));
    char* ws = c->ws;
    double* Om = reinterpret_cast<double*>(ws + oOm);
    const void* omq = hoist ? static_cast<const void*>(ws + oXq) : nullptr;
    double* H = reinterpret_cast<double*>(ws + oH);
    double* G = reinterpret_cast<double*>(ws + oG);
    double* Wb = reinterpret_cast<double*>(ws + oW);
    double* S = reinterpret_cast<double*>(ws + oS);
    double* L1 = reinterpret_cast<double*>(ws + oL1);
    double* R = reinterpret_cast<double*>(ws + oR);
    double* Rinv = reinterpret_cast<double*>(ws + oRi);
    double* U1T = reinterpret_cast<double*>(ws + oU1T);
    double* U2T = reinterpret_cast<double*>(ws + oU2T);
    char* stepp = ws + oStep;
    void* tpp = ws + oTp;
    int32_t* info = reinterpret_cast<int32_t*>(ws + oInfo);
    const long long launches0 = g_launches;
    PassTimer pt(c, rep != nullptr);
    if (rep) PLU_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    // Omega (m x k), Alg. singlepasslu step 1
    PLU_CUDA(c, launch_gaussian(m, k, seed, kStreamOmegaSP, Om, m, c->stream));
    if (hoist && prec == kPrecSplit)
        PLU_CUDA(c, launch_tcs_operand(m, k, Om, m, ws + oXq, c->num_sms, c->stream));
    else if (hoist)
        PLU_CUDA(c, launch_tc_operand(m, k, Om, m, ws + oXq, c->num_sms, c->stream));
    // G = A^T Omega and H = A G in one sweep over the columns of A (Sec. 5
    // remark): per column panel, G(panel, :) = A(:, panel)^T Omega, then
    // H += A(:, panel) G(panel, :) while the panel is still in L2
    pt.mark();
    for (int64_t j0 = 0; j0 < n; j0 += wc) {
        const int64_t w = (n - j0) < wc ? (n - j0) : wc;
        plu_matrix Ap = *A;
        Ap.n = w;
        Ap.data = static_cast<const char*>(A->data) + size_t(j0) * size_t(A->ld) * size_t(es);
        PLU_TRY(do_pass(c, &Ap, 1, Om, m, k, prec, G + j0, n, stepp, step, nullptr, 0, omq));
        PLU_TRY(do_pass(c, &Ap, 0, G + j0, n, k, prec, H, m, stepp, step, nullptr,
                        j0 > 0 ? 1 : 0));
    }
    pt.mark();
    // [L1, U1, P] = lu(H)
    PLU_CUDA(c, launch_lu(c, prec, m, k, H, m, 1, p, L1, m, 0, U1T, k, 1, info, stepp, c->d_status,
                                c->spin_budget, c->num_sms, c->stream));
    // G^{dagger T} = G (G^T G)^{-1} = Q1 R^{-T} with one CholeskyQR round,
    // G = Q1 R and R^T R = G^T G (in place: G becomes Q1)
    PLU_CUDA(c, launch_cholqr2(n, k, G, n, R, k, stepp, step, c->d_status, c->num_sms, c->stream,
                               0, 1, prec != PLU_FP64 ? 1 : 0));
    PLU_CUDA(c, launch_trinv_upper(k, R, Rinv, c->stream));
    // M = G^{dagger T} U1^T = Q1 S with S = R^{-T} U1^T (k x k, lower
    // triangular); the two m x k x k products take FP32 FMAs when the passes
    // are not FP64 (G and H carry the pass precision's rounding)
    PLU_CUDA(c, launch_gemm_f64(1, 0, k, k, k, Rinv, k, U1T, k, S, k, tpp, tp, c->num_sms,
                                c->stream));
    const bool f32 = prec != PLU_FP64;
    if (f32)
        PLU_CUDA(c, launch_gemm_f32_tri(3, n, k, k, G, n, S, k, Wb, n, tpp, tp, c->num_sms,
                                        c->stream));
    else
        PLU_CUDA(c, launch_gemm_f64_tri(0, 3, n, k, k, G, n, S, k, Wb, n, tpp, tp, c->num_sms,
                                        c->stream));
    // [L2, U2, Q] = lu(M), U = L2^T
    PLU_CUDA(c, launch_lu(c, prec, n, k, Wb, n, 1, q, U, ldU, 1, U2T, k, 1, info + 1, stepp,
                                c->d_status, c->spin_budget, c->num_sms, c->stream));
    // L = L1 U2^T (U2^T lower triangular)
    if (f32)
        PLU_CUDA(c, launch_gemm_f32_tri(3, m, k, k, L1, m, U2T, k, L, ldL, tpp, tp, c->num_sms,
                                        c->stream));
    else
        PLU_CUDA(c, launch_gemm_f64_tri(0, 3, m, k, k, L1, m, U2T, k, L, ldL, tpp, tp,
                                        c->num_sms, c->stream));
    if (rep) {
        PLU_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
        int32_t hinfo[2] = {0, 0};
        PLU_CUDA(c, cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        memset(rep, 0, sizeof(*rep));
        rep->ms_total = ms;
        rep->ms_passes = pt.pairs_ms();
        rep->passes = 1;
        rep->rank = k;
        rep->indicator = -1.0;
        rep->normA2 = -1.0;
        rep->info1 = hinfo[0];
        rep->info2 = hinfo[1];
        const double mnd = double(m) * double(n);
        rep->flops_passes = 4.0 * mnd * k;
        rep->bytes_passes = mnd * double(es) + double(m + n) * k * 8.0;
        rep->launches = int32_t(g_launches - launches0);
    }
    return finish(c);
}

plu_status plu_randlu(plu_ctx* c, const plu_matrix* A, int k, int l, int piter, uint64_t seed,
                      plu_prec prec, int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                      int64_t ldU, plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_matrix(c, A));
    PLU_TRY(check_prec(c, prec, A));
    const int64_t m = A->m, n = A->n;
    const int64_t mn = m < n ? m : n;
    if (k < 1 || l < k || l >= mn) return fail(c, PLU_EINVAL, "need 1 <= k <= l < min(m, n)");
    if (piter < 0) return fail(c, PLU_EINVAL, "need piter >= 0");
    if (l > 2048) return fail(c, PLU_EINVAL, "l > 2048 is not supported");
    if (!p || !q || !L || !U || ldL < m || ldU < k) return fail(c, PLU_EINVAL, "bad outputs");
    const int sms = c->num_sms;
    Layout lay;
    const size_t oX = lay.add(size_t(n) * l * sizeof(double));
    const size_t oY = lay.add(size_t(m) * l * sizeof(double));
    const size_t oL1 = lay.add(size_t(m) * l * sizeof(double));
    const size_t oUl = lay.add(size_t(l) * l * sizeof(double));
    const size_t oW = lay.add(size_t(m) * k * sizeof(double));
    const size_t oR = lay.add(size_t(k) * k * sizeof(double));
    const size_t oRi = lay.add(size_t(k) * k * sizeof(double));
    const size_t oT = lay.add(size_t(n) * k * sizeof(double));
    const size_t oBT = lay.add(size_t(n) * k * sizeof(double));
    const size_t oU2T = lay.add(size_t(k) * k * sizeof(double));
    size_t step = pass_ws(m, l, n, prec, sms), t;
    t = pass_ws(n, l, m, prec, sms);
    if (t > step) step = t;
    t = pass_ws(n, k, m, is_tc(prec) ? kPrecSplit : int(prec), sms);
    if (t > step) step = t;
    t = pass_ws(n, k, m, prec, sms);
    if (t > step) step = t;
    t = lu_scratch_bytes(m > n ? m : n, l);
    if (t > step) step = t;
    t = qr_scratch_bytes(m, k, sms, prec != PLU_FP64 ? 1 : 0);
    if (t > step) step = t;
    const size_t oStep = lay.add(step);
    size_t tp = gemm_f64_partials_bytes(n, k, k, sms);
    t = gemm_f64_partials_bytes(m, k, k, sms);
    if (t > tp) tp = t;
    const size_t oTp = lay.add(tp);
    const size_t oInfo = lay.add(2 * sizeof(int32_t));
    const bool quant = prec == PLU_BF16 || prec == PLU_FP8_E4M3;
    const size_t oQ = quant ? lay.add(tc_quant_bytes(m, n, prec)) : 0;
    PLU_TRY(ensure_ws(c, lay.total + 256));
    char* ws = c->ws;
    double* X = reinterpret_cast<double*>(ws + oX);
    double* Y = reinterpret_cast<double*>(ws + oY);
    double* L1 = reinterpret_cast<double*>(ws + oL1);
    double* Ul = reinterpret_cast<double*>(ws + oUl);
    double* W = reinterpret_cast<double*>(ws + oW);
    double* R = reinterpret_cast<double*>(ws + oR);
    double* Rinv = reinterpret_cast<double*>(ws + oRi);
    double* T = reinterpret_cast<double*>(ws + oT);
    double* BT = reinterpret_cast<double*>(ws + oBT);
    double* U2T = reinterpret_cast<double*>(ws + oU2T);
    char* stepp = ws + oStep;
    void* tpp = ws + oTp;
    int32_t* info = reinterpret_cast<int32_t*>(ws + oInfo);
    PassTimer pt(c, rep != nullptr);
    const long long launches0 = g_launches;
    if (rep) PLU_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    QuantA qa;
    if (quant)
        PLU_CUDA(c, launch_tc_quantize(prec, static_cast<const float*>(A->data), m, n, A->ld,
                                       ws + oQ, &qa, sms, c->stream));
    int np = 0;
    auto pass = [&](int trans, const double* Xin, int64_t ldx, int cols, int pr, double* Yout,
                    int64_t ldy) -> plu_status {
        pt.mark();
        PLU_TRY(do_pass(c, A, trans, Xin, ldx, cols, pr, Yout, ldy, stepp, step,
                        quant && pr == int(prec) ? &qa : nullptr));
        pt.mark();
        ++np;
        return PLU_OK;
    };
    auto reorth = [&](int64_t rows, double* Xr) -> plu_status {
        PLU_CUDA(c, launch_lu(c, prec, rows, l, Xr, rows, 0, nullptr, nullptr, 0, 0, nullptr, 0, 0,
                                    nullptr, stepp, c->d_status, c->spin_budget, sms, c->stream));
        return PLU_OK;
    };
    // Alg. basicpoweriteration: Y = A Omega, then piter rounds of A^T, A
    PLU_CUDA(c, launch_gaussian(n, l, seed, kStreamOmegaN, X, n, c->stream));
    PLU_TRY(pass(0, X, n, l, prec, Y, m));
    if (piter > 0) PLU_TRY(reorth(m, Y));
    for (int i = 1; i <= piter; ++i) {
        PLU_TRY(pass(1, Y, m, l, prec, X, n));
        PLU_TRY(reorth(n, X));
        PLU_TRY(pass(0, X, n, l, prec, Y, m));
        if (i < piter) PLU_TRY(reorth(m, Y));
    }
    // P Y = L_y U_y (full LU of the m x l product); L_y = its first k columns
    PLU_CUDA(c, launch_lu(c, prec, m, l, Y, m, 1, p, L1, m, 0, Ul, l, 1, info, stepp, c->d_status,
                                c->spin_budget, sms, c->stream));
    // B^T = (L_y^+ P A)^T = A^T W (W^T W)^{-1} with W = P^T L_y = Q R:
    // B^T = A^T Q R^{-T}.  The pass reads the FP32 A with FP32-accurate
    // split products in the mixed modes (B enters the result to first order).
    PLU_CUDA(c, launch_scatter_rows(m, k, p, L1, m, W, m, c->stream));
    PLU_CUDA(c, launch_cholqr2(m, k, W, m, R, k, stepp, step, c->d_status, sms, c->stream, 0, 2,
                               prec != PLU_FP64 ? 1 : 0));
    PLU_TRY(pass(1, W, m, k, is_tc(prec) ? kPrecSplit : int(prec), T, n));
    PLU_CUDA(c, launch_trinv_upper(k, R, Rinv, c->stream));
    PLU_CUDA(c, launch_gemm_f64(0, 1, n, k, k, T, n, Rinv, k, BT, n, tpp, tp, sms, c->stream));
    // Q B^T = L' U' (Alg. rlu step 5); U = L'^T written straight into U
    PLU_CUDA(c, launch_lu(c, prec, n, k, BT, n, 1, q, U, ldU, 1, U2T, k, 1, info + 1, stepp,
                                c->d_status, c->spin_budget, sms, c->stream));
    // L = L_y U'^T (U'^T lower triangular)
    if (prec != PLU_FP64)
        PLU_CUDA(c, launch_gemm_f32_tri(3, m, k, k, L1, m, U2T, k, L, ldL, tpp, tp, sms,
                                        c->stream));
    else
        PLU_CUDA(c, launch_gemm_f64_tri(0, 3, m, k, k, L1, m, U2T, k, L, ldL, tpp, tp, sms,
                                        c->stream));
    if (rep) {
        PLU_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
        int32_t hinfo[2] = {0, 0};
        PLU_CUDA(c, cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, c->stream));
        PLU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        memset(rep, 0, sizeof(*rep));
        rep->ms_total = ms;
        rep->ms_passes = pt.pairs_ms();
        rep->passes = np;
        rep->rank = k;
        rep->indicator = -1.0;
        rep->normA2 = -1.0;
        rep->info1 = hinfo[0];
        rep->info2 = hinfo[1];
        fill_pass_report(rep, A, np - 1, l, k, prec, true, c->csr);
        rep->launches = int32_t(g_launches - launches0);
    }
    return finish(c);
}

plu_status plu_set_batched_tile(plu_ctx* c, int bm, int bn) {
    if (!c) return PLU_EINVAL;
    if (bm == 0 && bn == 0) {
        c->forced_tile = -1;
        return PLU_OK;
    }
    for (int v = 0;; ++v) {
        int tm = 0, tn = 0;
        if (!batch_gemm_tile(v, &tm, &tn)) break;
        if (tm == bm && tn == bn) {
            c->forced_tile = v;
            return PLU_OK;
        }
    }
    return fail(c, PLU_EINVAL, "no grouped-GEMM tile shape %d x %d", bm, bn);
}

plu_status plu_batched_splitk(plu_ctx* c, int* kchunk, int cap, int* count) {
    if (!c || !count || cap < 0 || (cap > 0 && !kchunk)) return fail(c, PLU_EINVAL, "bad arguments");
    const int n = int(c->last_tiles.size());
    *count = n;
    for (int i = 0; i < n && i < cap; ++i) {
        kchunk[i] = batch_gemm_splitk(c->last_tiles[i]);
        if (kchunk[i] < 0) return fail(c, PLU_EINVAL, "bad choice index");
    }
    return PLU_OK;
}

plu_status plu_set_batched_tune_file(plu_ctx* c, const char* path) {
    if (!c) return PLU_EINVAL;
    if (!path || !*path) {
        c->tune_file.clear();
        return PLU_OK;
    }
    FILE* f = fopen(path, "a");
    if (!f) return fail(c, PLU_EINVAL, "cannot open the tuning file %s for appending", path);
    fclose(f);
    c->tune_file = path;
    return PLU_OK;
}

namespace {
// The autotuner's file: one line per batch signature,
//   plu-batched-tune 1 <signature, 16 hex digits> <launches> <choice> ...
// the last line of a signature wins; malformed lines are ignored.
bool load_tuned(const std::string& path, uint64_t sig, std::vector<int>* out) {
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[8192];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        unsigned long long fsig = 0;
        int ver = 0, n = 0, used = 0;
        if (sscanf(line, "plu-batched-tune %d %llx %d%n", &ver, &fsig, &n, &used) != 3) continue;
        if (ver != 1 || fsig != sig || n < 1 || n > 4096) continue;
        std::vector<int> v;
        const char* p = line + used;
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            int x = 0, u = 0;
            if (sscanf(p, "%d%n", &x, &u) != 1 || x < 0 || x >= batch_gemm_choices()) ok = false;
            else {
                v.push_back(x);
                p += u;
            }
        }
        if (ok) {
            *out = v;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void save_tuned(const std::string& path, uint64_t sig, const std::vector<int>& v) {
    std::string line;
    char buf[64];
    snprintf(buf, sizeof(buf), "plu-batched-tune 1 %016llx %d", (unsigned long long)sig,
             int(v.size()));
    line = buf;
    for (int x : v) {
        snprintf(buf, sizeof(buf), " %d", x);
        line += buf;
    }
    line += "\n";
    FILE* f = fopen(path.c_str(), "a");
    if (!f) return;
    fputs(line.c_str(), f);                 // one write per line
    fclose(f);
}
}  // namespace

plu_status plu_batched_tiles(plu_ctx* c, int* bm, int* bn, int cap, int* count) {
    if (!c || !count || cap < 0 || (cap > 0 && (!bm || !bn))) return fail(c, PLU_EINVAL, "bad arguments");
    const int n = int(c->last_tiles.size());
    *count = n;
    for (int i = 0; i < n && i < cap; ++i)
        if (!batch_gemm_tile(c->last_tiles[i], bm + i, bn + i))
            return fail(c, PLU_EINVAL, "bad tile index");
    return PLU_OK;
}

plu_status plu_batched(plu_ctx* c, const plu_batch_problem* P, int count, plu_prec prec,
                       plu_report* rep) {
    PLU_TRY(bind(c));
    if (!P || count < 1) return fail(c, PLU_EINVAL, "need at least one problem");
    if (prec != PLU_FP64 && prec != PLU_FP32)
        return fail(c, PLU_EUNSUPPORTED, "batched passes take PLU_FP64 or PLU_FP32");
    double flops = 0.0, bytes = 0.0;
    int passes = 0;
    for (int i = 0; i < count; ++i) {
        const plu_batch_problem& p = P[i];
        const int64_t mn = p.m < p.n ? p.m : p.n;
        if (!p.A || p.m < 2 || p.n < 2 || p.ld < p.m || (p.dtype != PLU_F32 && p.dtype != PLU_F64))
            return fail(c, PLU_EINVAL, "problem %d: bad matrix", i);
        if (p.m > (1 << 30) || p.n > (1 << 30)) return fail(c, PLU_EINVAL, "problem %d: too large", i);
        if (p.algo == 0) {
            if (p.k < 1 || p.l < p.k || p.l >= mn || p.v < 2 || p.l > 1024)
                return fail(c, PLU_EINVAL, "problem %d: need 1 <= k <= l < min(m, n), l <= 1024, v >= 2", i);
            passes += p.v;
            flops += 2.0 * double(p.m) * double(p.n) * (double(p.l) * (p.v - 1) + p.k);
            bytes += double(p.m) * double(p.n) * (p.dtype == PLU_F32 ? 4.0 : 8.0) * p.v;
        } else if (p.algo == 1) {
            if (p.k < 1 || p.k >= mn || p.k > 1024)
                return fail(c, PLU_EINVAL, "problem %d: need 1 <= k < min(m, n), k <= 1024", i);
            passes += 1;
            flops += 4.0 * double(p.m) * double(p.n) * p.k;
            bytes += double(p.m) * double(p.n) * (p.dtype == PLU_F32 ? 4.0 : 8.0);
        } else {
            return fail(c, PLU_EINVAL, "problem %d: algo must be 0 or 1", i);
        }
        if (!p.p || !p.q || !p.L || !p.U || p.ldL < p.m || p.ldU < p.k)
            return fail(c, PLU_EINVAL, "problem %d: bad outputs", i);
    }
    if (!c->capture) PLU_CUDA(c, cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    const size_t wsb = (batch_workspace_bytes(P, count) + 255) & ~size_t(255);
    const size_t tb = batch_tables_bytes(count);
    PLU_TRY(ensure_ws(c, wsb + tb));
    // the capture stream must see the work already queued on the context stream
    PLU_CUDA(c, cudaStreamSynchronize(c->stream));
    // the batch's signature (FNV-1a over the shapes that decide the plan)
    uint64_t sig = 1469598103934665603ULL;
    auto mix = [&](int64_t x) {
        for (int b = 0; b < 8; ++b) {
            sig ^= uint64_t(x >> (8 * b)) & 0xFF;
            sig *= 1099511628211ULL;
        }
    };
    mix(count);
    mix(prec);
    for (int i = 0; i < count; ++i) {
        mix(P[i].m); mix(P[i].n); mix(P[i].k); mix(P[i].l); mix(P[i].v); mix(P[i].algo);
        mix(P[i].dtype); mix(P[i].ld);
    }
    std::vector<int> forced;
    std::vector<int>& tiles = c->forced_tile >= 0 ? forced : c->batch_tiles[sig];
    // a signature not tuned in this context may have been tuned before (the file)
    const bool fresh = c->forced_tile < 0 && tiles.empty();
    bool loaded = false;
    if (fresh && !c->tune_file.empty()) loaded = load_tuned(c->tune_file, sig, &tiles);
    int nl = 0;
    float ms = 0.f;
    const size_t before = tiles.size();
    PLU_CUDA(c, run_batch(P, count, prec, c->ws, c->ws + wsb, tb, c->d_status, c->num_sms, c->stream,
                          c->capture, &nl, &ms, &tiles, c->forced_tile, &c->bpart, &c->bpart_cap));
    // save what the autotuner chose (a loaded entry of the wrong length was retuned)
    if (fresh && !c->tune_file.empty() && (!loaded || tiles.size() != before))
        save_tuned(c->tune_file, sig, tiles);
    c->last_tiles = tiles;
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        rep->ms_total = ms;
        rep->ms_passes = -1.0;
        rep->passes = passes;
        rep->rank = -1;
        rep->indicator = -1.0;
        rep->normA2 = -1.0;
        rep->flops_passes = flops;
        rep->bytes_passes = bytes;
        rep->launches = nl;
    }
    return finish(c);
}

plu_status plu_spmm(plu_ctx* c, const plu_csr* A, int trans, const double* X, int64_t ldx,
                    int cols, double* Y, int64_t ldy) {
    PLU_TRY(bind(c));
    PLU_TRY(check_csr(c, A));
    const int64_t M = trans ? A->n : A->m;
    const int64_t K = trans ? A->m : A->n;
    if (cols < 1 || !X || !Y || ldx < K || ldy < M) return fail(c, PLU_EINVAL, "bad spmm operands");
    const size_t sw = spmm_scratch_bytes(K, cols);
    PLU_TRY(ensure_ws(c, sw));
    CsrScope scope(c, A);
    PLU_TRY(do_pass(c, &scope.shape, trans, X, ldx, cols, PLU_FP64, Y, ldy, c->ws, sw));
    return finish(c);
}

plu_status plu_powerlu_csr(plu_ctx* c, const plu_csr* A, int k, int l, int v, uint64_t seed,
                           int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                           int64_t ldU, plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_csr(c, A));
    CsrScope scope(c, A);
    return plu_powerlu(c, &scope.shape, k, l, v, seed, PLU_FP64, p, q, L, ldL, U, ldU, rep);
}

plu_status plu_powerlu_fp_csr(plu_ctx* c, const plu_csr* A, double eps, int b, int l, int v,
                              int precise, int max_rounds, uint64_t seed, int* k_out,
                              int32_t* p, int32_t* q, double* L, int64_t ldL, double* U,
                              int64_t ldU, plu_report* rep) {
    PLU_TRY(bind(c));
    PLU_TRY(check_csr(c, A));
    CsrScope scope(c, A);
    return powerlu_fp_rounds(c, &scope.shape, eps, b, l, v, precise, max_rounds, seed, PLU_FP64,
                             k_out, p, q, L, ldL, U, ldU, rep);
}

}  // extern "C"
