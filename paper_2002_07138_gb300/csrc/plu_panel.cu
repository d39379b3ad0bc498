// Partial-pivoting LU of a tall-skinny FP64 panel (rows x cols, rows >= cols):
// the re-orthogonalising [X, ~] = lu(X) of Alg. gpowerlu (a3) and the
// [L, U, P] = lu(Y) / lu(B^T) of Alg. bpowerlu steps 4 and 6 (a8).
//
// One cooperative (co-resident) grid; CTA b owns a contiguous block of rows
// and keeps them in place ("virtual" pivoting: rows never move).  Column j:
//   1. each CTA finds the largest |x_ij| among its not-yet-pivoted rows,
//      ties going to the row with the smallest current position, and
//      publishes (|x|, position, row) -- warp shuffles, then shared memory;
//   2. grid barrier (one per column; bounded spin, error word on timeout);
//   3. every CTA reduces the published candidates to the same pivot row r,
//      applies LAPACK's row interchange to the positions of its own rows
//      (r takes position j, the row at position j takes r's old position),
//      stages row r's columns j.. in shared memory, and eliminates:
//      l_ij = x_ij (1 / u_jj) (LAPACK's scaling; x_ij / u_jj when u_jj is
//      subnormal), x_ic -= l_ij u_jc for its other active rows, and
//      computes its candidate for column j+1 in the same sweep.
// A column whose candidates are all exactly zero is skipped (no division),
// as LAPACK does; the first such column is reported in `info`.
// The tie rule reproduces LAPACK's idamax on the row-swapped matrix: the
// first maximum in the current row order.
//
// After the sweep each row holds its multipliers left of its pivot step and,
// for pivot rows, the U row from the pivot step on.  A finalising kernel
// writes either P^T L in place (a3) or perm, L (pivoted order) and U (a8).
//
// Blocked variant (used whenever a CTA's rows fit in shared memory): the
// columns are taken NB = 32 at a time.  Each CTA keeps its rows of the
// current NB-column block in shared memory, so a column step touches no
// global memory except the candidate slots: each CTA publishes its candidate
// with its whole NB-wide block row;
// after a grid barrier every CTA reads all candidates at once, picks the
// winner and copies its block row, then eliminates in shared memory.  After the block, every CTA forms
// U12 = L11^{-1} A12 for the block's pivot rows (forward substitution) and
// applies the FP64 trailing update X(:, J2) -= L(:, J1) U12 to its own rows.
// The U rows go to a separate buffer, so no CTA overwrites data that
// another one still reads.
#include "plu_internal.h"

#include <climits>
#include <cstddef>

namespace plu {

struct Cand {
    double v;
    int pos;
    int row;
};

struct PanelScratch {
    unsigned int barrier;
    int info;
    int any_nan;
    int pad;
    Cand cand[2][kMaxGrid];
};
static_assert(offsetof(PanelScratch, info) == offsetof(PanelHead, info) &&
                  offsetof(PanelScratch, any_nan) == offsetof(PanelHead, any_nan),
              "PanelScratch starts with a PanelHead");

namespace {

constexpr int NT = 256;
constexpr int kMaxCols = 2048;

// Candidate values are |x| (sign bit clear), so their IEEE bit patterns order
// as 64-bit integers and NaNs are exactly the patterns above +inf's: the
// comparisons run on the integer pipe instead of the narrow FP64 pipe.
__device__ __forceinline__ bool is_nan_abs(double a) {
    return __double_as_longlong(a) > 0x7FF0000000000000LL;
}

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
    // true when a should be the pivot rather than b: larger |x| first, then
    // the smaller current position; NaN loses to every number
    if (a.row < 0) return false;
    if (b.row < 0) return true;
    const long long ab = __double_as_longlong(a.v), bb = __double_as_longlong(b.v);
    const bool an = ab > 0x7FF0000000000000LL, bn = bb > 0x7FF0000000000000LL;
    if (an || bn) return an && bn ? a.pos < b.pos : bn;
    if (ab > bb) return true;
    if (ab < bb) return false;
    return a.pos < b.pos;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src_lane_xor) {
    Cand o;
    o.v = __shfl_xor_sync(0xffffffffu, c.v, src_lane_xor);
    o.pos = __shfl_xor_sync(0xffffffffu, c.pos, src_lane_xor);
    o.row = __shfl_xor_sync(0xffffffffu, c.row, src_lane_xor);
    return o;
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Cand o = shfl_cand(c, off);
        if (better(o, c)) c = o;
    }
    return c;
}

__device__ Cand block_best(Cand c, Cand* red) {
    c = warp_best(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (warp == 0) {
        Cand x = (lane < NT / 32) ? red[lane] : Cand{-1.0, INT_MAX, -1};
        x = warp_best(x);
        if (lane == 0) red[0] = x;
    }
    __syncthreads();
    const Cand out = red[0];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(NT)
k_panel_lu(int64_t rows, int cols, double* __restrict__ X, int64_t ldx,
           PanelScratch* __restrict__ ps, int* __restrict__ pos, int* __restrict__ pivstep,
           int* __restrict__ status, int64_t budget) {
    extern __shared__ double urow[];
    __shared__ Cand red[NT / 32];
    __shared__ Cand piv;
    const int nb = gridDim.x;
    const int t = threadIdx.x;
    const int64_t per = (rows + nb - 1) / nb;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = min(rows, r0 + per);
    const int steps = int(rows < int64_t(cols) ? rows : int64_t(cols));

    // own rows start unpivoted at their natural position; candidate for column 0
    Cand best{-1.0, INT_MAX, -1};
    for (int64_t i = r0 + t; i < r1; i += NT) {
        pos[i] = int(i);
        pivstep[i] = -1;
        const double a = fabs(X[i]);
        const Cand c{a, int(i), int(i)};
        if (better(c, best)) best = c;
    }

    for (int j = 0; j < steps; ++j) {
        const Cand cb = block_best(best, red);
        if (t == 0) ps->cand[j & 1][blockIdx.x] = cb;
        if (!grid_barrier(&ps->barrier, unsigned(j + 1) * unsigned(nb), status, budget)) return;
        if (t < 32) {
            Cand g{-1.0, INT_MAX, -1};
            for (int b = t; b < nb; b += 32) {
                const Cand* src = &ps->cand[j & 1][b];
                Cand c;
                c.v = __ldcg(&src->v);
                c.pos = __ldcg(&src->pos);
                c.row = __ldcg(&src->row);
                if (better(c, g)) g = c;
            }
            g = warp_best(g);
            if (t == 0) piv = g;
        }
        __syncthreads();
        const Cand pv = piv;
        if (pv.row < 0) {                    // no comparable candidate (NaN panel)
            if (blockIdx.x == 0 && t == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
            return;
        }
        // LAPACK interchange on the positions of own rows; retire the pivot row
        for (int64_t i = r0 + t; i < r1; i += NT) {
            if (i == pv.row) {
                pos[i] = j;
                pivstep[i] = j;
            } else if (pos[i] == j) {
                pos[i] = pv.pos;
            }
        }
        for (int c = j + t; c < cols; c += NT) urow[c] = __ldcg(&X[pv.row + int64_t(c) * ldx]);
        if (blockIdx.x == 0 && t == 0) {
            if (pv.v == 0.0 && ps->info == 0) ps->info = j + 1;
            if (!(pv.v <= 1.7976931348623157e308)) ps->any_nan = 1;   // pivot inf or NaN
        }
        __syncthreads();
        const double ujj = urow[j];
        const double rinv = 1.0 / ujj;
        best = Cand{-1.0, INT_MAX, -1};
        const bool next = j + 1 < steps;
        for (int64_t i = r0 + t; i < r1; i += NT) {
            if (pivstep[i] >= 0) continue;
            double* xi = X + i;
            if (ujj != 0.0) {
                const double lij = lu_multiplier(xi[int64_t(j) * ldx], ujj, rinv);
                xi[int64_t(j) * ldx] = lij;
                for (int c = j + 1; c < cols; ++c) {
                    double* p = xi + int64_t(c) * ldx;
                    *p = fma(-lij, urow[c], *p);
                }
            }
            if (next) {
                const Cand c{fabs(xi[int64_t(j + 1) * ldx]), pos[i], int(i)};
                if (better(c, best)) best = c;
            }
        }
        __syncthreads();
    }
}

constexpr int NB = 32;      // columns per block
constexpr int UC = 128;     // trailing columns per U12 chunk

// smem: P[NB][per] | U12[NB][UC] | PR[NB][NB] | pos_s[per] | piv_s[per] | prow_id[NB]
__global__ void __launch_bounds__(NT)
k_panel_lu_blocked(int64_t rows, int cols, double* __restrict__ X, int64_t ldx,
                   PanelScratch* __restrict__ ps, double* __restrict__ slots,
                   double* __restrict__ Ubuf, int* __restrict__ pos_g, int* __restrict__ piv_g,
                   int* __restrict__ status, int64_t budget, int per) {
    extern __shared__ double dsm[];
    double* P = dsm;
    double* U12 = P + NB * per;
    double* PR = U12 + NB * UC;
    int* pos_s = reinterpret_cast<int*>(PR + NB * NB);
    int* piv_s = pos_s + per;
    int* prow_id = piv_s + per;
    __shared__ Cand red[NT / 32];
    __shared__ Cand piv;
    __shared__ int win_slot;
    __shared__ int nan_seen;

    const int nb = gridDim.x;
    const int t = threadIdx.x;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = min(rows, r0 + per);
    const int R = int(r1 > r0 ? r1 - r0 : 0);
    const int steps = int(rows < int64_t(cols) ? rows : int64_t(cols));
    // slot: [0] |x|, [1] (pos, row), [2] unused, [3..] block row
    const int slot_w = NB + 3;

    for (int r = t; r < R; r += NT) {
        pos_s[r] = int(r0 + r);
        piv_s[r] = -1;
    }
    if (t == 0) nan_seen = 0;
    __syncthreads();

    for (int j0 = 0; j0 < steps; j0 += NB) {
        const int nbk = min(NB, steps - j0);
        for (int e = t; e < nbk * R; e += NT) {
            const int r = e % R, c = e / R;
            P[c * per + r] = X[(r0 + r) + int64_t(j0 + c) * ldx];
        }
        __syncthreads();
        // candidate of the block's first column; later columns get theirs from
        // the elimination loop of the step before
        Cand best{-1.0, INT_MAX, -1};
        for (int r = t; r < R; r += NT) {
            if (piv_s[r] >= 0) continue;
            const double a = fabs(P[r]);
            if (is_nan_abs(a)) nan_seen = 1;
            const Cand c{a, pos_s[r], int(r0 + r)};
            if (better(c, best)) best = c;
        }
        for (int sc = 0; sc < nbk; ++sc) {
            const int j = j0 + sc;
            const Cand cb = block_best(best, red);
            double* myslot = slots + (int64_t(j & 1) * nb + blockIdx.x) * slot_w;
            if (t == 0) {
                myslot[0] = cb.v;
                int2 pr;
                pr.x = cb.pos;
                pr.y = cb.row;
                reinterpret_cast<int2*>(myslot + 1)[0] = pr;
            }
            if (t < nbk && cb.row >= 0) myslot[3 + t] = P[t * per + int(cb.row - r0)];
            // grid barrier (one arrival counter: polled by one thread per CTA,
            // much cheaper than polling every CTA's slot), then warp 0 reads all
            // slots (a few per lane, in one round trip) and reduces them
            if (!grid_barrier(&ps->barrier, unsigned(j + 1) * unsigned(nb), status, budget)) return;
            if (t < 32) {
                Cand g{-1.0, INT_MAX, -1};
                int gs = -1;
                // eight slots per lane per round: all loads first, so they are in
                // flight together, then the comparisons
                for (int b0 = 0; b0 < nb; b0 += 256) {
                    double v[8];
                    int2 pr[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int b = b0 + t + 32 * k;
                        if (b < nb) {
                            const double* src = slots + (int64_t(j & 1) * nb + b) * slot_w;
                            v[k] = __ldcg(src);
                            pr[k] = __ldcg(reinterpret_cast<const int2*>(src + 1));
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int b = b0 + t + 32 * k;
                        if (b < nb) {
                            const Cand c{v[k], pr[k].x, pr[k].y};
                            if (better(c, g)) { g = c; gs = b; }
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const Cand o = shfl_cand(g, off);
                    const int os = __shfl_xor_sync(0xffffffffu, gs, off);
                    if (better(o, g)) { g = o; gs = os; }
                }
                if (t == 0) {
                    piv = g;
                    win_slot = gs;
                }
            }
            __syncthreads();
            const Cand pv = piv;
            if (pv.row < 0) {
                if (blockIdx.x == 0 && t == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
                return;
            }
            const double* wsrc = slots + (int64_t(j & 1) * nb + win_slot) * slot_w;
            if (t < nbk) PR[sc * NB + t] = __ldcg(wsrc + 3 + t);
            if (t == 0) prow_id[sc] = pv.row;
            for (int r = t; r < R; r += NT) {
                if (r0 + r == pv.row) {
                    pos_s[r] = j;
                    piv_s[r] = j;
                } else if (pos_s[r] == j) {
                    pos_s[r] = pv.pos;
                }
            }
            if (blockIdx.x == 0 && t == 0) {
                if (pv.v == 0.0 && ps->info == 0) ps->info = j + 1;
                if (!(pv.v <= 1.7976931348623157e308)) ps->any_nan = 1;
            }
            __syncthreads();
            // eliminate column sc from the own active rows of the block and,
            // in the same sweep, find the candidate for column sc + 1
            const double ujj = PR[sc * NB + sc];
            const double rinv = 1.0 / ujj;
            const bool next = sc + 1 < nbk;
            best = Cand{-1.0, INT_MAX, -1};
            for (int r = t; r < R; r += NT) {
                if (piv_s[r] >= 0) continue;
                if (ujj != 0.0) {
                    const double l = lu_multiplier(P[sc * per + r], ujj, rinv);
                    P[sc * per + r] = l;
                    for (int u = sc + 1; u < nbk; ++u)
                        P[u * per + r] = fma(-l, PR[sc * NB + u], P[u * per + r]);
                }
                if (next) {
                    const double a = fabs(P[(sc + 1) * per + r]);
                    if (is_nan_abs(a)) nan_seen = 1;
                    const Cand c{a, pos_s[r], int(r0 + r)};
                    if (better(c, best)) best = c;
                }
            }
        }
        __syncthreads();
        // block columns of own rows back to X (multipliers; pivot rows keep U11)
        for (int e = t; e < nbk * R; e += NT) {
            const int r = e % R, c = e / R;
            X[(r0 + r) + int64_t(j0 + c) * ldx] = P[c * per + r];
        }
        // U11 rows to the U buffer (CTA 0)
        if (blockIdx.x == 0) {
            for (int e = t; e < nbk * nbk; e += NT) {
                const int sr = e % nbk, c = e / nbk;
                if (c >= sr) Ubuf[(j0 + sr) + int64_t(j0 + c) * steps] = PR[sr * NB + c];
            }
        }
        // trailing columns, UC at a time
        for (int c0 = j0 + nbk; c0 < cols; c0 += UC) {
            const int cw = min(UC, cols - c0);
            __syncthreads();
            // U12 = L11^{-1} A12 over this chunk (every CTA, redundantly)
            for (int c = t; c < cw; c += NT) {
                for (int sr = 0; sr < nbk; ++sr) {
                    double acc = __ldcg(&X[prow_id[sr] + int64_t(c0 + c) * ldx]);
                    for (int u = 0; u < sr; ++u) acc = fma(-PR[sr * NB + u], U12[u * UC + c], acc);
                    U12[sr * UC + c] = acc;
                }
            }
            __syncthreads();
            if (blockIdx.x == 0) {
                for (int e = t; e < nbk * cw; e += NT) {
                    const int sr = e % nbk, c = e / nbk;
                    Ubuf[(j0 + sr) + int64_t(c0 + c) * steps] = U12[sr * UC + c];
                }
            }
            // X(own active rows, chunk) -= L(:, block) U12
            for (int e = t; e < R * cw; e += NT) {
                const int r = e % R, c = e / R;
                if (piv_s[r] >= 0) continue;
                double acc = 0.0;
                for (int u = 0; u < nbk; ++u) acc = fma(P[u * per + r], U12[u * UC + c], acc);
                double* xp = &X[(r0 + r) + int64_t(c0 + c) * ldx];
                *xp -= acc;
            }
        }
        __syncthreads();
    }
    for (int r = t; r < R; r += NT) {
        pos_g[r0 + r] = pos_s[r];
        piv_g[r0 + r] = piv_s[r];
    }
    if (nan_seen) atomicExch(&ps->any_nan, 1);
}

// Look-ahead variant of the blocked panel LU.  The column steps of a block
// are latency-bound (a grid barrier and a candidate exchange each), the
// trailing update is bound by the FP64 pipe; here they overlap.  Warps 0-3
// (the panel group) factor block b while warps 4-7 (the update group) apply
// block b-1's update to the columns beyond block b.  Block b's own columns
// received block b-1's update first (the catch-up, all warps, before its
// steps).  After the steps a grid barrier makes every CTA's deferred update
// visible, then every CTA forms U12 = L11^{-1} A12 of block b for all
// trailing columns.  Every number is produced by the same FP64 operations in
// the same order as in the non-overlapped kernel; only their timing moves.
// Rows pivoted in block b still receive block b-1's update (their pivot step
// is >= the block's first column), rows pivoted earlier do not.
//
// smem: Pa[NB][per] | Pb[NB][per] | U12[NB][cols] | PR[NB][NB] | pos_s[per] |
//       piv_s[per] | prow_id[NB]
constexpr int NTP = 128;    // panel group threads (warps 0-3)

__device__ __forceinline__ void panel_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ Cand panel_best(Cand c, Cand* red) {
    c = warp_best(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = c;
    panel_sync();
    if (warp == 0) {
        Cand x = (lane < NTP / 32) ? red[lane] : Cand{-1.0, INT_MAX, -1};
        x = warp_best(x);
        if (lane == 0) red[NTP / 32] = x;
    }
    panel_sync();
    return red[NTP / 32];
}

// grid barrier entered by the panel group only (one poller)
__device__ __forceinline__ bool panel_grid_barrier(unsigned* bar, unsigned target, int* status,
                                                   int64_t budget, volatile int* ok_s) {
    panel_sync();
    if (threadIdx.x == 0) {
        red_release_add_u32(bar, 1u);
        int good = 1;
        int64_t spins = 0;
        while (ld_acquire_u32(bar) < target) {
            if (ld_volatile_i32(status) != DEV_OK) { good = 0; break; }
            if (++spins > budget) {
                atomicCAS(status, DEV_OK, DEV_TIMEOUT);
                good = 0;
                break;
            }
        }
        *ok_s = good;
    }
    panel_sync();
    return *ok_s != 0;
}

__global__ void __launch_bounds__(NT)
k_panel_lu_la(int64_t rows, int cols, double* __restrict__ X, int64_t ldx,
              PanelScratch* __restrict__ ps, double* __restrict__ slots,
              double* __restrict__ Ubuf, int* __restrict__ pos_g, int* __restrict__ piv_g,
              int* __restrict__ status, int64_t budget, int per) {
    extern __shared__ double dsm[];
    double* Pa = dsm;
    double* Pb = Pa + NB * per;
    double* U12 = Pb + NB * per;
    double* PR = U12 + int64_t(NB) * cols;
    int* pos_s = reinterpret_cast<int*>(PR + NB * NB);
    int* piv_s = pos_s + per;
    int* prow_id = piv_s + per;
    __shared__ Cand red[NTP / 32 + 1];
    __shared__ Cand piv;
    __shared__ int win_slot;
    __shared__ int nan_seen;
    __shared__ volatile int panel_ok;
    __shared__ int abort_s;
    __shared__ double rinv_s;

    const int nb = gridDim.x;
    const int t = threadIdx.x;
    const bool panel = t < NTP;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = min(rows, r0 + per);
    const int R = int(r1 > r0 ? r1 - r0 : 0);
    const int steps = int(rows < int64_t(cols) ? rows : int64_t(cols));
    const int slot_w = NB + 3;
    unsigned nbar = 0;                        // grid barriers passed (same sequence in every CTA)

    for (int r = t; r < R; r += NT) {
        pos_s[r] = int(r0 + r);
        piv_s[r] = -1;
    }
    if (t == 0) {
        nan_seen = 0;
        abort_s = 0;
    }
    __syncthreads();

    double* Pc = Pa;                          // block being factored
    double* Lp = Pb;                          // previous block's multipliers
    for (int j0 = 0; j0 < steps; j0 += NB) {
        const int nbk = min(NB, steps - j0);
        const bool have_prev = j0 > 0;
        // ---- catch-up: the block's columns of own rows, minus block b-1's update
        for (int e = t; e < nbk * R; e += NT) {
            const int r = e % R, c = e / R;
            double x = X[(r0 + r) + int64_t(j0 + c) * ldx];
            const int ps_r = piv_s[r];
            if (have_prev && (ps_r < 0 || ps_r >= j0)) {
                double acc = 0.0;
                for (int u = 0; u < NB; ++u) acc = fma(Lp[u * per + r], U12[u * cols + j0 + c], acc);
                x -= acc;
            }
            Pc[c * per + r] = x;
        }
        __syncthreads();
        if (panel) {
            // ---------------------------------------------- panel group: steps
            Cand best{-1.0, INT_MAX, -1};
            for (int r = t; r < R; r += NTP) {
                if (piv_s[r] >= 0) continue;
                const double a = fabs(Pc[r]);
                if (is_nan_abs(a)) nan_seen = 1;
                const Cand c{a, pos_s[r], int(r0 + r)};
                if (better(c, best)) best = c;
            }
            for (int sc = 0; sc < nbk; ++sc) {
                const int j = j0 + sc;
                const Cand cb = panel_best(best, red);
                double* myslot = slots + (int64_t(j & 1) * nb + blockIdx.x) * slot_w;
                if (t == 0) {
                    myslot[0] = cb.v;
                    int2 pr;
                    pr.x = cb.pos;
                    pr.y = cb.row;
                    reinterpret_cast<int2*>(myslot + 1)[0] = pr;
                }
                if (t < nbk && cb.row >= 0) myslot[3 + t] = Pc[t * per + int(cb.row - r0)];
                ++nbar;
                if (!panel_grid_barrier(&ps->barrier, nbar * unsigned(nb), status, budget,
                                        &panel_ok)) {
                    if (t == 0) abort_s = 1;
                    break;
                }
                if (t < 32) {
                    Cand g{-1.0, INT_MAX, -1};
                    int gs = -1;
                    for (int b0 = 0; b0 < nb; b0 += 256) {
                        double v[8];
                        int2 pr[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int b = b0 + t + 32 * k;
                            if (b < nb) {
                                const double* src = slots + (int64_t(j & 1) * nb + b) * slot_w;
                                v[k] = __ldcg(src);
                                pr[k] = __ldcg(reinterpret_cast<const int2*>(src + 1));
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int b = b0 + t + 32 * k;
                            if (b < nb) {
                                const Cand c{v[k], pr[k].x, pr[k].y};
                                if (better(c, g)) { g = c; gs = b; }
                            }
                        }
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const Cand o = shfl_cand(g, off);
                        const int os = __shfl_xor_sync(0xffffffffu, gs, off);
                        if (better(o, g)) { g = o; gs = os; }
                    }
                    if (t == 0) {
                        piv = g;
                        win_slot = gs;
                    }
                }
                panel_sync();
                const Cand pv = piv;
                if (pv.row < 0) {
                    if (t == 0) {
                        if (blockIdx.x == 0) atomicCAS(status, DEV_OK, DEV_NUMERIC);
                        abort_s = 1;
                    }
                    break;
                }
                const double* wsrc = slots + (int64_t(j & 1) * nb + win_slot) * slot_w;
                if (t < nbk) {
                    const double u = __ldcg(wsrc + 3 + t);
                    PR[sc * NB + t] = u;
                    if (t == sc) rinv_s = 1.0 / u;   // one FP64 division per step
                }
                if (t == 0) prow_id[sc] = pv.row;
                for (int r = t; r < R; r += NTP) {
                    if (r0 + r == pv.row) {
                        pos_s[r] = j;
                        piv_s[r] = j;
                    } else if (pos_s[r] == j) {
                        pos_s[r] = pv.pos;
                    }
                }
                if (blockIdx.x == 0 && t == 0) {
                    if (pv.v == 0.0 && ps->info == 0) ps->info = j + 1;
                    if (!(pv.v <= 1.7976931348623157e308)) ps->any_nan = 1;
                }
                panel_sync();
                const double ujj = PR[sc * NB + sc];
                const bool next = sc + 1 < nbk;
                best = Cand{-1.0, INT_MAX, -1};
                for (int r = t; r < R; r += NTP) {
                    if (piv_s[r] >= 0) continue;
                    if (ujj != 0.0) {
                        const double l = lu_multiplier(Pc[sc * per + r], ujj, rinv_s);
                        Pc[sc * per + r] = l;
                        for (int u = sc + 1; u < nbk; ++u)
                            Pc[u * per + r] = fma(-l, PR[sc * NB + u], Pc[u * per + r]);
                    }
                    if (next) {
                        const double a = fabs(Pc[(sc + 1) * per + r]);
                        if (is_nan_abs(a)) nan_seen = 1;
                        const Cand c{a, pos_s[r], int(r0 + r)};
                        if (better(c, best)) best = c;
                    }
                }
            }
        } else {
            // ------------------------------ update group: block b-1's deferred update
            // of the columns beyond block b (rows not pivoted before block b; a
            // row the panel group pivots meanwhile has piv_s >= j0 either way)
            if (have_prev) {
                const int tu = t - NTP;
                const int c0 = j0 + NB;
                const int ncol = cols - c0;
                for (int64_t e = tu; e < int64_t(R) * (ncol > 0 ? ncol : 0); e += NT - NTP) {
                    const int r = int(e % R), c = c0 + int(e / R);
                    const int ps_r = piv_s[r];
                    if (ps_r >= 0 && ps_r < j0) continue;
                    double acc = 0.0;
                    for (int u = 0; u < NB; ++u)
                        acc = fma(Lp[u * per + r], U12[u * cols + c], acc);
                    X[(r0 + r) + int64_t(c) * ldx] -= acc;
                }
            }
            nbar += unsigned(nbk);            // the panel group's step barriers
        }
        __syncthreads();
        if (abort_s) return;
        // block columns of own rows back to X (multipliers; pivot rows keep U11)
        for (int e = t; e < nbk * R; e += NT) {
            const int r = e % R, c = e / R;
            X[(r0 + r) + int64_t(j0 + c) * ldx] = Pc[c * per + r];
        }
        if (blockIdx.x == 0) {
            for (int e = t; e < nbk * nbk; e += NT) {
                const int sr = e % nbk, c = e / nbk;
                if (c >= sr) Ubuf[(j0 + sr) + int64_t(j0 + c) * steps] = PR[sr * NB + c];
            }
        }
        // every CTA's deferred update is visible after this barrier: U12 of block
        // b over all trailing columns, from the fully updated pivot rows
        ++nbar;
        if (!grid_barrier(&ps->barrier, nbar * unsigned(nb), status, budget)) return;
        for (int c = j0 + nbk + t; c < cols; c += NT) {
            for (int sr = 0; sr < nbk; ++sr) {
                double acc = __ldcg(&X[prow_id[sr] + int64_t(c) * ldx]);
                for (int u = 0; u < sr; ++u) acc = fma(-PR[sr * NB + u], U12[u * cols + c], acc);
                U12[sr * cols + c] = acc;
            }
        }
        __syncthreads();
        if (blockIdx.x == 0) {
            for (int e = t; e < nbk * (cols - j0 - nbk); e += NT) {
                const int sr = e % nbk, c = j0 + nbk + e / nbk;
                Ubuf[(j0 + sr) + int64_t(c) * steps] = U12[sr * cols + c];
            }
        }
        double* tmp = Pc;
        Pc = Lp;
        Lp = tmp;
        __syncthreads();
    }
    for (int r = t; r < R; r += NT) {
        pos_g[r0 + r] = pos_s[r];
        piv_g[r0 + r] = piv_s[r];
    }
    if (nan_seen) atomicExch(&ps->any_nan, 1);
}

// After the factorisation: info and the NaN flag; mode 0 writes the unit
// diagonal and the zeros above it into X (X = P^T L in place); mode 1 writes
// perm (perm[pos[i]] = i) and the k pivot rows of U (or U^T).
__global__ void k_panel_finalize(int64_t rows, int cols, double* __restrict__ X, int64_t ldx,
                                 int mode, const int* __restrict__ pos,
                                 const int* __restrict__ pivstep, int32_t* __restrict__ perm,
                                 double* __restrict__ U, int64_t ldU, int u_trans,
                                 const PanelHead* __restrict__ ps, int32_t* __restrict__ info,
                                 int* __restrict__ status, const double* __restrict__ Ubuf) {
    const int r = int(rows < int64_t(cols) ? rows : int64_t(cols));
    // after a failed factorisation (barrier timeout, NaN panel) the row state
    // is incomplete: write nothing
    if (*reinterpret_cast<volatile int*>(status) != DEV_OK) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (info) *info = ps->info;
        if (ps->any_nan) atomicCAS(status, DEV_OK, DEV_NUMERIC);
    }
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int s = pivstep[i];
        if (s < -1 || s >= r) continue;                    // defensive: never index with junk
        if (mode != 0 && (pos[i] < 0 || int64_t(pos[i]) >= rows)) continue;
        if (mode == 0) {
            if (s >= 0) {
                X[i + int64_t(s) * ldx] = 1.0;
                for (int c = s + 1; c < cols; ++c) X[i + int64_t(c) * ldx] = 0.0;
            }
            continue;
        }
        const int64_t pp = pos[i];
        perm[pp] = int32_t(i);
        // L is written by k_panel_gather_l once perm is complete
        if (s >= 0) {
            for (int c = 0; c < cols; ++c) {
                const double v = (c < s) ? 0.0
                                         : (Ubuf ? Ubuf[s + int64_t(c) * r] : X[i + int64_t(c) * ldx]);
                if (u_trans) U[c + int64_t(s) * ldU] = v;
                else U[s + int64_t(c) * ldU] = v;
            }
        }
    }
}

// Mode 1, after k_panel_finalize has written perm: L(pp, c) = the factored
// row perm[pp] of X in column c, with a unit diagonal and zeros above it (or
// L^T when l_trans).  CTA row blockIdx.y covers columns 8 y .. 8 y + 7; each
// thread gathers its eight values before it stores any.
constexpr int GC = 8;
__global__ void k_panel_gather_l(int64_t rows, int r, const double* __restrict__ X, int64_t ldx,
                                 const int32_t* __restrict__ perm,
                                 const int* __restrict__ pivstep, double* __restrict__ L,
                                 int64_t ldL, int l_trans, const int* __restrict__ status) {
    if (*reinterpret_cast<const volatile int*>(status) != DEV_OK) return;
    const int c0 = blockIdx.y * GC;
    const int nc = min(GC, r - c0);
    for (int64_t pp = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; pp < rows;
         pp += int64_t(gridDim.x) * blockDim.x) {
        const int32_t i = perm[pp];
        if (i < 0 || int64_t(i) >= rows) continue;        // defensive: never index with junk
        const int s = pivstep[i];
        if (s < -1 || s >= r) continue;
        double v[GC];
#pragma unroll
        for (int q = 0; q < GC; ++q) {
            const int c = c0 + q;
            v[q] = 0.0;
            if (q < nc) {
                if (s >= 0 && c == s) v[q] = 1.0;
                else if (!(s >= 0 && c > s)) v[q] = X[i + int64_t(c) * ldx];
            }
        }
#pragma unroll
        for (int q = 0; q < GC; ++q) {
            if (q < nc) {
                const int c = c0 + q;
                if (l_trans) L[c + pp * ldL] = v[q];
                else L[pp + int64_t(c) * ldL] = v[q];
            }
        }
    }
}

}  // namespace

size_t panel_scratch_bytes(int64_t rows, int cols) {
    const size_t head = (sizeof(PanelScratch) + 255) & ~size_t(255);
    const size_t slots = size_t(2) * kMaxGrid * (NB + 3) * sizeof(double);
    const int64_t steps = rows < cols ? rows : cols;
    const size_t ubuf = size_t(steps) * size_t(cols) * sizeof(double);
    return head + slots + 256 + ubuf + 256 + 2 * size_t(rows) * sizeof(int) + 256;
}

cudaError_t launch_panel_lu(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                            int32_t* perm, double* L, int64_t ldL, int l_trans,
                            double* U, int64_t ldU, int u_trans, int32_t* info,
                            void* scratch, int* dev_status, int64_t spin_budget,
                            int num_sms, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (cols > kMaxCols) return cudaErrorInvalidValue;
    char* base = static_cast<char*>(scratch);
    PanelScratch* ps = reinterpret_cast<PanelScratch*>(base);
    size_t off = (sizeof(PanelScratch) + 255) & ~size_t(255);
    double* slots = reinterpret_cast<double*>(base + off);
    off += (size_t(2) * kMaxGrid * (NB + 3) * sizeof(double) + 255) & ~size_t(255);
    double* Ubuf = reinterpret_cast<double*>(base + off);
    const int64_t steps = rows < cols ? rows : cols;
    off += (size_t(steps) * size_t(cols) * sizeof(double) + 255) & ~size_t(255);
    int* pos = reinterpret_cast<int*>(base + off);
    int* pivstep = pos + rows;
    cudaError_t e = cudaMemsetAsync(ps, 0, sizeof(PanelScratch), s);
    if (e != cudaSuccess) return e;
    // grid: at most one CTA per SM, at least ~32 rows per CTA
    int64_t nb = (rows + 31) / 32;
    if (nb > num_sms) nb = num_sms;
    if (nb > kMaxGrid) nb = kMaxGrid;
    if (nb < 1) nb = 1;
    int64_t per = (rows + nb - 1) / nb;
    nb = (rows + per - 1) / per;
    // step tags of the candidate slots start below every step number
    e = cudaMemsetAsync(slots, 0, size_t(2) * nb * (NB + 3) * sizeof(double), s);
    if (e != cudaSuccess) return e;
    int64_t rows_ = rows;
    int cols_ = cols;
    int64_t ldx_ = ldx;
    int64_t budget = spin_budget;
    const size_t smem_blk = size_t(NB) * per * 8 + size_t(NB) * UC * 8 + size_t(NB) * NB * 8 +
                            size_t(2) * per * 4 + NB * 4 + 64;
    const size_t smem_la = size_t(2) * NB * per * 8 + size_t(NB) * cols * 8 +
                           size_t(NB) * NB * 8 + size_t(2) * per * 4 + NB * 4 + 64;
    const bool blocked = smem_blk <= 200 * 1024;
    const bool lookahead = cols > NB && smem_la <= 210 * 1024;
    if (lookahead) {
        e = cudaFuncSetAttribute(k_panel_lu_la, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem_la));
        if (e != cudaSuccess) return e;
        int per_ = int(per);
        void* args[] = {&rows_, &cols_, &X, &ldx_, &ps, &slots, &Ubuf, &pos, &pivstep,
                        &dev_status, &budget, &per_};
        count_launch();
        e = cudaLaunchCooperativeKernel((const void*)k_panel_lu_la, dim3(unsigned(nb)),
                                        dim3(NT), args, smem_la, s);
    } else if (blocked) {
        e = cudaFuncSetAttribute(k_panel_lu_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem_blk));
        if (e != cudaSuccess) return e;
        int per_ = int(per);
        void* args[] = {&rows_, &cols_, &X, &ldx_, &ps, &slots, &Ubuf, &pos, &pivstep,
                        &dev_status, &budget, &per_};
        count_launch();
        e = cudaLaunchCooperativeKernel((const void*)k_panel_lu_blocked, dim3(unsigned(nb)),
                                        dim3(NT), args, smem_blk, s);
    } else {
        const size_t smem = size_t(cols) * sizeof(double);
        void* args[] = {&rows_, &cols_, &X, &ldx_, &ps, &pos, &pivstep, &dev_status, &budget};
        count_launch();
        e = cudaLaunchCooperativeKernel((const void*)k_panel_lu, dim3(unsigned(nb)), dim3(NT),
                                        args, smem, s);
    }
    if (e != cudaSuccess) return e;
    return launch_panel_finish(rows, cols, X, ldx, mode, perm, L, ldL, l_trans, U, ldU, u_trans,
                               info, ps, pos, pivstep, (blocked || lookahead) ? Ubuf : nullptr,
                               dev_status, num_sms, s);
}

size_t panel_head_bytes() { return sizeof(PanelScratch); }

cudaError_t launch_panel_finish(int64_t rows, int cols, double* X, int64_t ldx, int mode,
                                int32_t* perm, double* L, int64_t ldL, int l_trans, double* U,
                                int64_t ldU, int u_trans, int32_t* info, const void* head,
                                const int* pos, const int* pivstep, const double* Ubuf,
                                int* dev_status, int num_sms, cudaStream_t s) {
    int64_t fb = (rows + 255) / 256;
    if (fb > int64_t(num_sms) * 8) fb = int64_t(num_sms) * 8;
    count_launch();
    k_panel_finalize<<<unsigned(fb), 256, 0, s>>>(rows, cols, X, ldx, mode, pos, pivstep, perm,
                                                  U, ldU, u_trans,
                                                  static_cast<const PanelHead*>(head), info,
                                                  dev_status, Ubuf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || mode == 0) return e;
    const int r = int(rows < int64_t(cols) ? rows : int64_t(cols));
    const int64_t gy = (r + GC - 1) / GC;
    int64_t gx = (rows + 255) / 256;
    const int64_t gcap = (int64_t(num_sms) * 16 + gy - 1) / gy;
    if (gx > gcap) gx = gcap;
    if (gy > 65535) return cudaErrorInvalidValue;
    count_launch();
    k_panel_gather_l<<<dim3(unsigned(gx), unsigned(gy)), 256, 0, s>>>(rows, r, X, ldx, perm,
                                                                       pivstep, L, ldL, l_trans,
                                                                       dev_status);
    return cudaGetLastError();
}

}  // namespace plu
