// lsqr.cu -- LSQR (Paige & Saunders 1982) on the augmented operator
// A = [G; w L] (or [G D; w L D; lambda D] with a right diagonal scaling),
// the solver of the paper's least-squares module ("Solver for the
// Large-scale Linear System"; the paper names LSQR beside LSMR).
//
// One iteration is five kernels:
//   k_step the FP64 scalar recurrence of the previous adjoint (rotations, norm
//          estimates, stopping rules), one warp, run beside k_fwd, which needs
//          only alpha and beta (on B300 the step's chain of dependent FP64
//          operations takes ~16 us; at the end of k_adj it was ~14 % of a
//          64 x 64 x 16 adjoint sweep)
//   k_fwd  u-bar <- A v - alpha u and beta = ||u-bar||   (G rows: warp per CSR
//          row, gather of v; L rows: 7-point stencil, thread per column)
//   k_upd  x += t1 w, w = v + t2 w in FP64 and ||w||^2 with the step's
//          coefficients; after k_step on the same side branch, beside k_fwd
//          (it reads v-bar and writes x, w, which the forward does not touch)
//   k_pub  one block: publishes the step once both branches have joined
//   k_adj  v-bar <- A^T u - beta v and alpha = ||v-bar|| (warp per CSC column,
//          gather of u; the stencil term added by the same warp); its last
//          block leaves the scalar step pending for the next k_step (the
//          damping sweep advances its recurrences there instead)
// Both products are gathers (no atomics).  Vectors are never normalised in
// place: u-bar and v-bar are kept with their norms and the 1/beta, 1/alpha
// factors are folded into the next product, so each Golub-Kahan step is one
// sweep plus one fused norm reduction.  Every reduction is a fixed-order
// block sum followed by a fixed-order sum over blocks done by the last block,
// so results are bit-reproducible run to run.  The iteration is replayed from
// a CUDA graph; kernels return at entry once the stopping rule has fired.
#include <cfloat>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "lsqr_dev.cuh"

namespace pdst {

constexpr int LT = 256;         // threads per block of the LSQR kernels
constexpr int MAXBLK = 4096;    // upper bound on blocks per reduction kernel

enum { FMT_ELEM = 0, FMT_BLK = 1 };

template <class VT, class ST> struct OpArgs {
    int64_t m;
    int32_t n;
    int nx, ny, nz;
    const int64_t *row_ptr;   // element CSR
    const int32_t *col;
    const int64_t *col_ptr;   // element CSC
    const int32_t *row_idx;
    const int64_t *row_cptr;  // blocked
    const int32_t *row_cells;
    const int64_t *cell_rptr;
    const int32_t *cell_rows;
    const int32_t *cell_cnt;
    const int32_t *cell_order;
    const VT *val;            // CSR order
    const VT *valT;           // element CSC order (element layout only)
    const VT *valB;           // blocked CSC order
    double *hbar;             // LSMR h-bar (n)
    LsqrScalars *lam_sc;      // damping sweep: one recurrence per damping value
    double *cell_ss;          // H: sum of v-bar^2 over a cell split over several items
    int32_t n_cells;          // H
    int32_t n_lam;            // 0: ordinary solve
    const int32_t *adj_item;  // (cell, first row) per adjoint work item
    int32_t adj_chunk;        // rows per adjoint work item
    int64_t n_adj;
    ST *chunk_part;           // n_adj x nz partial column sums (multi-chunk cells)
    unsigned *cell_done;      // H finished-chunk counters
    const double *D;          // right diagonal scaling or nullptr
    const void *Pb;           // per-cell depth blocks P_h (ST-typed, H x nz x nz) or nullptr
    const void *PbT;          // the blocks transposed (P_h^T, row-major)
    int lam_rows_on;          // append lambda*D (or lambda*P) rows
    ST *ubar;                 // M = m + n (+ n)
    ST *vbar;                 // n
    ST *vsc;                  // n: D o v-bar (== vbar when no scaling)
    double *x, *wv;           // n, FP64
    double *partial;          // 3 x MAXBLK
    LsqrScalars *sc;
    LsqrScalars *sc_stage;    // the deferred scalar step's copy (k_step; published by k_upd)
    LsqrSync *sy;
};

// ---------------------------------------------- programmatic dependent launch

// The sweeps of an iteration are launched with programmatic stream
// serialisation: a kernel's blocks may be scheduled while the kernel before it
// is still finishing (its last block's fixed-order sums), and wait here until
// that kernel has completed and its writes are visible.  Without the launch
// attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel's blocks be scheduled as this kernel's blocks leave.
__device__ __forceinline__ void pdl_allow_next() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------ dot products

// sum_p val[p] * x[idx[p]] over p in [ptr[r], ptr[r+1]) by one warp: ragged
// head and tail by single lanes, the aligned body four entries per lane with
// 128-bit index loads and streaming (evict-first) value loads.
template <class VT, class AT, class XT>
__device__ __forceinline__ AT dot_elem(const int64_t *__restrict__ ptr,
                                       const int32_t *__restrict__ idx,
                                       const VT *__restrict__ val, const XT *__restrict__ x,
                                       int64_t r, int lane) {
    const int64_t p0 = ptr[r], p1 = ptr[r + 1];
    int64_t a = (p0 + 3) & ~int64_t(3);
    if (a > p1) a = p1;
    const int64_t b = a + ((p1 - a) & ~int64_t(3));
    AT s = 0;
    if (p0 + lane < a) s += (AT)widen(val[p0 + lane]) * (AT)__ldg(x + idx[p0 + lane]);
    for (int64_t p = a + 4 * lane; p < b; p += 128) {
        int4 c = __ldcs(reinterpret_cast<const int4 *>(idx + p));
        typename Wide<VT>::T v[4];
        Pack4<VT>::ld(val + p, v);
        s += (AT)v[0] * (AT)__ldg(x + c.x);
        s += (AT)v[1] * (AT)__ldg(x + c.y);
        s += (AT)v[2] * (AT)__ldg(x + c.z);
        s += (AT)v[3] * (AT)__ldg(x + c.w);
    }
    if (b + lane < p1) s += (AT)widen(val[b + lane]) * (AT)__ldg(x + idx[b + lane]);
    return warp_sum(s);
}

// Blocked CSR row: runs e in [row_cptr[r], row_cptr[r+1]) of nz consecutive
// columns cells[e]*nz + k, values val[nz*e + k].  With nz % 4 == 0 every group
// of four entries lies in one run and gathers a contiguous 4-vector of x.
template <class VT, class AT, class XT>
__device__ __forceinline__ AT dot_blk_row(const int64_t *__restrict__ row_cptr,
                                          const int32_t *__restrict__ cells,
                                          const VT *__restrict__ val, const XT *__restrict__ x,
                                          int64_t r, int nz, int lane) {
    const int64_t e0 = row_cptr[r], e1 = row_cptr[r + 1];
    const int64_t p0 = e0 * nz;
    const uint32_t len = (uint32_t)((e1 - e0) * nz);
    AT s = 0;
    if ((nz & 3) == 0) {
        for (uint32_t rel = 4u * lane; rel < len; rel += 128u) {
            uint32_t ee = rel / (uint32_t)nz;
            uint32_t k = rel - ee * (uint32_t)nz;
            int h = __ldg(cells + e0 + ee);
            typename Wide<VT>::T v[4];
            Pack4<VT>::ld(val + p0 + rel, v);
            XT xv[4];
            ldx4<XT>(x + (int64_t)h * nz + k, xv);
            s += (AT)v[0] * (AT)xv[0];
            s += (AT)v[1] * (AT)xv[1];
            s += (AT)v[2] * (AT)xv[2];
            s += (AT)v[3] * (AT)xv[3];
        }
    } else {
        for (uint32_t rel = lane; rel < len; rel += 32u) {
            uint32_t ee = rel / (uint32_t)nz;
            uint32_t k = rel - ee * (uint32_t)nz;
            int h = __ldg(cells + e0 + ee);
            s += (AT)widen(val[p0 + rel]) * (AT)__ldg(x + (int64_t)h * nz + k);
        }
    }
    return warp_sum(s);
}

// Blocked CSC column j = h*nz + k: rows cell_rows[cell_rptr[h] + q], values
// valB[(cell_rptr[h] + q)*nz + k] (used by pdst_apply_G).
template <class VT, class AT, class XT>
__device__ __forceinline__ AT dot_blk_col(const int64_t *__restrict__ cell_rptr,
                                          const int32_t *__restrict__ cell_cnt,
                                          const int32_t *__restrict__ cell_rows,
                                          const VT *__restrict__ valB, const XT *__restrict__ u,
                                          int64_t j, int nz, int lane) {
    const int64_t h = j / nz;
    const int k = (int)(j - h * nz);
    const int64_t c0 = cell_rptr[h];
    const int cnt = cell_cnt[h];
    const VT *v = valB + c0 * nz + k;
    const int32_t *rows = cell_rows + c0;
    AT s = 0;
    for (int q = lane; q < cnt; q += 32) s += (AT)widen(v[(int64_t)q * nz]) * (AT)__ldg(u + rows[q]);
    return warp_sum(s);
}

// ------------------------------------------- blocked products, LSQR sweeps

// Lane partial of one blocked CSR row for a half-warp (nz = 4 Q, Q known at
// compile time).  The row's entries are read as consecutive 4-entry quads:
// quad f covers entries 4f..4f+3 of run f / Q, so a half-warp instruction
// reads 256 contiguous bytes of values and whole 64-byte stretches of x (the
// Q lanes of one run share its cell, read from L1).  UN quads per lane are
// requested before any is used.
template <class VT, class AT, class XT, int Q>
__device__ __forceinline__ AT blk_row_quads(const VT *__restrict__ vrow, const XT *__restrict__ x,
                                            const int32_t *__restrict__ cells_row, uint32_t nrun,
                                            int hl) {
    constexpr int UN = Unroll<AT>::U;
    constexpr uint32_t NZ = 4u * Q;
    const uint32_t nquad = nrun * Q;
    AT s = 0;
    for (uint32_t base = 0; base < nquad; base += 16u * UN) {
        int h[UN];
        uint32_t off[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const uint32_t f = base + hl + 16u * u;
            const uint32_t run = f / Q;
            off[u] = 4u * (f - run * Q);
            h[u] = f < nquad ? __ldg(cells_row + run) : -1;
        }
        typename Wide<VT>::T vv[UN][4];
        XT xx[UN][4];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const uint32_t f = base + hl + 16u * u;
            if (h[u] >= 0) {
                Pack4<VT>::ld(vrow + 4u * f, vv[u]);
                ldx4<XT>(x + (size_t)h[u] * NZ + off[u], xx[u]);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    vv[u][t] = 0;
                    xx[u][t] = 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
            for (int t = 0; t < 4; ++t) s += (AT)vv[u][t] * (AT)xx[u][t];
    }
    return s;
}

// floor(f / q) for a divisor fixed per row, by one high multiply with
// m = ceil(2^32 / q) (Granlund & Montgomery, division by invariant integers):
// f / q + f e / (q 2^32), e = m q - 2^32 < q, keeps the floor while
// f (q - 1) < 2^32, far above any row's entry count.
struct DivQ {
    uint32_t q, m;
    __device__ __forceinline__ explicit DivQ(uint32_t q_) : q(q_), m(q_ > 1u ? 0xFFFFFFFFu / q_ + 1u : 0u) {}
    __device__ __forceinline__ uint32_t div(uint32_t f) const { return q > 1u ? __umulhi(f, m) : f; }
};

// Same for any nz % 4 == 0 (run and quad from a run-time division).
template <class VT, class AT, class XT>
__device__ __forceinline__ AT blk_row_quads_rt(const VT *__restrict__ vrow,
                                               const XT *__restrict__ x,
                                               const int32_t *__restrict__ cells_row,
                                               uint32_t nrun, uint32_t nz, int hl) {
    const uint32_t q = nz >> 2, nquad = nrun * q;
    AT s = 0;
    for (uint32_t f = hl; f < nquad; f += 16u) {
        const uint32_t run = f / q;   // (the high-multiply division measured slower here)
        const int h = __ldg(cells_row + run);
        typename Wide<VT>::T vv[4];
        XT xx[4];
        Pack4<VT>::ld(vrow + 4u * f, vv);
        ldx4<XT>(x + (size_t)h * nz + 4u * (f - run * q), xx);
#pragma unroll
        for (int t = 0; t < 4; ++t) s += (AT)vv[t] * (AT)xx[t];
    }
    return s;
}

// Rows per forward block of one warp (even).  Two: at any moment the warps
// of the grid stream one narrow band of consecutive rows, whose values are
// contiguous; blocks of 8, 16 or 32 consecutive rows per warp (more L1 reuse
// of x between rows of one station pair) measured 25-80 % slower on B300.
constexpr int FWD_RB = 2;

// Any even nz (the quads need nz % 4 == 0): consecutive 2-entry pairs, so a
// half-warp instruction reads 128 contiguous bytes of FP32 values and 8-byte
// stretches of x (aligned: h * nz + 2j is even); four pairs per lane in
// flight.
template <class VT, class AT, class XT>
__device__ __forceinline__ AT blk_row_pairs_rt(const VT *__restrict__ vrow,
                                               const XT *__restrict__ x,
                                               const int32_t *__restrict__ cells_row,
                                               uint32_t nrun, uint32_t nz, int hl) {
    constexpr int UP = 4;
    const uint32_t q = nz >> 1, npair = nrun * q;
    const DivQ dq(q);
    AT s = 0;
    for (uint32_t base = 0; base < npair; base += 16u * UP) {
        int h[UP];
        uint32_t off[UP];
#pragma unroll
        for (int u = 0; u < UP; ++u) {
            const uint32_t f = base + hl + 16u * u;
            const uint32_t run = dq.div(f);
            off[u] = 2u * (f - run * q);
            h[u] = f < npair ? __ldg(cells_row + run) : -1;
        }
        typename Wide<VT>::T vv[UP][2];
        XT xx[UP][2];
#pragma unroll
        for (int u = 0; u < UP; ++u) {
            const uint32_t f = base + hl + 16u * u;
            if (h[u] >= 0) {
                Pack2<VT>::ld(vrow + 2u * f, vv[u]);
                ldx2<XT>(x + (size_t)h[u] * nz + off[u], xx[u]);
            } else {
                vv[u][0] = vv[u][1] = 0;
                xx[u][0] = xx[u][1] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < UP; ++u) s += (AT)vv[u][0] * (AT)xx[u][0] + (AT)vv[u][1] * (AT)xx[u][1];
    }
    return s;
}

// nz % 6 == 0 off the quad paths (e.g. 18 depth nodes): groups of 6
// entries (three pairs) of one run per lane, three groups (72 bytes of FP32
// values) in flight; at nz = 18 measured 1.37x faster than pairs, whose four
// pairs in flight (32 bytes) leave the stream latency-bound.  FP32 and BF16
// sums only: with FP64 sums the groups do not fit the registers (one group in
// flight measured 1.3x slower than pairs).
template <class VT, class AT, class XT, int US = 3>
__device__ __forceinline__ AT blk_row_sextets(const VT *__restrict__ vrow,
                                              const XT *__restrict__ x,
                                              const int32_t *__restrict__ cells_row,
                                              uint32_t nrun, uint32_t nz, int hl) {
    const uint32_t q = nz / 6u, ng = nrun * q;
    const DivQ dq(q);
    AT s = 0;
    for (uint32_t base = 0; base < ng; base += 16u * US) {
        int h[US];
        uint32_t off[US];
#pragma unroll
        for (int u = 0; u < US; ++u) {
            const uint32_t f = base + hl + 16u * u;
            const uint32_t run = dq.div(f);
            off[u] = 6u * (f - run * q);
            h[u] = f < ng ? __ldg(cells_row + run) : -1;
        }
        typename Wide<VT>::T vv[US][6];
        XT xx[US][6];
#pragma unroll
        for (int u = 0; u < US; ++u) {
            const uint32_t f = base + hl + 16u * u;
            if (h[u] >= 0) {
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    Pack2<VT>::ld(vrow + 6u * f + 2 * t, vv[u] + 2 * t);
                    ldx2<XT>(x + (size_t)h[u] * nz + off[u] + 2 * t, xx[u] + 2 * t);
                }
            } else {
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    vv[u][t] = 0;
                    xx[u][t] = 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < US; ++u)
#pragma unroll
            for (int t = 0; t < 6; ++t) s += (AT)vv[u][t] * (AT)xx[u][t];
    }
    return s;
}

template <class VT, class ST, int Q, int SX = 3>
__device__ __forceinline__ double fwd_rows_halfwarp(const OpArgs<VT, ST> &a, ST ia, ST cu,
                                                    int64_t gw, int64_t nw, int lane) {
    using AT = ST;
    double ss = 0.0;
    const uint32_t nz = (uint32_t)a.nz;
    const int hl = lane & 15, hw = lane >> 4;
    // warp gw takes blocks of FWD_RB consecutive rows (blocks gw, gw + nw, ...),
    // the two half-warps alternate rows inside a block
    constexpr int RBH = FWD_RB / 2;
    auto row_of = [&](int64_t i) -> int64_t {
        return (gw + (i / RBH) * nw) * FWD_RB + 2 * (i % RBH) + hw;
    };
    int64_t r = row_of(0);
    int64_t e0 = 0, e1 = 0, e0n = 0, e1n = 0;
    if (r < a.m) {
        e0 = __ldg(a.row_cptr + r);
        e1 = __ldg(a.row_cptr + r + 1);
    }
    if (row_of(1) < a.m) {
        e0n = __ldg(a.row_cptr + row_of(1));
        e1n = __ldg(a.row_cptr + row_of(1) + 1);
    }
    // both half-warps loop the same number of times so that the reduction
    // shuffles see all 32 lanes
    const int64_t nblk = (a.m + FWD_RB - 1) / FWD_RB;
    const int64_t rows_warp = gw < nblk ? ((nblk - gw + nw - 1) / nw) * RBH : 0;
    for (int64_t it = 0; it < rows_warp; ++it) {
        const bool live = r < a.m;
        const int64_t rn = row_of(it + 1), rnn = row_of(it + 2);
        int64_t e0nn = 0, e1nn = 0;
        if (rn < a.m) {
            // warm L1 with the next row's cells (up to 64 runs) and L2 with its values
            const int64_t nrn = e1n - e0n;
            if (hl * 4 < nrn) prefetch_l1(a.row_cells + e0n + hl * 4);
            if (hl == 0)
                prefetch_l2_bulk(a.val + e0n * (int64_t)nz, (uint64_t)nrn * nz * sizeof(VT));
        }
        if (rnn < a.m) {
            e0nn = __ldg(a.row_cptr + rnn);
            e1nn = __ldg(a.row_cptr + rnn + 1);
        }
        const AT uprev = (live && hl == 0) ? (AT)a.ubar[r] : (AT)0;
        AT part = 0;
        if (live) {
            if (Q > 0)
                part = blk_row_quads<VT, AT, ST, (Q > 0 ? Q : 1)>(
                    a.val + e0 * (int64_t)nz, a.vsc, a.row_cells + e0, (uint32_t)(e1 - e0), hl);
            else if (Q == 0)
                part = blk_row_quads_rt<VT, AT, ST>(a.val + e0 * (int64_t)nz, a.vsc,
                                                    a.row_cells + e0, (uint32_t)(e1 - e0), nz, hl);
            else if (Q == -6)
                part = blk_row_sextets<VT, AT, ST, SX>(a.val + e0 * (int64_t)nz, a.vsc,
                                                       a.row_cells + e0, (uint32_t)(e1 - e0), nz,
                                                       hl);
            else
                part = blk_row_pairs_rt<VT, AT, ST>(a.val + e0 * (int64_t)nz, a.vsc,
                                                    a.row_cells + e0, (uint32_t)(e1 - e0), nz, hl);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        if (live && hl == 0) {
            AT u = part * ia - cu * uprev;
            a.ubar[r] = u;
            ss += (double)u * (double)u;
        }
        r = rn;
        e0 = e0n;
        e1 = e1n;
        e0n = e0nn;
        e1n = e1nn;
    }
    return ss;
}

template <class VT, class ST>
__device__ __forceinline__ double fwd_rows_blk(const OpArgs<VT, ST> &a, ST ia, ST cu,
                                               int64_t gw, int64_t nw, int lane) {
    using AT = ST;
    const uint32_t nz = (uint32_t)a.nz;
    if ((nz & 3u) == 0u) {
        if (nz == 16) return fwd_rows_halfwarp<VT, ST, 4>(a, ia, cu, gw, nw, lane);
        if (nz == 8) return fwd_rows_halfwarp<VT, ST, 2>(a, ia, cu, gw, nw, lane);
        if (nz == 20) return fwd_rows_halfwarp<VT, ST, 5>(a, ia, cu, gw, nw, lane);
        return fwd_rows_halfwarp<VT, ST, 0>(a, ia, cu, gw, nw, lane);
    }
    if constexpr (Unroll<ST>::U == 4) {
        if (nz % 6u == 0u) return fwd_rows_halfwarp<VT, ST, -6>(a, ia, cu, gw, nw, lane);
    }
    if ((nz & 1u) == 0u) return fwd_rows_halfwarp<VT, ST, -1>(a, ia, cu, gw, nw, lane);
    double ss = 0.0;
    const DivQ dq(nz);
    for (int64_t r = gw; r < a.m; r += nw) {
        const int64_t e0 = __ldg(a.row_cptr + r), e1 = __ldg(a.row_cptr + r + 1);
        const uint32_t len = (uint32_t)(e1 - e0) * nz;
        AT part = 0;
        for (uint32_t rel = lane; rel < len; rel += 32u) {
            const uint32_t ee = dq.div(rel), k = rel - ee * nz;
            const int h = __ldg(a.row_cells + e0 + ee);
            part += (AT)widen(a.val[e0 * (int64_t)nz + rel]) * (AT)__ldg(a.vsc + (int64_t)h * nz + k);
        }
        const AT dot = warp_sum(part);
        if (lane == 0) {
            AT u = dot * ia - cu * a.ubar[r];
            a.ubar[r] = u;
            ss += (double)u * (double)u;
        }
    }
    return ss;
}

// Entries per lane of the blocked adjoint for a depth count: 4 (nz % 4 == 0),
// 6 (nz % 6 == 0, e.g. 18 depth nodes: 3 lanes per row, measured 1.45x
// faster than pairs at nz = 18), 2 (other even nz), 1.  G = 2 and G = 1 run
// as kernels of their own (measured 9 % and 14 % faster on B300 than inside
// the kernel that holds every group); G = 4 and 6 share G_ANY, which picks
// the group at run time (equal or faster for them).
constexpr int G_ANY = 0;
__host__ __device__ constexpr int adj_group(int nz) {
    return (nz & 3) == 0 && nz <= 64   ? 4
           : nz % 6 == 0 && nz <= 96   ? 6
           : (nz & 1) == 0 && nz <= 64 ? 2
                                       : 1;
}

// Final value of column j of the adjoint sweep from its G^T u dot product:
// add w L^T u2 (+ lambda u3), scale by D_j, subtract (beta/alpha) v-bar_j.
template <class VT, class ST>
__device__ __forceinline__ double adj_finish(const OpArgs<VT, ST> &a, int64_t j, ST dot, ST ib,
                                             ST cv, ST wsm, ST lamr, int init) {
    using AT = ST;
    AT s = dot + wsm * laplace<AT, ST>(a.ubar + a.m, j, a.nx, a.ny, a.nz);
    if (a.lam_rows_on) s += lamr * (AT)a.ubar[a.m + a.n + j];
    const AT dj = a.D ? (AT)a.D[j] : (AT)1;
    s *= dj;
    // the start step does not read v-bar: the buffer may hold another dtype's
    // bits from an earlier solve on this handle
    const AT v = init ? s * ib : s * ib - cv * a.vbar[j];
    a.vbar[j] = v;
    if (a.D) a.vsc[j] = dj * v;
    return (double)v * (double)v;
}

// The per-cell finish with the depth-block preconditioner P = blockdiag(P_h)
// (P_h upper triangular, nz <= 32): lane k < nz holds the cell's G^T u sum of
// depth k.  s = (A^T u)_h (stencil and lambda terms added per lane),
// t = P_h^T s, v-bar_h <- t / beta - (beta/alpha) v-bar_h, and the forward's
// input P_h v-bar_h; both products by shuffles over the cell's lanes, their
// block entries read row by row (P_h for t, P_h^T for P_h v: each read of a
// row is one contiguous segment across the lanes), CH at a time.  With
// nz <= 16 the two half-warps each take half of every sum's terms and add
// the halves with one shuffle.  Returns this lane's v-bar^2.
template <int CH, class VT, class ST>
__device__ __forceinline__ double adj_finish_blk_ch(const OpArgs<VT, ST> &a, int64_t h, ST dot,
                                                    ST ib, ST cv, ST wsm, ST lamr, int init,
                                                    int lane) {
    using AT = ST;
    const int nz = a.nz;
    const bool split = nz <= 16;
    const int k = split ? (lane & 15) : lane;     // the output depth this lane sums for
    const bool on = k < nz;
    const bool own = lane < nz;                   // the lane that holds depth k's values
    const int ih = split ? (nz + 1) >> 1 : nz;    // terms per half
    const int i0 = (split && lane >= 16) ? ih : 0;
    const int64_t j = h * nz + lane;
    AT sj = 0;
    if (own) {
        sj = dot + wsm * laplace<AT, ST>(a.ubar + a.m, j, a.nx, a.ny, a.nz);
        if (a.lam_rows_on) sj += lamr * (AT)a.ubar[a.m + a.n + j];
    }
    const ST *P = static_cast<const ST *>(a.Pb) + h * nz * nz;
    const ST *PT = static_cast<const ST *>(a.PbT) + h * nz * nz;
    // t_k = sum_{i <= k} P[i][k] s_i over this half's terms i0 .. i0 + ih - 1
    AT t = 0;
    for (int u0 = 0; u0 < ih; u0 += CH) {
        AT pv[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int i = i0 + u0 + u;
            pv[u] = (on && u0 + u < ih && i < nz && i <= k) ? (AT)P[i * nz + k] : (AT)0;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) t += pv[u] * __shfl_sync(FULL, sj, (i0 + u0 + u) & 31);
    }
    if (split) t += __shfl_xor_sync(FULL, t, 16);
    AT v = 0;
    if (own) {
        v = init ? t * ib : t * ib - cv * a.vbar[j];
        a.vbar[j] = v;
    }
    // q_k = sum_{i >= k} P[k][i] v_i = sum_{i >= k} P^T[i][k] v_i
    AT q = 0;
    for (int u0 = 0; u0 < ih; u0 += CH) {
        AT pv[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int i = i0 + u0 + u;
            pv[u] = (on && u0 + u < ih && i < nz && i >= k) ? (AT)PT[i * nz + k] : (AT)0;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) q += pv[u] * __shfl_sync(FULL, v, (i0 + u0 + u) & 31);
    }
    if (split) q += __shfl_xor_sync(FULL, q, 16);
    if (own) a.vsc[j] = q;
    return (double)v * (double)v;
}

// Batches of eight terms: with nz <= 16 one per half-warp and product.
// Batches of sixteen for nz in 17..32 measured no faster (18 depth nodes);
// batches of 32 made the kernel spill.
// nz <= 16 with every load of the lane issued before the first use: its
// block entries for both products (at most eight each) and its old v-bar,
// then the stencil terms; one round trip to L2 instead of three.
template <class VT, class ST>
__device__ __forceinline__ double adj_finish_blk16(const OpArgs<VT, ST> &a, int64_t h, ST dot,
                                                   ST ib, ST cv, ST wsm, ST lamr, int init,
                                                   int lane) {
    using AT = ST;
    const int nz = a.nz;
    const int k = lane & 15;
    const bool on = k < nz;
    const bool own = lane < nz;
    const int ih = (nz + 1) >> 1;
    const int i0 = lane >= 16 ? ih : 0;
    const int64_t j = h * nz + lane;
    const ST *P = static_cast<const ST *>(a.Pb) + h * nz * nz;
    const ST *PT = static_cast<const ST *>(a.PbT) + h * nz * nz;
    AT p1[8], p2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + u;
        const bool in = on && u < ih && i < nz;
        p1[u] = (in && i <= k) ? (AT)P[i * nz + k] : (AT)0;
        p2[u] = (in && i >= k) ? (AT)PT[i * nz + k] : (AT)0;
    }
    const AT vold = (own && !init) ? (AT)a.vbar[j] : (AT)0;
    AT sj = 0;
    if (own) {
        sj = dot + wsm * laplace<AT, ST>(a.ubar + a.m, j, a.nx, a.ny, a.nz);
        if (a.lam_rows_on) sj += lamr * (AT)a.ubar[a.m + a.n + j];
    }
    AT t = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) t += p1[u] * __shfl_sync(FULL, sj, (i0 + u) & 31);
    t += __shfl_xor_sync(FULL, t, 16);
    AT v = 0;
    if (own) {
        v = init ? t * ib : t * ib - cv * vold;
        a.vbar[j] = v;
    }
    AT q = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) q += p2[u] * __shfl_sync(FULL, v, (i0 + u) & 31);
    q += __shfl_xor_sync(FULL, q, 16);
    if (own) a.vsc[j] = q;
    return (double)v * (double)v;
}

template <class VT, class ST>
__device__ __forceinline__ double adj_finish_blk(const OpArgs<VT, ST> &a, int64_t h, ST dot,
                                                 ST ib, ST cv, ST wsm, ST lamr, int init,
                                                 int lane) {
    if constexpr (sizeof(ST) == 4) {   // with 8-byte vectors the preloads spill
        if (a.nz <= 16) return adj_finish_blk16(a, h, dot, ib, cv, wsm, lamr, init, lane);
    }
    return adj_finish_blk_ch<8>(a, h, dot, ib, cv, wsm, lamr, init, lane);
}

// G^T rows of the adjoint sweep in the blocked CSC layout.  Work item = a
// chunk of up to adj_chunk rows of one cell (cells longest first).  A row's
// nz values are contiguous, so L = nz / G lanes share a row, each reading G
// consecutive depths (G = 4: one 16-byte vector) and the row's u once
// (broadcast); 32 / L rows per step, UN steps of loads in flight, row
// indices fetched one step ahead.  Per-depth sums are combined across the
// warp through shared memory in a fixed order; a cell split over several
// chunks is finished by its last chunk, which adds the chunks' partial sums
// in chunk order.
template <class VT, class ST, int G>
__device__ __forceinline__ double adj_cells_chunked(const OpArgs<VT, ST> &a, ST ib, ST cv, ST wsm,
                                                    ST lamr, int init, int64_t gw, int64_t nw,
                                                    int lane, unsigned first) {
    using AT = ST;
    constexpr int UN = Unroll<AT>::U;
    __shared__ AT red[LT / 32][32][G];
    __shared__ int last_flag[LT / 32];
    const int warp = threadIdx.x >> 5;
    const int nz = a.nz;
    const int L = nz / G;                  // lanes per row
    const int rps = 32 / L;                // rows per step
    const int act = rps * L;
    const int rl = lane / L, gi = lane - (lane / L) * L;
    // dynamic work list: lane 0 takes item indices from a counter (reset by
    // the last block), one item ahead, so that warps that drew short items
    // take more; the result does not depend on the assignment because each
    // cell's sum of squares goes to the cell's slot
    unsigned *next_item = &a.sy->count[4];
    unsigned nxt = first;   // lane 0: the item k_adj drew before its wait
    int64_t it = __shfl_sync(FULL, nxt, 0);
    for (; it < a.n_adj; it = __shfl_sync(FULL, nxt, 0)) {
        if (lane == 0) nxt = atomicAdd(next_item, 1u);
        const int h = __ldg(a.adj_item + 2 * it);
        const int q0 = __ldg(a.adj_item + 2 * it + 1);
        const int64_t c0 = __ldg(a.cell_rptr + h);
        const int cnt = __ldg(a.cell_cnt + h);
        const int q1 = q0 + a.adj_chunk < cnt ? q0 + a.adj_chunk : cnt;
        const int32_t *rows = a.cell_rows + c0;
        const VT *vb = a.valB + c0 * nz + G * gi;
        AT acc[G];
#pragma unroll
        for (int t = 0; t < G; ++t) acc[t] = 0;
        int rn[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int q = q0 + rl + rps * u;
            rn[u] = (lane < act && q < q1) ? __ldg(rows + q) : -1;
        }
        const int step = rps * UN;
        const uint64_t step_bytes = (uint64_t)step * nz * sizeof(VT);
        for (int qb = q0; qb < q1; qb += step) {
            // lane 0 has the copy engine bring the next step's values into L2
            // (one step ahead: enough lead, few bytes held in L2)
            if (lane == 0 && qb + step < q1)
                prefetch_l2_bulk(a.valB + (c0 + qb + step) * nz,
                                 min((uint64_t)(q1 - qb - step) * nz * sizeof(VT), step_bytes));
            int rr[UN];
            AT uu[UN];
            AT vv[UN][G];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                rr[u] = rn[u];
                const int q = qb + rps * UN + rl + rps * u;
                rn[u] = (lane < act && q < q1) ? __ldg(rows + q) : -1;
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int q = qb + rl + rps * u;
                if (rr[u] >= 0) {
                    if (G == 4) {
                        typename Wide<VT>::T w4[4];
                        Pack4<VT>::ld(vb + (int64_t)q * nz, w4);
#pragma unroll
                        for (int t = 0; t < G; ++t) vv[u][t] = (AT)w4[t];
                    } else if (G % 2 == 0) {
#pragma unroll
                        for (int t2 = 0; t2 < G / 2; ++t2) {
                            typename Wide<VT>::T w2[2];
                            Pack2<VT>::ld(vb + (int64_t)q * nz + 2 * t2, w2);
                            vv[u][2 * t2] = (AT)w2[0];
                            vv[u][2 * t2 + 1] = (AT)w2[1];
                        }
                    } else {
                        vv[u][0] = (AT)ldval(vb + (int64_t)q * nz);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < G; ++t) vv[u][t] = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) uu[u] = rr[u] >= 0 ? (AT)__ldg(a.ubar + rr[u]) : (AT)0;
#pragma unroll
            for (int u = 0; u < UN; ++u)
#pragma unroll
                for (int t = 0; t < G; ++t) acc[t] += vv[u][t] * uu[u];
        }
        // per-depth sums over the rows of the step, in a fixed order
#pragma unroll
        for (int t = 0; t < G; ++t) red[warp][lane][t] = acc[t];
        __syncwarp();
        AT dot[2] = {0, 0};   // depths lane and lane + 32 (nz <= 64)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int k = lane + 32 * half;
            if (k < nz) {
                const int g = k / G, t = k - (k / G) * G;
                AT sum = 0;
                for (int r = 0; r < rps; ++r) sum += red[warp][g + L * r][t];
                dot[half] = sum;
            }
        }
        __syncwarp();
        const int nch = cnt > a.adj_chunk ? (cnt + a.adj_chunk - 1) / a.adj_chunk : 1;
        bool finish = true;
        if (nch > 1) {
            const int64_t first = it - q0 / a.adj_chunk;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int k = lane + 32 * half;
                if (k < nz) a.chunk_part[it * nz + k] = dot[half];
            }
            // the lanes' partial writes reach lane 0 through __syncwarp; its
            // acquire-release add publishes them and, for the last item of
            // the cell, orders the reads of the other items' partials (from
            // L2) after their writers' adds
            __syncwarp();
            if (lane == 0) {
                unsigned prev;
                asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;"
                             : "=r"(prev) : "l"(a.cell_done + h) : "memory");
                last_flag[warp] = prev == (unsigned)(nch - 1);
            }
            __syncwarp();
            finish = last_flag[warp] != 0;
            if (finish) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int k = lane + 32 * half;
                    if (k < nz) {
                        AT sum = 0;
                        for (int c = 0; c < nch; ++c)
                            sum += (AT)__ldcg(a.chunk_part + (first + c) * nz + k);
                        dot[half] = sum;
                    }
                }
                if (lane == 0) a.cell_done[h] = 0u;
            }
        }
        if (finish) {
            double css = 0.0;
            if (a.Pb) {
                css = adj_finish_blk(a, (int64_t)h, dot[0], ib, cv, wsm, lamr, init, lane);
            } else {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int k = lane + 32 * half;
                    if (k < nz)
                        css += adj_finish(a, (int64_t)h * nz + k, dot[half], ib, cv, wsm, lamr,
                                          init);
                }
            }
            // the cell's sum goes to its slot (which warp, and which of a
            // split cell's items, finishes it depends on arrival order); the
            // last block adds the slots in cell order
            css = warp_sum(css);
            if (lane == 0) a.cell_ss[h] = css;   // read by the last block after the grid barrier
        }
    }
    return 0.0;   // all sums went to the cell slots
}

// ------------------------------------------------------------- reductions

// v[i0] + v[i0 + st] + v[i0 + 2 st] + ... (i < n), added in that order, the
// loads issued eight at a time: one L2 round trip per eight terms instead of
// one per term (the last block's sums of block partials and cell slots were
// latency chains of up to 40 round trips, ~20 us per launch).  Slots past n
// add +0.0, which leaves a sum of squares unchanged bit for bit.
__device__ __forceinline__ double strided_sum(const double *v, int64_t n, int i0, int st) {
    double s = 0.0;
    for (int64_t i = i0; i < n; i += 8 * (int64_t)st) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = i + (int64_t)u * st < n ? __ldcg(v + i + (int64_t)u * st) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += t[u];
    }
    return s;
}

// Block sum of v, then the block that finishes last sums the per-block
// partials in index order.  Returns true in that block; `total` is valid in
// its first warp.
__device__ __forceinline__ bool grid_sum_last(double v, double *partial, unsigned *counter,
                                              double &total) {
    __shared__ double red[LT / 32];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += red[i];
        partial[blockIdx.x] = b;
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s = 0.0;
    if (warp == 0) {
        s = strided_sum(partial, (int64_t)gridDim.x, lane, 32);
        s = warp_sum(s);
    }
    if (threadIdx.x == 0) *counter = 0u;
    total = s;
    return true;
}

// Sum of v[0..n) by the calling block in a fixed order (thread t takes
// t, t + blockDim, ...; then warps in order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum_ordered(const double *v, int64_t n) {
    __shared__ double red2[LT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = strided_sum(v, n, (int)threadIdx.x, (int)blockDim.x);
    s = warp_sum(s);
    if (lane == 0) red2[warp] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red2[i];
    return t;
}

// ------------------------------------------------------------------ kernels

// beta_1 u_1 = [d; 0]: u-bar = [d; 0], beta_1 = ||d||, x = 0.
template <class ST>
__global__ void __launch_bounds__(LT) k_init(int64_t m, int64_t M, int32_t n,
                                             const double *__restrict__ d,
                                             const double *__restrict__ baug, ST *ubar, double *x,
                                             double *wv, double *partial, LsqrScalars *sc,
                                             LsqrSync *sy) {
    double ss = 0.0;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t0; i < M; i += st) {
        // b = [d; 0], or a full augmented right-hand side (refinement sweeps)
        double v = baug ? baug[i] : (i < m ? d[i] : 0.0);
        ubar[i] = (ST)v;
        ss += v * v;
    }
    for (int64_t j = t0; j < n; j += st) {
        x[j] = 0.0;
        wv[j] = 0.0;
    }
    double tot;
    if (grid_sum_last(ss, partial, &sy->count[0], tot) && threadIdx.x == 0) {
        const double b = sqrt(tot);
        sc->beta = b;
        sc->bnorm = b;
        sc->rnorm = b;
        sc->phibar = b;
        if (!isfinite(b)) sc->err = 1;
        if (!(b > 0.0) || !isfinite(b)) sc->done = 1;
    }
}

// Copy of the scalars by the calling threads (8-byte words).
__device__ __forceinline__ void copy_scalars(LsqrScalars *dst, const LsqrScalars *src, int t,
                                             int nt) {
    static_assert(sizeof(LsqrScalars) % 8 == 0, "LsqrScalars: whole 8-byte words");
    for (int i = t; i < (int)(sizeof(LsqrScalars) / 8); i += nt)
        reinterpret_cast<unsigned long long *>(dst)[i] =
            reinterpret_cast<const unsigned long long *>(src)[i];
}

// The scalar step the adjoint left pending (alpha_new = alpha_{i+1}), one
// warp, launched beside the next forward sweep: its chain of dependent FP64
// operations (B300's FP64 pipe is narrow) took ~17 us at the end of every
// adjoint sweep.  It works on a staging copy, since the forward reads the
// scalars meanwhile; k_upd, which follows both, publishes it.
__global__ void __launch_bounds__(32) k_step(const LsqrScalars *sc, LsqrScalars *stage) {
    if (!sc->step_pending || (sc->done | sc->istop)) return;
    copy_scalars(stage, sc, threadIdx.x, 32);
    __syncwarp();
    if (threadIdx.x == 0) {
        if (stage->method == 1) lsmr_step(stage, stage->alpha_next);
        else lsqr_step(stage, stage->alpha_next);
    }
}

// The damping sweep's pending steps, one per value still running, beside the
// forward: warp w advances values w, w + 8, ... on staging copies (published
// by k_upd_sweep); beta_{i+1} and alpha_{i+1} come from the shared scalars.
__global__ void __launch_bounds__(LT) k_step_sweep(const LsqrScalars *base, const LsqrScalars *ls,
                                                    LsqrScalars *stage, int L) {
    if (!base->step_pending || (base->done | base->istop)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < L; l += (int)(blockDim.x >> 5)) {
        copy_scalars(stage + l, ls + l, lane, 32);
        __syncwarp();
        if (lane == 0) {
            LsqrScalars *c = stage + l;
            if (!(c->done | c->istop)) {
                c->beta = base->beta;
                lsqr_step(c, base->alpha_next);
            }
        }
        __syncwarp();
    }
}

// u-bar <- (A v-bar)/alpha - (alpha/beta) u-bar;  beta <- ||u-bar||.  BF16
// values: three blocks per SM, as in the adjoint.
// PATH 6: a kernel of its own for the six-entry groups (nz % 6 == 0 off the
// quads, FP32 values), with two groups in flight instead of three (2.3 %
// faster on 18 depth nodes).  The generic kernel keeps the path too: without
// it the quads of 4 measured 9 % slower (a different schedule, although the
// generic kernel then no longer spilled).
template <class VT, class ST, int FMT, int MB = (sizeof(VT) == 2 ? 3 : 4), int PATH = 0>
__global__ void __launch_bounds__(LT, MB) k_fwd(OpArgs<VT, ST> a) {
    if constexpr (FMT == FMT_BLK) {
        // the first row's values do not depend on the adjoint: into L2 before the wait
        const int64_t gw0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t r0 = gw0 * FWD_RB + ((threadIdx.x >> 4) & 1);
        if ((threadIdx.x & 15) == 0 && r0 < a.m) {
            const int64_t e0 = __ldg(a.row_cptr + r0), e1 = __ldg(a.row_cptr + r0 + 1);
            prefetch_l2_bulk(a.val + e0 * (int64_t)a.nz, (uint64_t)(e1 - e0) * a.nz * sizeof(VT));
        }
    }
    pdl_wait();
    LsqrScalars *sc = a.sc;
    if (sc->done | sc->istop) return;
    using AT = ST;
    // alpha_{i+1} and beta_{i+1}: the scalar step of iteration i (k_step, run
    // beside this kernel) is not needed here
    const double alpha = sc->alpha_next, beta = sc->beta;
    const AT ia = alpha > 0.0 ? (AT)(1.0 / alpha) : (AT)0;
    const AT cu = beta > 0.0 ? (AT)(alpha / beta) : (AT)0;
    const AT wsm = (AT)sc->w_smooth, lamr = (AT)sc->lam_rows;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0.0;
    if constexpr (FMT == FMT_BLK) {
        if constexpr (PATH == 6)
            ss = fwd_rows_halfwarp<VT, ST, -6, 2>(a, ia, cu, gw, nw, lane);
        else
            ss = fwd_rows_blk<VT, ST>(a, ia, cu, gw, nw, lane);
    } else {
        for (int64_t r = gw; r < a.m; r += nw) {
            AT dot = dot_elem<VT, AT, ST>(a.row_ptr, a.col, a.val, a.vsc, r, lane);
            if (lane == 0) {
                AT u = dot * ia - cu * a.ubar[r];
                a.ubar[r] = u;
                ss += (double)u * (double)u;
            }
        }
    }
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = t0; j < a.n; j += st) {
        AT lap = laplace<AT, ST>(a.vsc, j, a.nx, a.ny, a.nz);
        ST *ur = a.ubar + a.m + j;
        AT u = wsm * lap * ia - cu * *ur;
        *ur = u;
        ss += (double)u * (double)u;
        if (a.lam_rows_on) {
            ST *ul = a.ubar + a.m + a.n + j;
            AT u2 = lamr * (AT)a.vsc[j] * ia - cu * *ul;
            *ul = u2;
            ss += (double)u2 * (double)u2;
        }
    }
    double tot;
    if (grid_sum_last(ss, a.partial, &a.sy->count[1], tot) && threadIdx.x == 0) {
        const double b = sqrt(tot);
        if (!isfinite(b)) {
            sc->err = 1;
            sc->done = 1;
        }
        // a pending step still reads beta_{i+1}: k_upd moves beta_next in
        // (the flag is read here, not kept live through the sweep: one more
        // live register cost the FP32 forward up to 4 % at 64 registers)
        if (sc->step_pending) sc->beta_next = b;
        else sc->beta = b;
    }
}

static __device__ void sweep_step(LsqrScalars *base, LsqrScalars *ls, int L, double an, int init) {
    // the values are independent: lane 0 of warp l advances values l, l + 8, ...
    // (their FP64 chains overlap), then thread 0 counts the running ones
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int l = warp; l < L; l += (int)(blockDim.x >> 5)) {
            LsqrScalars *c = ls + l;
            if (init) {
                c->beta = base->beta;
                c->bnorm = base->bnorm;
                c->rnorm = base->rnorm;
                c->phibar = base->phibar;
                c->alpha = an;
                c->rhobar = an;
                c->arnorm = an * base->beta;
                c->pending = 2;
                if (!(c->arnorm > 0.0)) c->done = 1;
            } else if (!(c->done | c->istop)) {
                c->beta = base->beta;
                lsqr_step(c, an);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int running = 0;
        for (int l = 0; l < L; ++l) {
            const LsqrScalars *c = ls + l;
            if (c->err) base->err = 1;
            running += !(c->done | c->istop);
        }
        base->alpha = an;
        if (!init) base->itn += 1;
        if (!running) {
            if (init) base->done = 1;
            else base->istop = 1;
        }
    }
}

// v-bar <- (A^T u-bar)/beta - (beta/alpha) v-bar;  alpha <- ||v-bar||, then
// the scalar recurrence (or its initialisation when init != 0).  With BF16
// values three blocks per SM (up to 85 registers) measured faster than four.
template <class VT, class ST, int FMT, int G>
__global__ void __launch_bounds__(LT, sizeof(VT) == 2 ? 3 : 4) k_adj(OpArgs<VT, ST> a, int init) {
    // the blocked sweep's first work item is drawn, and its first values sent
    // to L2, before the wait: the item counter was reset by the previous
    // adjoint, which completed before the kernel this one waits for started
    unsigned first = 0;
    if constexpr (FMT == FMT_BLK) {
        if ((threadIdx.x & 31) == 0) {
            first = atomicAdd(&a.sy->count[4], 1u);
            if (first < a.n_adj) {
                const int h0 = __ldg(a.adj_item + 2 * first), q0 = __ldg(a.adj_item + 2 * first + 1);
                const int cnt = __ldg(a.cell_cnt + h0);
                const int q1 = min(q0 + a.adj_chunk, cnt);
                if (q1 > q0)
                    prefetch_l2_bulk(a.valB + (__ldg(a.cell_rptr + h0) + q0) * (int64_t)a.nz,
                                     min((uint64_t)(q1 - q0) * a.nz * sizeof(VT), (uint64_t)4096));
            }
        }
    }
    pdl_wait();
    pdl_allow_next();
    LsqrScalars *sc = a.sc;
    if (sc->done | sc->istop) return;
    if (FMT == FMT_BLK && G != G_ANY && adj_group(a.nz) != G) {   // another depth count
        if (blockIdx.x == 0 && threadIdx.x == 0) sc->err = sc->done = 1;
        return;
    }
    using AT = ST;
    const double alpha = sc->alpha, beta = sc->beta;
    const bool skip = !init && !(beta > 0.0);
    const AT ib = beta > 0.0 ? (AT)(1.0 / beta) : (AT)0;
    const AT cv = init ? (AT)0 : (alpha > 0.0 ? (AT)(beta / alpha) : (AT)0);
    const AT wsm = (AT)sc->w_smooth, lamr = (AT)sc->lam_rows;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0.0;
    if (!skip) {
        if constexpr (FMT == FMT_BLK) {
            if constexpr (G == G_ANY) {
                switch (adj_group(a.nz)) {
                case 4: ss = adj_cells_chunked<VT, ST, 4>(a, ib, cv, wsm, lamr, init, gw, nw, lane, first); break;
                case 6: ss = adj_cells_chunked<VT, ST, 6>(a, ib, cv, wsm, lamr, init, gw, nw, lane, first); break;
                case 2: ss = adj_cells_chunked<VT, ST, 2>(a, ib, cv, wsm, lamr, init, gw, nw, lane, first); break;
                default: ss = adj_cells_chunked<VT, ST, 1>(a, ib, cv, wsm, lamr, init, gw, nw, lane, first);
                }
            } else {
                ss = adj_cells_chunked<VT, ST, (G > 0 ? G : 1)>(a, ib, cv, wsm, lamr, init, gw, nw,
                                                                lane, first);
            }
        } else {
            for (int64_t j = gw; j < a.n; j += nw) {
                AT dot = dot_elem<VT, AT, ST>(a.col_ptr, a.row_idx, a.valT, a.ubar, j, lane);
                if (lane == 0) ss += adj_finish(a, j, dot, ib, cv, wsm, lamr, init);
            }
        }
    }
    double tot;
    const bool last = grid_sum_last(ss, a.partial + MAXBLK, &a.sy->count[2], tot);
    if (!last) return;
    // the blocked sweep's sums, in cell order
    const double cells = (FMT == FMT_BLK && !skip) ? block_sum_ordered(a.cell_ss, a.n_cells) : 0.0;
    if (a.n_lam > 0) {
        // damping sweep: the start step here (one warp per damping value); later
        // steps are left pending for k_step_sweep, beside the next forward
        __shared__ double an_s;
        if (threadIdx.x == 0) {
            if (FMT == FMT_BLK) a.sy->count[4] = 0u;   // adjoint work counter for the next launch
            an_s = skip ? alpha : sqrt(tot + cells);
            if (!isfinite(an_s)) sc->err = sc->done = 1;
            sc->alpha_next = an_s;
            if (!init && isfinite(an_s)) {
                // the values' states as the last k_upd_sweep published them: the
                // sweep stops one adjoint after its last value stopped
                int running = 0;
                for (int l = 0; l < a.n_lam; ++l) {
                    const LsqrScalars *c = a.lam_sc + l;
                    if (c->err) sc->err = 1;
                    running += !(c->done | c->istop);
                }
                sc->alpha = an_s;
                sc->itn += 1;
                if (running) sc->step_pending = 1;
                else sc->istop = 1;
            }
        }
        if (init) {
            __syncthreads();
            if (isfinite(an_s)) sweep_step(sc, a.lam_sc, a.n_lam, an_s, init);
        }
        return;
    }
    if (threadIdx.x == 0) {
        if (FMT == FMT_BLK) a.sy->count[4] = 0u;   // adjoint work counter for the next launch
        tot += cells;
        double an = skip ? alpha : sqrt(tot);
        if (!isfinite(an)) {
            sc->err = 1;
            sc->done = 1;
            return;
        }
        sc->alpha_next = an;
        if (init) {
            sc->alpha = an;
            sc->rhobar = an;
            sc->arnorm = an * beta;
            sc->pending = 2;
            if (sc->method == 1) lsmr_init(sc, an);
            if (!(sc->arnorm > 0.0)) sc->done = 1;
        } else {
            sc->step_pending = 1;   // the scalar step runs in k_step
        }
    }
}

// The LSQR update of one column with fixed rounding (explicit round-to-nearest
// operations, so that every kernel that applies it gives the same bits):
// v = v-bar / alpha; start step: w = v; otherwise x += t1 w, w = v + t2 w.
__device__ __forceinline__ void lsqr_xw(double vbar_j, double ia, double t1, double t2, int pend,
                                        double &x, double &w) {
    const double v = __dmul_rn(vbar_j, ia);
    if (pend == 2) {
        w = v;
    } else {
        x = __fma_rn(t1, w, x);
        w = __fma_rn(t2, w, v);
    }
}

// Publication of a deferred step (k_step's copy) by one block: everything but
// beta, which the forward that ran beside k_step left in beta_next, and the
// forward's error flags, which are kept.
__device__ __forceinline__ void publish_step(LsqrScalars *sc, const LsqrScalars *stage) {
    __shared__ double bnext;
    __shared__ int err, done;
    if (threadIdx.x == 0) {
        bnext = sc->beta_next;
        err = sc->err;
        done = sc->done;
    }
    __syncthreads();
    copy_scalars(sc, stage, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        sc->beta = bnext;
        sc->err |= err;
        sc->done |= done;
        sc->step_pending = 0;
    }
    __syncthreads();
}

// LSQR: x += t1 w; w = v + t2 w (FP64), v = v-bar/alpha;  ||w||^2.
// LSMR (wv holds h): hbar = h - t1 hbar; x += t2 hbar; h = v - t3 h;  ||x||^2,
// then the stopping tests on the new ||x|| (last block).  The coefficients
// come from k_step's copy when a deferred step is pending; the last block
// (block 0 when there is no update) then publishes it -- or, with defer = 1
// (the update running on k_step's branch beside the forward, which still
// writes beta), leaves its results in the copy for k_pub to publish.
template <class ST>
__global__ void __launch_bounds__(LT) k_upd(int32_t n, const ST *__restrict__ vbar, double *x,
                                            double *wv, double *hbar, double *partial,
                                            LsqrScalars *sc, LsqrScalars *stage, LsqrSync *sy,
                                            int defer = 0) {
    const bool pub = sc->step_pending != 0;
    const LsqrScalars *src = pub ? stage : sc;
    const int pend = src->pending;
    if (!pend) {
        if (pub && !defer && blockIdx.x == 0) publish_step(sc, stage);
        return;
    }
    // where the last block leaves the results: the copy when publishing later
    LsqrScalars *dst = (pub && defer) ? stage : sc;
    const double alpha = src->alpha;
    const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
    const double t1 = src->t1, t2 = src->t2;
    double ss = 0.0;
    if (src->method == 1) {
        const double t3 = src->t3;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            const double v = (double)vbar[j] * ia;
            double h = wv[j], xj = x[j];
            if (pend == 2) {
                h = v;
                hbar[j] = 0.0;
            } else {
                const double hb = h - t1 * hbar[j];
                hbar[j] = hb;
                xj += t2 * hb;
                x[j] = xj;
                h = v - t3 * h;
            }
            wv[j] = h;
            ss += xj * xj;
        }
        double tot;
        if (grid_sum_last(ss, partial + 2 * MAXBLK, &sy->count[3], tot)) {
            if (pub && !defer) publish_step(sc, stage);
            if (threadIdx.x == 0) {
                dst->xnorm = sqrt(tot);
                if (pend != 2) stop_tests(dst);
                dst->pending = 0;
            }
        }
        return;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double w = wv[j], xj = x[j];
        lsqr_xw((double)vbar[j], ia, t1, t2, pend, xj, w);
        if (pend != 2) x[j] = xj;
        wv[j] = w;
        ss = __fma_rn(w, w, ss);
    }
    double tot;
    if (grid_sum_last(ss, partial + 2 * MAXBLK, &sy->count[3], tot)) {
        if (pub && !defer) publish_step(sc, stage);
        if (threadIdx.x == 0) {
            dst->wnorm2 = tot;
            dst->pending = 0;
        }
    }
}

// The damping sweep's shared scalars after a deferred k_upd_sweep: beta_{i+2},
// which the forward left aside, moves in (one thread, after the join).
__global__ void k_pub_base(LsqrScalars *base) {
    if (threadIdx.x == 0 && base->step_pending) {
        base->beta = base->beta_next;
        base->step_pending = 0;
    }
}

// Publication of the step that k_step and a deferred k_upd left in the copy
// (one block, once both branches of the iteration have joined: the forward
// wrote beta_{i+2} beside them).
__global__ void __launch_bounds__(LT) k_pub(LsqrScalars *sc, const LsqrScalars *stage) {
    pdl_allow_next();
    if (sc->step_pending) publish_step(sc, stage);
}


// Damping sweep, y-slice l of the grid: x_l += t1 w_l; w_l = v + t2 w_l with
// damping value l's coefficients (from k_step_sweep's copy when a step is
// pending; the slice's last block publishes it); ||w_l||^2 to its recurrence.
// Every block then arrives on counters[L]; the last one moves beta_next into
// the shared scalars (all blocks have read step_pending by then) -- unless
// defer = 1 (the update running beside the forward, which still writes
// beta_next): then k_pub_base does that after the join.
template <class ST>
__global__ void __launch_bounds__(LT) k_upd_sweep(int32_t n, const ST *__restrict__ vbar, double *X,
                                                  double *W, double *partial, LsqrScalars *base,
                                                  LsqrScalars *ls, LsqrScalars *stage, int L,
                                                  unsigned *counters, int defer = 0) {
    const int l = blockIdx.y;
    const bool pub = base->step_pending != 0;
    LsqrScalars *sc = ls + l;
    const LsqrScalars *src = pub ? stage + l : sc;
    const int pend = src->pending;
    if (pend) {
        const double alpha = src->alpha;
        const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
        const double t1 = src->t1, t2 = src->t2;
        double *x = X + (int64_t)l * n, *wv = W + (int64_t)l * n;
        double ss = 0.0;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            double w = wv[j], xj = x[j];
            lsqr_xw((double)vbar[j], ia, t1, t2, pend, xj, w);
            if (pend != 2) x[j] = xj;
            wv[j] = w;
            ss = __fma_rn(w, w, ss);
        }
        double tot;
        if (grid_sum_last(ss, partial + (int64_t)l * MAXBLK, counters + l, tot)) {
            if (pub) {
                copy_scalars(sc, stage + l, threadIdx.x, blockDim.x);
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                sc->wnorm2 = tot;
                sc->pending = 0;
            }
        }
    } else if (pub && blockIdx.x == 0) {
        copy_scalars(sc, stage + l, threadIdx.x, blockDim.x);   // stopped or broken down
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counters + L, 1u);
        if (t == gridDim.x * gridDim.y - 1) {
            counters[L] = 0u;
            if (pub && !defer) {
                base->beta = base->beta_next;
                base->step_pending = 0;
            }
        }
    }
}

__global__ void k_finalize(int32_t n, const double *__restrict__ x, const double *__restrict__ D,
                           double *m_out, int accumulate = 0) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double v = D ? D[j] * x[j] : x[j];
        m_out[j] = accumulate ? m_out[j] + v : v;
    }
}

// (P y)_j = sum_{i >= k} P_h[k][i] y_{h nz + i}  (j = h nz + k; P_h upper
// triangular, in the precision the solve used, widened to FP64).
template <class ST>
__device__ __forceinline__ double blk_apply_row(const ST *__restrict__ P,
                                                const double *__restrict__ y, int64_t j, int nz) {
    const int64_t h = j / nz;
    const int k = (int)(j - h * nz);
    const ST *Pr = P + (h * nz + k) * nz;
    const double *yh = y + h * nz;
    double s = 0.0;
    for (int i = k; i < nz; ++i) s += (double)Pr[i] * yh[i];
    return s;
}

// m = P x (or m += P x) with the depth-block preconditioner.
template <class ST>
__global__ void k_finalize_blk(int32_t n, int nz, const double *__restrict__ x,
                               const ST *__restrict__ P, double *m_out, int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double v = blk_apply_row(P, x, j, nz);
        m_out[j] = accumulate ? m_out[j] + v : v;
    }
}

// y = G x or G^T x with FP64 vectors (pdst_apply_G).
template <class VT, int FMT>
__global__ void __launch_bounds__(LT) k_spmv(OpArgs<VT, double> a, int trans,
                                             const double *__restrict__ xin, double *y) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t rows = trans ? a.n : a.m;
    for (int64_t r = gw; r < rows; r += nw) {
        double s;
        if (!trans)
            s = FMT == FMT_ELEM ? dot_elem<VT, double, double>(a.row_ptr, a.col, a.val, xin, r, lane)
                                : dot_blk_row<VT, double, double>(a.row_cptr, a.row_cells, a.val,
                                                                  xin, r, a.nz, lane);
        else
            s = FMT == FMT_ELEM
                    ? dot_elem<VT, double, double>(a.col_ptr, a.row_idx, a.valT, xin, r, lane)
                    : dot_blk_col<VT, double, double>(a.cell_rptr, a.cell_cnt, a.cell_rows,
                                                      a.valB, xin, r, a.nz, lane);
        if (lane == 0) y[r] = s;
    }
}

// ||[G; w L; lam I]_{:,j}||^2 -> D_j = 1/sqrt(.)  (column-norm scaling).
template <class VT>
__global__ void __launch_bounds__(LT) k_colnorm_scale(OpArgs<VT, double> a, double w, double lam,
                                                      double *D, int mode, double pw) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < a.n; j += nw) {
        const int64_t h = j / a.nz;
        const int k = (int)(j - h * a.nz);
        const int64_t c0 = a.cell_rptr[h];
        const int cnt = a.cell_cnt[h];
        const VT *v = a.valB + c0 * a.nz + k;
        double s = 0.0;
        for (int q = lane; q < cnt; q += 32) {
            double t = (double)widen(v[(int64_t)q * a.nz]);
            s += t * t;
        }
        s = warp_sum(s);
        if (lane == 0) {
            const int ix = (int)(h % a.nx), iy = (int)(h / a.nx);
            const int deg = (k > 0) + (k < a.nz - 1) + (ix > 0) + (ix < a.nx - 1) + (iy > 0) +
                            (iy < a.ny - 1);
            const double c = s + w * w * ((double)deg * deg + deg) + lam * lam;
            // mode 0: 1/||A_:j||; 1: ||A_:j||^(-pw); 2: ||A_:j||
            if (mode == 0) D[j] = c > 0.0 ? 1.0 / sqrt(c) : 1.0;
            else if (mode == 1) D[j] = c > 0.0 ? pow(c, -0.5 * pw) : 1.0;
            else D[j] = sqrt(c);
        }
    }
}

// ------------------------------------------------------------------- driver

struct LsqrWork {
    int dtype = -1, format = -1, lamrows = -1;
    int blk = 0;                     // the solve runs with the depth-block preconditioner
    const void *graph_D = nullptr;
    int64_t M = 0;
    DevBuf ubar, vbar, vsc, x, wv, hbar, partial, scal, sync, chunk_part, cell_done, cell_ss;
    DevBuf ones, baug, corr;         // refinement: unit scaling, augmented residual, norms
    DevBuf sw_x, sw_w, sw_sc, sw_part, sw_cnt;   // damping sweep: x, w, scalars per value
    DevBuf sw_stage;                             // damping sweep: k_step_sweep's copies
    LsqrScalars *h_scal = nullptr;   // pinned
    unsigned grid_rows = 0, grid_cols = 0, grid_vec = 0;
    std::map<int, cudaGraphExec_t> graphs;   // key: kblock (+ PROF_KEY with event nodes)
    std::vector<cudaEvent_t> prof_ev;        // event nodes of the profiled graph (4 per iteration)
    cudaStream_t side = nullptr;             // k_step beside k_fwd
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~LsqrWork() {
        for (auto &g : graphs)
            if (g.second) cudaGraphExecDestroy(g.second);
        for (auto e : prof_ev) cudaEventDestroy(e);
        if (h_scal) cudaFreeHost(h_scal);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
};

void destroy_work(LsqrWork *w) { delete w; }

template <class VT, class ST>
static OpArgs<VT, ST> make_args(pdst_handle *h, int dtype, LsqrWork *w, bool scaled, bool lamrows) {
    OpArgs<VT, ST> a{};
    a.m = h->m;
    a.n = h->n;
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.nz = h->nz;
    a.row_ptr = h->row_ptr.as<int64_t>();
    a.col = h->col.as<int32_t>();
    a.col_ptr = h->col_ptr.as<int64_t>();
    a.row_idx = h->row_idx.as<int32_t>();
    a.row_cptr = h->row_cptr.as<int64_t>();
    a.row_cells = h->row_cells.as<int32_t>();
    a.cell_rptr = h->cell_rptr.as<int64_t>();
    a.cell_rows = h->cell_rows.as<int32_t>();
    a.cell_cnt = h->cell_cnt.as<int32_t>();
    a.cell_order = h->cell_order.as<int32_t>();
    a.val = h->vals[dtype].csr.as<VT>();
    a.valT = h->vals[dtype].csc.as<VT>();
    a.valB = h->vals[dtype].bcsc.as<VT>();
    a.adj_item = h->adj_item.as<int32_t>();
    a.adj_chunk = h->adj_chunk;
    a.n_cells = h->H;
    a.n_adj = h->n_adj;
    a.D = scaled ? h->colscale.as<double>() : nullptr;
    a.Pb = a.PbT = nullptr;
    if (w && w->blk) {
        a.D = nullptr;
        a.Pb = sizeof(ST) == sizeof(double) ? h->blkP64.p : h->blkP32.p;
        a.PbT = sizeof(ST) == sizeof(double) ? h->blkP64T.p : h->blkP32T.p;
    }
    a.lam_rows_on = lamrows ? 1 : 0;
    if (w) {
        a.ubar = w->ubar.as<ST>();
        a.vbar = w->vbar.as<ST>();
        a.vsc = scaled ? w->vsc.as<ST>() : w->vbar.as<ST>();
        a.x = w->x.as<double>();
        a.wv = w->wv.as<double>();
        a.hbar = w->hbar.as<double>();
        a.partial = w->partial.as<double>();
        a.sc = w->scal.as<LsqrScalars>();
        a.sc_stage = a.sc + 1;
        a.sy = w->sync.as<LsqrSync>();
        a.chunk_part = w->chunk_part.as<ST>();
        a.cell_done = w->cell_done.as<unsigned>();
        a.cell_ss = w->cell_ss.as<double>();
    }
    return a;
}

// The blocked adjoint kernel for a handle's depth count.
template <class VT, class ST, int FMT> static auto adj_kernel(int nz) {
    if constexpr (FMT == FMT_BLK) {
        const int g = adj_group(nz);
        if (g == 2) return k_adj<VT, ST, FMT, 2>;
        if (g == 1) return k_adj<VT, ST, FMT, 1>;
    }
    return k_adj<VT, ST, FMT, G_ANY>;
}

// The forward kernel for a handle.  With FP32 values three blocks per SM (up
// to 85 registers) against four, measured per depth path on B300: run-time
// quads -7 % (nz = 12) and -18 % (24), compile-time quads of 5 -12 % (20),
// pairs -6 % (10); but quads of 4 +2 % (16), six-entry groups +12 % (18) and
// one entry per lane +19 % (15), which keep four (as do quads of 2, nz = 8).
__host__ __device__ constexpr bool fwd_three_blocks(int nz) {
    return (nz & 3) == 0 ? (nz != 16 && nz != 8) : ((nz & 1) == 0 && nz % 6 != 0);
}
template <class VT, class ST, int FMT> static auto fwd_kernel(int nz) {
    if constexpr (FMT == FMT_BLK && sizeof(VT) == 4 && sizeof(ST) == 4) {
        if ((nz & 3) != 0 && nz % 6 == 0) return k_fwd<VT, ST, FMT, 4, 6>;
        if (fwd_three_blocks(nz)) return k_fwd<VT, ST, FMT, 3>;
    }
    return k_fwd<VT, ST, FMT>;
}

constexpr int PROF_KEY = 1 << 20;   // graph cache key offset of the profiled graphs

template <class K> static unsigned persistent_grid(K kernel, int device, int64_t work_items) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, LT, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)num_sms(device) * per_sm;
    int64_t need = (work_items + LT - 1) / LT;
    if (need < 1) need = 1;
    if (g > need) g = need;
    if (g > MAXBLK) g = MAXBLK;
    return (unsigned)g;
}

// The forward's grid: one block short of a full persistent grid, so that
// k_step (one warp, launched beside it) always finds a free slot.
template <class K> static unsigned fwd_grid(K kernel, int device, int64_t work_items) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, LT, 0);
    const unsigned g = persistent_grid(kernel, device, work_items);
    const int64_t full = (int64_t)num_sms(device) * (per_sm < 1 ? 1 : per_sm);
    return (g > 1 && (int64_t)g >= full) ? g - 1 : g;
}

struct RunStats {
    int launches = 0, profiled_iters = 0;
    double fwd_ms = 0, adj_ms = 0, upd_ms = 0;
};

template <class VT, class ST, int FMT> struct Solver {
    using VTy = VT;
    using STy = ST;
    static constexpr int FMTv = FMT;
    static pdst_status prepare(pdst_handle *h, LsqrWork *w, bool lamrows) {
        const int64_t M = h->m + h->n + (lamrows ? h->n : 0);
        PDST_TRY(w->ubar.alloc(sizeof(ST) * std::max<int64_t>(M, 1)));
        PDST_TRY(w->vbar.alloc(sizeof(ST) * std::max<int32_t>(h->n, 1)));
        PDST_TRY(w->vsc.alloc(sizeof(ST) * std::max<int32_t>(h->n, 1)));
        PDST_TRY(w->x.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
        PDST_TRY(w->wv.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
        PDST_TRY(w->hbar.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
        PDST_TRY(w->partial.alloc(sizeof(double) * 3 * MAXBLK));
        PDST_TRY(w->scal.alloc(2 * sizeof(LsqrScalars)));   // scalars, k_step's copy
        PDST_TRY(w->sync.alloc(sizeof(LsqrSync)));
        PDST_TRY(w->chunk_part.alloc(sizeof(ST) * std::max<int64_t>(h->n_adj * h->nz, 1)));
        PDST_TRY(w->cell_done.alloc(sizeof(unsigned) * std::max<int32_t>(h->H, 1)));
        PDST_TRY(w->cell_ss.alloc(sizeof(double) * std::max<int32_t>(h->H, 1)));
        PDST_CUDA(cudaMemset(w->cell_ss.p, 0, sizeof(double) * std::max<int32_t>(h->H, 1)));
        if (!w->h_scal) PDST_CUDA(cudaMallocHost(&w->h_scal, sizeof(LsqrScalars)));
        w->M = M;
        // warp-per-row kernels: items = rows * 32 threads
        w->grid_rows = fwd_grid(fwd_kernel<VT, ST, FMT>(h->nz), h->device, (h->m + h->n) * 32);
        if (!w->side) PDST_CUDA(cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking));
        if (!w->ev_fork) PDST_CUDA(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
        if (!w->ev_join) PDST_CUDA(cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming));
        w->grid_cols = persistent_grid(adj_kernel<VT, ST, FMT>(h->nz), h->device, (int64_t)h->n * 32);
        w->grid_vec = persistent_grid(k_upd<ST>, h->device, h->n);
        return PDST_OK;
    }

    // One iteration: the previous adjoint's scalar step (k_step) and its x/w
    // update (k_upd, which reads v-bar_{i+1}) on a side stream, beside the
    // forward, which needs only alpha_{i+1}; then, once both branches are
    // done, k_pub publishes the step and the adjoint overwrites v-bar.
    // (Profile mode 1 and the allocation-free solve run the same kernels in
    // line with k_upd publishing; the arithmetic, and so every bit, is the same.)
    static void fork_step(LsqrWork *w, const OpArgs<VT, ST> &a, cudaStream_t s) {
        cudaEventRecord(w->ev_fork, s);
        cudaStreamWaitEvent(w->side, w->ev_fork, 0);
        k_step<<<1, 32, 0, w->side>>>(a.sc, a.sc_stage);
        cudaEventRecord(w->ev_join, w->side);
    }
    // The scalar step and then the x/w update on the side branch (the update
    // reads v-bar and writes x and w, which the forward does not touch; it
    // leaves its results in the step's copy), beside the forward.
    static void fork_step_update(pdst_handle *h, LsqrWork *w, const OpArgs<VT, ST> &a,
                                 cudaStream_t s) {
        cudaEventRecord(w->ev_fork, s);
        cudaStreamWaitEvent(w->side, w->ev_fork, 0);
        k_step<<<1, 32, 0, w->side>>>(a.sc, a.sc_stage);
        k_upd<ST><<<w->grid_vec, LT, 0, w->side>>>(h->n, a.vbar, a.x, a.wv, a.hbar, a.partial,
                                                   a.sc, a.sc_stage, a.sy, 1);
        cudaEventRecord(w->ev_join, w->side);
    }
    // ev (profile mode 2): four events recorded around the forward, the
    // update and the adjoint on the main stream, captured as event-record
    // nodes (external records: a plain record inside a capture only orders).
    // A sweep launched with programmatic stream serialisation (see pdl_wait):
    // the forward directly after the previous adjoint, the adjoint directly
    // after k_pub.  Profile mode 2 puts event nodes between them and launches
    // plainly.
    template <class K, class... Args>
    static void launch_dep(K kernel, unsigned grid, cudaStream_t s, bool pdl, Args... args) {
        if (!pdl) {
            kernel<<<grid, LT, 0, s>>>(args...);
            return;
        }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(LT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, kernel, args...);
    }
    static void launch_iter(pdst_handle *h, LsqrWork *w, const OpArgs<VT, ST> &a, cudaStream_t s,
                            const cudaEvent_t *ev = nullptr) {
        const bool pdl = ev == nullptr;
        fork_step_update(h, w, a, s);
        if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
        launch_dep(fwd_kernel<VT, ST, FMT>(h->nz), w->grid_rows, s, pdl, a);
        if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
        cudaStreamWaitEvent(s, w->ev_join, 0);
        k_pub<<<1, LT, 0, s>>>(a.sc, a.sc_stage);
        if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
        launch_dep(adj_kernel<VT, ST, FMT>(h->nz), w->grid_cols, s, pdl, a, 0);
        if (ev) cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal);
    }

    // Per-kernel device time of `iters` plain-launched iterations, each kernel
    // bracketed by CUDA events on the launching stream.  k_step runs in line
    // here (so the forward's time is its own) and counts with the update.
    static pdst_status profiled_block(pdst_handle *h, LsqrWork *w, const OpArgs<VT, ST> &a,
                                      int iters, cudaStream_t s, RunStats &rs) {
        constexpr int E = 5;
        std::vector<cudaEvent_t> ev(E * (size_t)iters);
        for (auto &e : ev) PDST_CUDA(cudaEventCreate(&e));
        for (int i = 0; i < iters; ++i) {
            cudaEventRecord(ev[E * i], s);
            k_step<<<1, 32, 0, s>>>(a.sc, a.sc_stage);
            cudaEventRecord(ev[E * i + 1], s);
            fwd_kernel<VT, ST, FMT>(h->nz)<<<w->grid_rows, LT, 0, s>>>(a);
            cudaEventRecord(ev[E * i + 2], s);
            k_upd<ST><<<w->grid_vec, LT, 0, s>>>(h->n, a.vbar, a.x, a.wv, a.hbar, a.partial, a.sc,
                                                 a.sc_stage, a.sy);
            cudaEventRecord(ev[E * i + 3], s);
            adj_kernel<VT, ST, FMT>(h->nz)<<<w->grid_cols, LT, 0, s>>>(a, 0);
            cudaEventRecord(ev[E * i + 4], s);
        }
        PDST_CUDA(cudaGetLastError());
        PDST_CUDA(cudaStreamSynchronize(s));
        rs.launches += 4 * iters;
        for (int i = 0; i < iters; ++i) {
            float ts = 0.f, tf = 0.f, tu = 0.f, ta = 0.f;
            cudaEventElapsedTime(&ts, ev[E * i], ev[E * i + 1]);
            cudaEventElapsedTime(&tf, ev[E * i + 1], ev[E * i + 2]);
            cudaEventElapsedTime(&tu, ev[E * i + 2], ev[E * i + 3]);
            cudaEventElapsedTime(&ta, ev[E * i + 3], ev[E * i + 4]);
            rs.fwd_ms += tf;
            rs.adj_ms += ta;
            rs.upd_ms += ts + tu;
        }
        for (auto &e : ev) cudaEventDestroy(e);
        return PDST_OK;
    }

    static pdst_status run(pdst_handle *h, LsqrWork *w, int dtype, bool scaled, bool lamrows,
                           const double *d, const LsqrScalars &init, int kblock, bool use_graph,
                           int profile, double *m_out, cudaStream_t s, RunStats &rs,
                           const double *baug = nullptr, bool accumulate = false,
                           const double *Dover = nullptr) {
        OpArgs<VT, ST> a = make_args<VT, ST>(h, dtype, w, scaled, lamrows);
        if (Dover) a.D = Dover;
        PDST_CUDA(cudaMemsetAsync(w->sync.p, 0, sizeof(LsqrSync), s));
        PDST_CUDA(cudaMemsetAsync(w->cell_done.p, 0, sizeof(unsigned) * std::max<int32_t>(h->H, 1), s));
        *w->h_scal = init;
        PDST_CUDA(cudaMemcpyAsync(w->scal.p, w->h_scal, sizeof(LsqrScalars),
                                  cudaMemcpyHostToDevice, s));
        unsigned ginit = persistent_grid(k_init<ST>, h->device, w->M);
        k_init<ST><<<ginit, LT, 0, s>>>(h->m, w->M, h->n, d, baug, a.ubar, a.x, a.wv, a.partial, a.sc,
                                        a.sy);
        adj_kernel<VT, ST, FMT>(h->nz)<<<w->grid_cols, LT, 0, s>>>(a, 1);
        k_upd<ST><<<w->grid_vec, LT, 0, s>>>(h->n, a.vbar, a.x, a.wv, a.hbar, a.partial, a.sc,
                                             a.sc_stage, a.sy);
        PDST_CUDA(cudaGetLastError());
        rs.launches += 3;

        // profile 2: the graph replay itself, with event nodes around each kernel
        const bool in_graph_prof = profile == 2;
        cudaGraphExec_t exec = nullptr;
        if (use_graph && profile != 1) {
            const int key = kblock + (in_graph_prof ? PROF_KEY : 0);
            auto it = w->graphs.find(key);
            if (it != w->graphs.end()) {
                exec = it->second;
            } else {
                if (in_graph_prof && w->prof_ev.size() < 4 * (size_t)kblock) {
                    // profiled graphs captured earlier hold the old events
                    for (auto g = w->graphs.begin(); g != w->graphs.end();) {
                        if (g->first >= PROF_KEY) {
                            if (g->second) cudaGraphExecDestroy(g->second);
                            g = w->graphs.erase(g);
                        } else {
                            ++g;
                        }
                    }
                    for (auto e : w->prof_ev) cudaEventDestroy(e);
                    w->prof_ev.assign(4 * (size_t)kblock, nullptr);
                    for (auto &e : w->prof_ev) PDST_CUDA(cudaEventCreate(&e));
                }
                cudaStream_t cs;
                PDST_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    for (int i = 0; i < kblock; ++i)
                        launch_iter(h, w, a, cs, in_graph_prof ? &w->prof_ev[4 * (size_t)i] : nullptr);
                    e = cudaStreamEndCapture(cs, &g);
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                if (e != cudaSuccess) {
                    set_error("LSQR graph capture: %s", cudaGetErrorString(e));
                    return PDST_ERR_CUDA;
                }
                w->graphs[key] = exec;
            }
        }
        int prof_it0 = -1;   // iteration count before the last profiled replay
        for (;;) {
            PDST_CUDA(cudaMemcpyAsync(w->h_scal, w->scal.p, sizeof(LsqrScalars),
                                      cudaMemcpyDeviceToHost, s));
            PDST_CUDA(cudaStreamSynchronize(s));
            const LsqrScalars &c = *w->h_scal;
            if (prof_it0 >= 0) {
                // only the iterations that ran (later kernels of a replay return at entry)
                const int ran = std::min(c.itn - prof_it0, kblock);
                for (int i = 0; i < ran; ++i) {
                    float tf = 0.f, tu = 0.f, ta = 0.f;
                    const cudaEvent_t *ev = &w->prof_ev[4 * (size_t)i];
                    PDST_CUDA(cudaEventElapsedTime(&tf, ev[0], ev[1]));
                    PDST_CUDA(cudaEventElapsedTime(&tu, ev[1], ev[2]));
                    PDST_CUDA(cudaEventElapsedTime(&ta, ev[2], ev[3]));
                    rs.fwd_ms += tf;
                    rs.upd_ms += tu;
                    rs.adj_ms += ta;
                }
                rs.profiled_iters += std::max(ran, 0);
                prof_it0 = -1;
            }
            if (c.done || c.istop || c.itn >= c.itmax) break;
            if (profile == 1) {
                PDST_TRY(profiled_block(h, w, a, 1, s, rs));
            } else if (exec) {
                if (in_graph_prof) prof_it0 = c.itn;
                PDST_CUDA(cudaGraphLaunch(exec, s));
                rs.launches += 5 * kblock;   // k_step, k_upd, k_fwd, k_pub, k_adj
            } else {
                for (int i = 0; i < kblock; ++i) launch_iter(h, w, a, s);
                PDST_CUDA(cudaGetLastError());
                rs.launches += 5 * kblock;   // k_step, k_upd, k_fwd, k_pub, k_adj
            }
        }
        if (a.Pb)
            k_finalize_blk<ST><<<w->grid_vec, LT, 0, s>>>(h->n, h->nz, a.x,
                                                          static_cast<const ST *>(a.Pb), m_out,
                                                          accumulate ? 1 : 0);
        else
            k_finalize<<<w->grid_vec, LT, 0, s>>>(h->n, a.x, a.D, m_out, accumulate ? 1 : 0);
        PDST_CUDA(cudaGetLastError());
        rs.launches += 1;
        PDST_CUDA(cudaMemcpyAsync(w->h_scal, w->scal.p, sizeof(LsqrScalars),
                                  cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        if (profile == 1) rs.profiled_iters = w->h_scal->itn;
        return PDST_OK;
    }
};

template <class VT, class ST, int FMT>
static pdst_status dispatch_run(pdst_handle *h, LsqrWork *w, int dtype, bool scaled, bool lamrows,
                                const double *d, const LsqrScalars &init, int kblock,
                                bool use_graph, int profile, double *m_out, cudaStream_t s,
                                bool fresh, RunStats &rs, const double *baug = nullptr,
                                bool accumulate = false, const double *Dover = nullptr) {
    if (fresh) PDST_TRY((Solver<VT, ST, FMT>::prepare(h, w, lamrows)));
    return Solver<VT, ST, FMT>::run(h, w, dtype, scaled, lamrows, d, init, kblock, use_graph,
                                    profile, m_out, s, rs, baug, accumulate, Dover);
}

// ------------------------------------------------ mixed-precision refinement

// FP64 residual of the augmented system at the current model m:
// baug = [d - G m; -w L m; -lam m] (lam rows only when lamrows).
template <int FMT>
__global__ void __launch_bounds__(LT) k_resid(OpArgs<double, double> a, const double *__restrict__ d,
                                              const double *__restrict__ mv, double w, double lam,
                                              int lamrows, double *baug) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw; r < a.m; r += nw) {
        const double y = FMT == FMT_ELEM
                             ? dot_elem<double, double, double>(a.row_ptr, a.col, a.val, mv, r, lane)
                             : dot_blk_row<double, double, double>(a.row_cptr, a.row_cells, a.val,
                                                                   mv, r, a.nz, lane);
        if (lane == 0) baug[r] = d[r] - y;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        baug[a.m + j] = -w * laplace<double, double>(mv, j, a.nx, a.ny, a.nz);
        if (lamrows) baug[a.m + a.n + j] = -lam * mv[j];
    }
}

// out[0] = ||D x||^2 (or ||P x||^2 with depth blocks P), out[1] = ||m||^2
// (one block, fixed order).
template <class ST>
__global__ void k_corr_norms(int32_t n, const double *__restrict__ x, const double *__restrict__ D,
                             const double *__restrict__ mv, double *out,
                             const ST *__restrict__ P = nullptr, int nz = 1) {
    __shared__ double s0[32], s1[32];
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double c = P ? blk_apply_row(P, x, j, nz) : (D ? D[j] * x[j] : x[j]);
        a += c * c;
        b += mv[j] * mv[j];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s0[warp] = a;
        s1[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ta += s0[i];
            tb += s1[i];
        }
        out[0] = ta;
        out[1] = tb;
    }
}

__global__ void k_fill(int64_t n, double v, double *x) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        x[j] = v;
}

static bool blocked_nz_ok(int nz) { return (nz % 2 == 0) ? nz <= 64 : nz <= 32; }

static pdst_status lsqr_impl(pdst_handle *h, const double *d_dev, double w_s, double lam,
                             int32_t itmax, double tol, double *m_out, pdst_lsqr_info *info,
                             const pdst_lsqr_opts *o, cudaStream_t s) {
    pdst_lsqr_opts opts;
    pdst_lsqr_opts_default(&opts);
    if (o) opts = *o;
    const int dtype = opts.dtype, fmt = opts.format;
    PDST_CHECK_ARG(dtype >= 0 && dtype <= 3, "pdst_lsqr: unknown dtype %d", dtype);
    PDST_CHECK_ARG(fmt == PDST_FMT_ELEMENT || fmt == PDST_FMT_BLOCKED, "pdst_lsqr: unknown format");
    PDST_CHECK_ARG(itmax >= 0, "pdst_lsqr: itmax must be >= 0");
    PDST_CHECK_ARG(std::isfinite(w_s) && w_s >= 0.0, "pdst_lsqr: w must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(lam) && lam >= 0.0, "pdst_lsqr: lambda must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(tol) && tol >= 0.0, "pdst_lsqr: tol must be finite and >= 0");
    PDST_CHECK_ARG(h->m == 0 || d_dev, "pdst_lsqr: d is NULL");
    PDST_CHECK_ARG(m_out, "pdst_lsqr: m_out is NULL");
    if (!h->vals[dtype].present) {
        set_error("pdst_lsqr: values of dtype %d were not kept by pdst_build_G", dtype);
        return PDST_ERR_STATE;
    }
    if (fmt == PDST_FMT_ELEMENT && !(h->formats & (1u << PDST_FMT_ELEMENT))) {
        set_error("pdst_lsqr: element indices were not built");
        return PDST_ERR_STATE;
    }
    if (fmt == PDST_FMT_BLOCKED && !blocked_nz_ok(h->nz)) {
        set_error("pdst_lsqr: the blocked layout needs nz <= 64 (nz <= 32 unless nz %% 4 == 0)");
        return PDST_ERR_LIMIT;
    }
    const bool user_scaled = opts.precond == 1;
    const bool user_blk = opts.precond == 2;
    if (user_scaled && !h->has_colscale) {
        set_error("pdst_lsqr: precond = 1 needs pdst_set_col_scaling first");
        return PDST_ERR_STATE;
    }
    PDST_CHECK_ARG(opts.precond >= 0 && opts.precond <= 2, "pdst_lsqr: unknown precond %d",
                   opts.precond);
    if (user_blk) {
        if (!h->has_blkprec) {
            set_error("pdst_lsqr: precond = 2 needs pdst_set_block_precond first");
            return PDST_ERR_STATE;
        }
        PDST_CHECK_ARG(fmt == PDST_FMT_BLOCKED, "pdst_lsqr: precond = 2 runs on the blocked layout");
        PDST_CHECK_ARG(dtype != PDST_DF64 && opts.refine_dtype != PDST_DF64,
                       "pdst_lsqr: precond = 2 is not available in the double-float form");
        if (h->nz > 32) {
            set_error("pdst_lsqr: precond = 2 needs nz <= 32");
            return PDST_ERR_LIMIT;
        }
    }
    PDST_CHECK_ARG(opts.refine >= 0 && opts.refine <= 100, "pdst_lsqr: refine must be in 0..100");
    const bool refine = opts.refine > 0;
    PDST_CHECK_ARG(opts.refine_dtype >= -1 && opts.refine_dtype <= 3,
                   "pdst_lsqr: unknown refine_dtype %d", opts.refine_dtype);
    if ((dtype == PDST_DF64 || (refine && opts.refine_dtype == PDST_DF64)) &&
        fmt != PDST_FMT_BLOCKED) {
        set_error("pdst_lsqr: the double-float form runs on the blocked layout only");
        return PDST_ERR_ARG;
    }
    if (refine && opts.refine_dtype >= 0 && !h->vals[opts.refine_dtype].present) {
        set_error("pdst_lsqr: values of refine_dtype %d were not kept", opts.refine_dtype);
        return PDST_ERR_STATE;
    }
    if (refine && !h->vals[PDST_F64].present) {
        set_error("pdst_lsqr: refinement needs the FP64 values (keep PDST_F64 in pdst_build_G)");
        return PDST_ERR_STATE;
    }
    PDST_CHECK_ARG(!(refine && opts.profile), "pdst_lsqr: profile and refine are exclusive");
    PDST_CHECK_ARG(opts.method == PDST_LSQR || opts.method == PDST_LSMR,
                   "pdst_lsqr: unknown method %d", opts.method);
    // refinement sweeps solve for a correction with a full augmented right-hand
    // side, so they always use the form with explicit lambda rows (unit scaling
    // when none is set)
    const bool scaled = user_scaled || user_blk || refine;
    const bool lamrows = scaled && lam > 0.0;
    PDST_CHECK_ARG(opts.profile >= 0 && opts.profile <= 2, "pdst_lsqr: unknown profile mode %d",
                   opts.profile);
    const int kblock = opts.profile == 1 ? 1 : (opts.kblock > 0 ? opts.kblock : 16);
    PDST_CHECK_ARG(kblock <= 1024, "pdst_lsqr: kblock must be <= 1024");

    LsqrScalars init{};
    init.cs2 = -1.0;
    init.damp = scaled ? 0.0 : lam;
    init.lam_rows = lamrows ? lam : 0.0;
    init.atol = opts.atol >= 0.0 ? opts.atol : tol;
    init.btol = opts.btol >= 0.0 ? opts.btol : tol;
    const double conlim = opts.conlim > 0.0 ? opts.conlim : 1e8;
    init.ctol = 1.0 / conlim;
    init.w_smooth = w_s;
    init.itmax = itmax;
    init.hist = opts.rnorm_hist_dev;
    init.method = opts.method;

    if (!h->work) h->work = new LsqrWork();
    LsqrWork *w = h->work;
    const bool fresh = w->dtype != dtype || w->format != fmt || w->lamrows != (int)lamrows;
    const double *Dover = nullptr;
    w->blk = user_blk ? 1 : 0;
    if (refine && !user_scaled && !user_blk) {
        PDST_TRY(w->ones.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
        k_fill<<<num_sms(h->device) * 4, LT, 0, s>>>(h->n, 1.0, w->ones.as<double>());
        PDST_CUDA(cudaGetLastError());
        Dover = w->ones.as<double>();
    }
    // captured graphs hold the workspace and scaling pointers: rebuild on change
    const void *dptr = Dover         ? (const void *)Dover
                       : user_scaled ? h->colscale.p
                       : user_blk    ? h->blkP64.p
                                     : nullptr;
    if (fresh || w->graph_D != dptr) {
        for (auto &g : w->graphs)
            if (g.second) cudaGraphExecDestroy(g.second);
        w->graphs.clear();
        w->graph_D = dptr;
    }
    const bool ug = opts.use_graph != 0;
    const int prof = opts.profile;
    RunStats rs;

    auto solve_once = [&](const double *baug, bool accumulate, bool fresh_,
                          int dtype) -> pdst_status {
        if (dtype == PDST_DF64)
            return dispatch_run<dfl, dfl, FMT_BLK>(h, w, dtype, scaled, lamrows, d_dev, init,
                                                   kblock, ug, prof, m_out, s, fresh_, rs, baug,
                                                   accumulate, Dover);
        if (dtype == PDST_F64)
            return fmt == PDST_FMT_ELEMENT
                       ? dispatch_run<double, double, FMT_ELEM>(h, w, dtype, scaled, lamrows, d_dev,
                                                               init, kblock, ug, prof, m_out, s,
                                                               fresh_, rs, baug, accumulate, Dover)
                       : dispatch_run<double, double, FMT_BLK>(h, w, dtype, scaled, lamrows, d_dev,
                                                              init, kblock, ug, prof, m_out, s,
                                                              fresh_, rs, baug, accumulate, Dover);
        if (dtype == PDST_F32)
            return fmt == PDST_FMT_ELEMENT
                       ? dispatch_run<float, float, FMT_ELEM>(h, w, dtype, scaled, lamrows, d_dev,
                                                             init, kblock, ug, prof, m_out, s,
                                                             fresh_, rs, baug, accumulate, Dover)
                       : dispatch_run<float, float, FMT_BLK>(h, w, dtype, scaled, lamrows, d_dev,
                                                            init, kblock, ug, prof, m_out, s,
                                                            fresh_, rs, baug, accumulate, Dover);
        return fmt == PDST_FMT_ELEMENT
                   ? dispatch_run<__nv_bfloat16, float, FMT_ELEM>(h, w, dtype, scaled, lamrows,
                                                                 d_dev, init, kblock, ug, prof,
                                                                 m_out, s, fresh_, rs, baug,
                                                                 accumulate, Dover)
                   : dispatch_run<__nv_bfloat16, float, FMT_BLK>(h, w, dtype, scaled, lamrows,
                                                                d_dev, init, kblock, ug, prof,
                                                                m_out, s, fresh_, rs, baug,
                                                                accumulate, Dover);
    };

    pdst_status st = PDST_OK;
    int total_iters = 0, sweeps = 0;
    double correction = 0.0;
    if (!refine) {
        st = solve_once(nullptr, false, fresh, dtype);
        total_iters = w->h_scal ? w->h_scal->itn : 0;
    } else {
        // mixed-precision refinement: m <- m + D * argmin ||A_D dy - r(m)||, with the
        // residual r(m) of the augmented system in FP64 (FP64 values of G) and the
        // correction from the reduced-precision LSQR
        const int64_t M = h->m + h->n + (lamrows ? h->n : 0);
        PDST_TRY(w->baug.alloc(sizeof(double) * std::max<int64_t>(M, 1)));
        PDST_TRY(w->corr.alloc(sizeof(double) * 2));
        PDST_CUDA(cudaMemsetAsync(m_out, 0, sizeof(double) * h->n, s));
        const double rtol = opts.refine_tol > 0.0 ? opts.refine_tol : 1e-5;
        const bool elem64 = (h->formats & (1u << PDST_FMT_ELEMENT)) != 0;
        auto a64 = make_args<double, double>(h, PDST_F64, nullptr, false, false);
        const unsigned gres = persistent_grid(elem64 ? k_resid<FMT_ELEM> : k_resid<FMT_BLK>,
                                              h->device, (h->m + h->n) * 32);
        bool fr = fresh;
        const int rdtype = opts.refine_dtype >= 0 ? opts.refine_dtype : dtype;
        int cur_dtype = dtype;
        for (int sweep = 0; sweep < opts.refine; ++sweep) {
            // sweep 0 in dtype at tol; later sweeps in refine_dtype at refine_tol
            const int sd = sweep == 0 ? dtype : rdtype;
            if (sweep == 1) {
                init.atol = init.btol = rtol;
                if (sd != cur_dtype) fr = true;
            }
            cur_dtype = sd;
            if (elem64)
                k_resid<FMT_ELEM><<<gres, LT, 0, s>>>(a64, d_dev, m_out, w_s, lam, lamrows ? 1 : 0,
                                                      w->baug.as<double>());
            else
                k_resid<FMT_BLK><<<gres, LT, 0, s>>>(a64, d_dev, m_out, w_s, lam, lamrows ? 1 : 0,
                                                     w->baug.as<double>());
            PDST_CUDA(cudaGetLastError());
            rs.launches += 1;
            if (fr && w->dtype != sd) {
                for (auto &g : w->graphs)
                    if (g.second) cudaGraphExecDestroy(g.second);
                w->graphs.clear();
            }
            st = solve_once(w->baug.as<double>(), true, fr || w->dtype != sd, sd);
            fr = false;
            if (st != PDST_OK) break;
            w->dtype = sd;
            w->format = fmt;
            w->lamrows = (int)lamrows;
            total_iters += w->h_scal->itn;
            ++sweeps;
            if (w->h_scal->err) break;
            const double *Dp = Dover ? Dover : h->colscale.as<double>();
            if (user_blk && sd == PDST_F64)
                k_corr_norms<double><<<1, 1024, 0, s>>>(h->n, w->x.as<double>(), nullptr, m_out,
                                                        w->corr.as<double>(),
                                                        h->blkP64.as<double>(), h->nz);
            else if (user_blk)
                k_corr_norms<float><<<1, 1024, 0, s>>>(h->n, w->x.as<double>(), nullptr, m_out,
                                                       w->corr.as<double>(),
                                                       h->blkP32.as<float>(), h->nz);
            else
                k_corr_norms<double><<<1, 1024, 0, s>>>(h->n, w->x.as<double>(), Dp, m_out,
                                                        w->corr.as<double>());
            rs.launches += 1;
            double cn[2];
            PDST_CUDA(cudaMemcpyAsync(cn, w->corr.p, sizeof(cn), cudaMemcpyDeviceToHost, s));
            PDST_CUDA(cudaStreamSynchronize(s));
            correction = cn[1] > 0.0 ? std::sqrt(cn[0] / cn[1]) : 0.0;
            if (sweep > 0 && (correction <= 1e-3 * rtol || w->h_scal->itn == 0)) break;
        }
        w->dtype = cur_dtype;
    }
    if (st != PDST_OK) {
        w->dtype = -1;
        return st;
    }
    if (!refine) w->dtype = dtype;
    w->format = fmt;
    w->lamrows = (int)lamrows;
    const LsqrScalars &c = *w->h_scal;
    if (info) {
        info->iters = total_iters;
        info->istop = c.istop;
        info->rnorm = c.rnorm;
        info->arnorm = c.arnorm;
        info->anorm = c.anorm;
        info->acond = c.acond;
        info->xnorm = c.xnorm;
        info->bnorm = c.bnorm;
        info->kernel_launches = rs.launches;
        info->profiled_iters = prof ? rs.profiled_iters : 0;
        info->fwd_ms = rs.fwd_ms;
        info->adj_ms = rs.adj_ms;
        info->upd_ms = rs.upd_ms;
        info->sweeps = sweeps;
        info->correction = correction;
    }
    if (c.err) {
        set_error("pdst_lsqr: non-finite value in the LSQR recurrence (iteration %d)", c.itn);
        return PDST_ERR_BREAKDOWN;
    }
    return PDST_OK;
}

pdst_status spmv_f64(pdst_handle *h, int dtype, int trans, const double *x, double *y,
                     cudaStream_t s) {
    const bool elem = (h->formats & (1u << PDST_FMT_ELEMENT)) != 0;
    const int64_t rows = trans ? h->n : h->m;
    if (rows == 0) return PDST_OK;
    if (dtype == PDST_F64) {
        auto a = make_args<double, double>(h, dtype, nullptr, false, false);
        if (elem) {
            unsigned g = persistent_grid(k_spmv<double, FMT_ELEM>, h->device, rows * 32);
            k_spmv<double, FMT_ELEM><<<g, LT, 0, s>>>(a, trans, x, y);
        } else {
            unsigned g = persistent_grid(k_spmv<double, FMT_BLK>, h->device, rows * 32);
            k_spmv<double, FMT_BLK><<<g, LT, 0, s>>>(a, trans, x, y);
        }
    } else if (dtype == PDST_F32) {
        auto a = make_args<float, double>(h, dtype, nullptr, false, false);
        if (elem) {
            unsigned g = persistent_grid(k_spmv<float, FMT_ELEM>, h->device, rows * 32);
            k_spmv<float, FMT_ELEM><<<g, LT, 0, s>>>(a, trans, x, y);
        } else {
            unsigned g = persistent_grid(k_spmv<float, FMT_BLK>, h->device, rows * 32);
            k_spmv<float, FMT_BLK><<<g, LT, 0, s>>>(a, trans, x, y);
        }
    } else {
        auto a = make_args<__nv_bfloat16, double>(h, dtype, nullptr, false, false);
        if (elem) {
            unsigned g = persistent_grid(k_spmv<__nv_bfloat16, FMT_ELEM>, h->device, rows * 32);
            k_spmv<__nv_bfloat16, FMT_ELEM><<<g, LT, 0, s>>>(a, trans, x, y);
        } else {
            unsigned g = persistent_grid(k_spmv<__nv_bfloat16, FMT_BLK>, h->device, rows * 32);
            k_spmv<__nv_bfloat16, FMT_BLK><<<g, LT, 0, s>>>(a, trans, x, y);
        }
    }
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}

static pdst_status colnorm_scaling(pdst_handle *h, double w, double lam, double *D,
                                   cudaStream_t s, int mode = 0, double pw = 1.0) {
    if (h->n == 0) return PDST_OK;
    if (h->vals[PDST_F64].present) {
        auto a = make_args<double, double>(h, PDST_F64, nullptr, false, false);
        unsigned g = persistent_grid(k_colnorm_scale<double>, h->device, (int64_t)h->n * 32);
        k_colnorm_scale<double><<<g, LT, 0, s>>>(a, w, lam, D, mode, pw);
    } else if (h->vals[PDST_F32].present) {
        auto a = make_args<float, double>(h, PDST_F32, nullptr, false, false);
        unsigned g = persistent_grid(k_colnorm_scale<float>, h->device, (int64_t)h->n * 32);
        k_colnorm_scale<float><<<g, LT, 0, s>>>(a, w, lam, D, mode, pw);
    } else {
        auto a = make_args<__nv_bfloat16, double>(h, PDST_BF16, nullptr, false, false);
        unsigned g = persistent_grid(k_colnorm_scale<__nv_bfloat16>, h->device, (int64_t)h->n * 32);
        k_colnorm_scale<__nv_bfloat16><<<g, LT, 0, s>>>(a, w, lam, D, mode, pw);
    }
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}

// ------------------------------------------------------------ damping sweep

constexpr int MAX_SWEEP = 64;

template <class VT, class ST, int FMT>
static pdst_status sweep_run(pdst_handle *h, LsqrWork *w, int dtype, const double *d,
                             const LsqrScalars &base0, std::vector<LsqrScalars> &lam,
                             int kblock, double *const *m_out, cudaStream_t s, int &launches) {
    const int L = (int)lam.size();
    const int64_t n = h->n;
    PDST_TRY(w->sw_x.alloc(sizeof(double) * std::max<int64_t>(L * n, 1)));
    PDST_TRY(w->sw_w.alloc(sizeof(double) * std::max<int64_t>(L * n, 1)));
    PDST_TRY(w->sw_sc.alloc(sizeof(LsqrScalars) * L));
    PDST_TRY(w->sw_part.alloc(sizeof(double) * L * MAXBLK));
    PDST_TRY(w->sw_cnt.alloc(sizeof(unsigned) * (L + 1)));   // per value, + all blocks
    PDST_TRY(w->sw_stage.alloc(sizeof(LsqrScalars) * L));
    OpArgs<VT, ST> a = make_args<VT, ST>(h, dtype, w, false, false);
    a.lam_sc = w->sw_sc.as<LsqrScalars>();
    a.n_lam = L;
    double *X = w->sw_x.as<double>(), *W = w->sw_w.as<double>();
    PDST_CUDA(cudaMemsetAsync(w->sync.p, 0, sizeof(LsqrSync), s));
    PDST_CUDA(cudaMemsetAsync(w->cell_done.p, 0, sizeof(unsigned) * std::max<int32_t>(h->H, 1), s));
    PDST_CUDA(cudaMemsetAsync(w->sw_cnt.p, 0, sizeof(unsigned) * (L + 1), s));
    PDST_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * L * n, s));
    *w->h_scal = base0;
    PDST_CUDA(cudaMemcpyAsync(w->scal.p, w->h_scal, sizeof(LsqrScalars), cudaMemcpyHostToDevice, s));
    PDST_CUDA(cudaMemcpyAsync(w->sw_sc.p, lam.data(), sizeof(LsqrScalars) * L,
                              cudaMemcpyHostToDevice, s));
    const dim3 gu(w->grid_vec, L);
    const unsigned ginit = persistent_grid(k_init<ST>, h->device, w->M);
    k_init<ST><<<ginit, LT, 0, s>>>(h->m, w->M, h->n, d, nullptr, a.ubar, a.x, a.wv, a.partial,
                                    a.sc, a.sy);
    adj_kernel<VT, ST, FMT>(h->nz)<<<w->grid_cols, LT, 0, s>>>(a, 1);
    LsqrScalars *stage = w->sw_stage.as<LsqrScalars>();
    k_upd_sweep<ST><<<gu, LT, 0, s>>>(h->n, a.vbar, X, W, w->sw_part.as<double>(), a.sc,
                                      a.lam_sc, stage, L, w->sw_cnt.as<unsigned>());
    PDST_CUDA(cudaGetLastError());
    launches += 3;
    for (;;) {
        PDST_CUDA(cudaMemcpyAsync(w->h_scal, w->scal.p, sizeof(LsqrScalars),
                                  cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        const LsqrScalars &c = *w->h_scal;
        if (c.done || c.istop || c.err || c.itn >= c.itmax) break;
        // the order of Solver::launch_iter, with the sweep's steps and updates
        // beside the forward (the per-value scalars, x and w are theirs alone)
        for (int i = 0; i < kblock; ++i) {
            cudaEventRecord(w->ev_fork, s);
            cudaStreamWaitEvent(w->side, w->ev_fork, 0);
            k_step_sweep<<<1, LT, 0, w->side>>>(a.sc, a.lam_sc, stage, L);
            k_upd_sweep<ST><<<gu, LT, 0, w->side>>>(h->n, a.vbar, X, W, w->sw_part.as<double>(),
                                                    a.sc, a.lam_sc, stage, L,
                                                    w->sw_cnt.as<unsigned>(), 1);
            cudaEventRecord(w->ev_join, w->side);
            fwd_kernel<VT, ST, FMT>(h->nz)<<<w->grid_rows, LT, 0, s>>>(a);
            cudaStreamWaitEvent(s, w->ev_join, 0);
            k_pub_base<<<1, 32, 0, s>>>(a.sc);
            adj_kernel<VT, ST, FMT>(h->nz)<<<w->grid_cols, LT, 0, s>>>(a, 0);
        }
        PDST_CUDA(cudaGetLastError());
        launches += 5 * kblock;
    }
    for (int l = 0; l < L; ++l)
        k_finalize<<<w->grid_vec, LT, 0, s>>>(h->n, X + (int64_t)l * n, nullptr, m_out[l], 0);
    PDST_CUDA(cudaGetLastError());
    launches += L;
    PDST_CUDA(cudaMemcpyAsync(lam.data(), w->sw_sc.p, sizeof(LsqrScalars) * L,
                              cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    return PDST_OK;
}

static pdst_status sweep_impl(pdst_handle *h, const double *d_dev, double w_s, int32_t nlam,
                              const double *lambda_host, int32_t itmax, double tol,
                              double *const *m_out, pdst_lsqr_info *infos,
                              const pdst_lsqr_opts *o, cudaStream_t s) {
    pdst_lsqr_opts opts;
    pdst_lsqr_opts_default(&opts);
    if (o) opts = *o;
    const int dtype = opts.dtype, fmt = opts.format;
    PDST_CHECK_ARG(nlam >= 1 && nlam <= MAX_SWEEP, "pdst_lsqr_damping_sweep: nlam must be in 1..%d",
                   MAX_SWEEP);
    PDST_CHECK_ARG(lambda_host && m_out, "pdst_lsqr_damping_sweep: NULL lambda or m_out");
    for (int l = 0; l < nlam; ++l) {
        PDST_CHECK_ARG(std::isfinite(lambda_host[l]) && lambda_host[l] >= 0.0,
                       "pdst_lsqr_damping_sweep: lambda[%d] must be finite and >= 0", l);
        PDST_CHECK_ARG(m_out[l], "pdst_lsqr_damping_sweep: m_out[%d] is NULL", l);
    }
    PDST_CHECK_ARG(dtype >= 0 && dtype <= 3, "pdst_lsqr_damping_sweep: unknown dtype %d", dtype);
    PDST_CHECK_ARG(fmt == PDST_FMT_ELEMENT || fmt == PDST_FMT_BLOCKED,
                   "pdst_lsqr_damping_sweep: unknown format");
    PDST_CHECK_ARG(itmax >= 0, "pdst_lsqr_damping_sweep: itmax must be >= 0");
    PDST_CHECK_ARG(std::isfinite(w_s) && w_s >= 0.0, "pdst_lsqr_damping_sweep: bad w");
    PDST_CHECK_ARG(std::isfinite(tol) && tol >= 0.0, "pdst_lsqr_damping_sweep: bad tol");
    PDST_CHECK_ARG(h->m == 0 || d_dev, "pdst_lsqr_damping_sweep: d is NULL");
    PDST_CHECK_ARG(opts.precond == 0 && opts.refine == 0 && opts.profile == 0 &&
                       opts.method == PDST_LSQR,
                   "pdst_lsqr_damping_sweep: plain LSQR only (no scaling, refinement, profile "
                   "or LSMR)");
    if (!h->vals[dtype].present) {
        set_error("pdst_lsqr_damping_sweep: values of dtype %d were not kept", dtype);
        return PDST_ERR_STATE;
    }
    if (dtype == PDST_DF64 && fmt != PDST_FMT_BLOCKED) {
        set_error("pdst_lsqr_damping_sweep: the double-float form runs on the blocked layout only");
        return PDST_ERR_ARG;
    }
    if (fmt == PDST_FMT_ELEMENT && !(h->formats & (1u << PDST_FMT_ELEMENT))) {
        set_error("pdst_lsqr_damping_sweep: element indices were not built");
        return PDST_ERR_STATE;
    }
    if (fmt == PDST_FMT_BLOCKED && !blocked_nz_ok(h->nz)) {
        set_error("pdst_lsqr_damping_sweep: the blocked layout needs nz <= 64");
        return PDST_ERR_LIMIT;
    }
    const int kblock = opts.kblock > 0 ? opts.kblock : 16;
    LsqrScalars base{};
    base.cs2 = -1.0;
    base.itmax = itmax;
    base.w_smooth = w_s;
    std::vector<LsqrScalars> lam(nlam);
    for (int l = 0; l < nlam; ++l) {
        LsqrScalars &c = lam[l];
        c = LsqrScalars{};
        c.cs2 = -1.0;
        c.damp = lambda_host[l];
        c.atol = opts.atol >= 0.0 ? opts.atol : tol;
        c.btol = opts.btol >= 0.0 ? opts.btol : tol;
        c.ctol = 1.0 / (opts.conlim > 0.0 ? opts.conlim : 1e8);
        c.w_smooth = w_s;
        c.itmax = itmax;
    }
    if (itmax == 0) {
        for (int l = 0; l < nlam; ++l) PDST_CUDA(cudaMemsetAsync(m_out[l], 0, sizeof(double) * h->n, s));
        if (infos)
            for (int l = 0; l < nlam; ++l) infos[l] = pdst_lsqr_info{};
        PDST_CUDA(cudaStreamSynchronize(s));
        return PDST_OK;
    }
    if (!h->work) h->work = new LsqrWork();
    LsqrWork *w = h->work;
    w->blk = 0;   // the sweep runs unpreconditioned
    const bool fresh = w->dtype != dtype || w->format != fmt || w->lamrows != 0;
    if (fresh) {
        // buffers may move: the ordinary solve's captured graphs are stale
        for (auto &g : w->graphs)
            if (g.second) cudaGraphExecDestroy(g.second);
        w->graphs.clear();
    }
    int launches = 0;
    pdst_status st;
    auto prep_run = [&](auto tag) -> pdst_status {
        using S = decltype(tag);
        if (fresh) PDST_TRY((S::prepare(h, w, false)));
        return sweep_run<typename S::VTy, typename S::STy, S::FMTv>(h, w, dtype, d_dev, base, lam,
                                                                   kblock, m_out, s, launches);
    };
    if (dtype == PDST_DF64)
        st = prep_run(Solver<dfl, dfl, FMT_BLK>{});
    else if (dtype == PDST_F64)
        st = fmt == PDST_FMT_ELEMENT ? prep_run(Solver<double, double, FMT_ELEM>{})
                                     : prep_run(Solver<double, double, FMT_BLK>{});
    else if (dtype == PDST_F32)
        st = fmt == PDST_FMT_ELEMENT ? prep_run(Solver<float, float, FMT_ELEM>{})
                                     : prep_run(Solver<float, float, FMT_BLK>{});
    else
        st = fmt == PDST_FMT_ELEMENT ? prep_run(Solver<__nv_bfloat16, float, FMT_ELEM>{})
                                     : prep_run(Solver<__nv_bfloat16, float, FMT_BLK>{});
    if (st != PDST_OK) {
        w->dtype = -1;
        return st;
    }
    w->dtype = dtype;
    w->format = fmt;
    w->lamrows = 0;
    bool err = w->h_scal->err != 0;
    for (int l = 0; l < nlam; ++l) {
        const LsqrScalars &c = lam[l];
        err |= c.err != 0;
        if (infos) {
            pdst_lsqr_info &f = infos[l];
            f = pdst_lsqr_info{};
            f.iters = c.itn;
            f.istop = c.istop;
            f.rnorm = c.rnorm;
            f.arnorm = c.arnorm;
            f.anorm = c.anorm;
            f.acond = c.acond;
            f.xnorm = c.xnorm;
            f.bnorm = c.bnorm;
            f.kernel_launches = launches;
        }
    }
    if (err) {
        set_error("pdst_lsqr_damping_sweep: non-finite value in a recurrence");
        return PDST_ERR_BREAKDOWN;
    }
    return PDST_OK;
}

}  // namespace pdst

using namespace pdst;

extern "C" void pdst_lsqr_opts_default(pdst_lsqr_opts *o) {
    if (!o) return;
    o->dtype = PDST_F64;
    o->format = PDST_FMT_ELEMENT;
    o->atol = -1.0;
    o->btol = -1.0;
    o->conlim = 0.0;
    o->precond = 0;
    o->kblock = 16;
    o->use_graph = 1;
    o->profile = 0;
    o->rnorm_hist_dev = nullptr;
    o->refine = 0;
    o->refine_dtype = -1;
    o->method = PDST_LSQR;
    o->reserved0 = 0;
    o->refine_tol = 1e-5;
}

extern "C" pdst_status pdst_lsqr(pdst_handle_t h, const double *d_dev, double w, double lambda,
                                 int32_t itmax, double tol, double *m_out_dev,
                                 pdst_lsqr_info *info, const pdst_lsqr_opts *opts, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_lsqr: handle is NULL");
    return lsqr_impl(h, d_dev, w, lambda, itmax, tol, m_out_dev, info, opts,
                     (cudaStream_t)stream);
}

extern "C" pdst_status pdst_lsqr_damping_sweep(pdst_handle_t h, const double *d_dev, double w,
                                               int32_t nlam, const double *lambda_host,
                                               int32_t itmax, double tol,
                                               double *const *m_out_dev, pdst_lsqr_info *infos,
                                               const pdst_lsqr_opts *opts, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_lsqr_damping_sweep: handle is NULL");
    return sweep_impl(h, d_dev, w, nlam, lambda_host, itmax, tol, m_out_dev, infos, opts,
                      (cudaStream_t)stream);
}

extern "C" pdst_status pdst_lsqr_host(pdst_handle_t h, const double *d_host, double w,
                                      double lambda, int32_t itmax, double tol,
                                      double *m_out_host, pdst_lsqr_info *info,
                                      const pdst_lsqr_opts *opts, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_lsqr_host: handle is NULL");
    PDST_CHECK_ARG(h->m == 0 || d_host, "pdst_lsqr_host: d is NULL");
    PDST_CHECK_ARG(m_out_host, "pdst_lsqr_host: m_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    static thread_local DevBuf dd, mm;
    PDST_TRY(dd.alloc(sizeof(double) * std::max<int64_t>(h->m, 1)));
    PDST_TRY(mm.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
    if (h->m)
        PDST_CUDA(cudaMemcpyAsync(dd.p, d_host, sizeof(double) * h->m, cudaMemcpyHostToDevice, s));
    PDST_TRY(lsqr_impl(h, dd.as<double>(), w, lambda, itmax, tol, mm.as<double>(), info, opts, s));
    PDST_CUDA(cudaMemcpyAsync(m_out_host, mm.p, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    return PDST_OK;
}

extern "C" pdst_status pdst_apply_G(pdst_handle_t h, int32_t dtype, int32_t trans,
                                    const double *x_dev, double *y_dev, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_apply_G: handle is NULL");
    PDST_CHECK_ARG(dtype >= 0 && dtype <= 2, "pdst_apply_G: unknown dtype");
    PDST_CHECK_ARG(trans == 0 || trans == 1, "pdst_apply_G: trans must be 0 or 1");
    PDST_CHECK_ARG(x_dev && y_dev, "pdst_apply_G: NULL vector");
    if (!h->vals[dtype].present) {
        set_error("pdst_apply_G: values of dtype %d were not kept", dtype);
        return PDST_ERR_STATE;
    }
    return spmv_f64(h, dtype, trans, x_dev, y_dev, (cudaStream_t)stream);
}

extern "C" pdst_status pdst_set_col_scaling(pdst_handle_t h, const double *D_dev, double w,
                                            double lambda, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_set_col_scaling: handle is NULL");
    PDST_CHECK_ARG(std::isfinite(w) && std::isfinite(lambda) && w >= 0 && lambda >= 0,
                   "pdst_set_col_scaling: w and lambda must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    PDST_TRY(h->colscale.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
    if (D_dev) {
        PDST_CUDA(cudaMemcpyAsync(h->colscale.p, D_dev, sizeof(double) * h->n,
                                  cudaMemcpyDeviceToDevice, s));
    } else {
        PDST_TRY(colnorm_scaling(h, w, lambda, h->colscale.as<double>(), s));
    }
    PDST_CUDA(cudaStreamSynchronize(s));
    h->has_colscale = true;
    return PDST_OK;
}

extern "C" pdst_status pdst_col_norms(pdst_handle_t h, double w, double lambda, double *c_dev,
                                      void *stream) {
    PDST_CHECK_ARG(h != nullptr && c_dev != nullptr, "pdst_col_norms: NULL argument");
    PDST_CHECK_ARG(std::isfinite(w) && std::isfinite(lambda) && w >= 0 && lambda >= 0,
                   "pdst_col_norms: w and lambda must be finite and >= 0");
    return colnorm_scaling(h, w, lambda, c_dev, (cudaStream_t)stream, 2, 0.0);
}

extern "C" pdst_status pdst_set_col_scaling_power(pdst_handle_t h, double w, double lambda,
                                                  double p, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_set_col_scaling_power: handle is NULL");
    PDST_CHECK_ARG(std::isfinite(w) && std::isfinite(lambda) && w >= 0 && lambda >= 0,
                   "pdst_set_col_scaling_power: w and lambda must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(p), "pdst_set_col_scaling_power: p must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    PDST_TRY(h->colscale.alloc(sizeof(double) * std::max<int32_t>(h->n, 1)));
    PDST_TRY(colnorm_scaling(h, w, lambda, h->colscale.as<double>(), s, 1, p));
    PDST_CUDA(cudaStreamSynchronize(s));
    h->has_colscale = true;
    return PDST_OK;
}

// --------------------------------------------------- allocation-free solve
//
// pdst_lsqr_noalloc runs the same LSQR kernels as pdst_lsqr, but every scratch
// buffer of the solve (the recurrence scalars, the reduction partials and
// counters, u-bar, v-bar, the scaled v, x and w) is carved out of one
// file-scope device array instead of memory the handle allocates.  The host
// side allocates nothing either: no graph, no events, no pinned buffers.

namespace pdst {

constexpr size_t NOALLOC_BYTES = size_t(16) << 20;   // 16 MiB per device
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// symbol name is only a stand-in, so the address is looked up once per device
// (with that device current) and passed to the kernels.
static void *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

static pdst_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) {
        set_error("pdst_lsqr_noalloc: device ordinal %d out of range", device);
        return PDST_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("pdst_lsqr_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return PDST_ERR_CUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[device]);
    return PDST_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of scratch one solve needs, in the carving order used below.
static size_t noalloc_need(int64_t M, int64_t n, size_t st, int64_t chunk_vals, int64_t H) {
    return align256(2 * sizeof(LsqrScalars)) + align256(sizeof(LsqrSync)) +
           align256(sizeof(double) * 3 * MAXBLK) + align256(st * M) + 2 * align256(st * n) +
           2 * align256(sizeof(double) * n) + align256(st * chunk_vals) +
           align256(sizeof(unsigned) * H) + align256(sizeof(double) * H);
}

template <class VT, class ST, int FMT>
static pdst_status noalloc_run(pdst_handle *h, unsigned char *base, int dtype, bool scaled,
                               bool lamrows, const double *d, const LsqrScalars &init,
                               int kblock, double *m_out, cudaStream_t s, LsqrScalars &fin,
                               int &launches) {
    const int64_t M = h->m + h->n + (lamrows ? h->n : 0);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += align256(bytes);
        return p;
    };
    auto *sc = reinterpret_cast<LsqrScalars *>(carve(2 * sizeof(LsqrScalars)));   // + k_step's copy
    auto *sy = reinterpret_cast<LsqrSync *>(carve(sizeof(LsqrSync)));
    auto *partial = reinterpret_cast<double *>(carve(sizeof(double) * 3 * MAXBLK));
    auto *ubar = reinterpret_cast<ST *>(carve(sizeof(ST) * M));
    auto *vbar = reinterpret_cast<ST *>(carve(sizeof(ST) * h->n));
    auto *vsc = reinterpret_cast<ST *>(carve(sizeof(ST) * h->n));
    auto *x = reinterpret_cast<double *>(carve(sizeof(double) * h->n));
    auto *wv = reinterpret_cast<double *>(carve(sizeof(double) * h->n));
    auto *cpart = reinterpret_cast<ST *>(carve(sizeof(ST) * h->n_adj * h->nz));
    auto *cdone = reinterpret_cast<unsigned *>(carve(sizeof(unsigned) * h->H));
    auto *css = reinterpret_cast<double *>(carve(sizeof(double) * h->H));

    OpArgs<VT, ST> a = make_args<VT, ST>(h, dtype, nullptr, scaled, lamrows);
    a.chunk_part = cpart;
    a.cell_done = cdone;
    a.cell_ss = css;
    a.ubar = ubar;
    a.vbar = vbar;
    a.vsc = scaled ? vsc : vbar;
    a.x = x;
    a.wv = wv;
    a.partial = partial;
    a.sc = sc;
    a.sc_stage = sc + 1;
    a.sy = sy;
    const unsigned g_rows = fwd_grid(fwd_kernel<VT, ST, FMT>(h->nz), h->device, (h->m + h->n) * 32);
    const unsigned g_cols = persistent_grid(adj_kernel<VT, ST, FMT>(h->nz), h->device, (int64_t)h->n * 32);
    const unsigned g_vec = persistent_grid(k_upd<ST>, h->device, h->n);
    const unsigned g_init = persistent_grid(k_init<ST>, h->device, M);

    // the array keeps the previous call's contents: the counters must start at
    // zero and the scalars from this call's values; every vector is written
    // before it is read (k_init, the start step of k_adj, k_upd)
    PDST_CUDA(cudaMemsetAsync(sy, 0, sizeof(LsqrSync), s));
    PDST_CUDA(cudaMemsetAsync(cdone, 0, sizeof(unsigned) * h->H, s));
    PDST_CUDA(cudaMemsetAsync(css, 0, sizeof(double) * h->H, s));
    LsqrScalars hs = init;
    PDST_CUDA(cudaMemcpyAsync(sc, &hs, sizeof(LsqrScalars), cudaMemcpyHostToDevice, s));
    k_init<ST><<<g_init, LT, 0, s>>>(h->m, M, h->n, d, nullptr, ubar, x, wv, partial, sc, sy);
    adj_kernel<VT, ST, FMT>(h->nz)<<<g_cols, LT, 0, s>>>(a, 1);
    k_upd<ST><<<g_vec, LT, 0, s>>>(h->n, vbar, x, wv, nullptr, partial, sc, sc + 1, sy);
    PDST_CUDA(cudaGetLastError());
    launches += 3;
    for (;;) {
        PDST_CUDA(cudaMemcpyAsync(&fin, sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        if (fin.done || fin.istop || fin.itn >= fin.itmax) break;
        // the kernels of Solver::launch_iter, k_step in line (one stream)
        for (int i = 0; i < kblock; ++i) {
            k_step<<<1, 32, 0, s>>>(sc, sc + 1);
            fwd_kernel<VT, ST, FMT>(h->nz)<<<g_rows, LT, 0, s>>>(a);
            k_upd<ST><<<g_vec, LT, 0, s>>>(h->n, vbar, x, wv, nullptr, partial, sc, sc + 1, sy);
            adj_kernel<VT, ST, FMT>(h->nz)<<<g_cols, LT, 0, s>>>(a, 0);
        }
        PDST_CUDA(cudaGetLastError());
        launches += 4 * kblock;
    }
    k_finalize<<<g_vec, LT, 0, s>>>(h->n, x, a.D, m_out);
    PDST_CUDA(cudaGetLastError());
    launches += 1;
    PDST_CUDA(cudaMemcpyAsync(&fin, sc, sizeof(LsqrScalars), cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    return PDST_OK;
}

}  // namespace pdst

extern "C" pdst_status pdst_lsqr_noalloc(pdst_handle_t h, const double *d_dev, double w,
                                         double lambda, int32_t itmax, double tol,
                                         double *m_out_dev, pdst_lsqr_info *info,
                                         const pdst_lsqr_opts *o, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_lsqr_noalloc: handle is NULL");
    pdst_lsqr_opts opts;
    pdst_lsqr_opts_default(&opts);
    if (o) opts = *o;
    const int dtype = opts.dtype, fmt = opts.format;
    PDST_CHECK_ARG(dtype >= 0 && dtype <= 2, "pdst_lsqr_noalloc: unknown dtype %d", dtype);
    PDST_CHECK_ARG(opts.method == PDST_LSQR, "pdst_lsqr_noalloc: LSQR only (method %d)",
                   opts.method);
    PDST_CHECK_ARG(fmt == PDST_FMT_ELEMENT || fmt == PDST_FMT_BLOCKED,
                   "pdst_lsqr_noalloc: unknown format");
    PDST_CHECK_ARG(itmax >= 0, "pdst_lsqr_noalloc: itmax must be >= 0");
    PDST_CHECK_ARG(std::isfinite(w) && w >= 0.0, "pdst_lsqr_noalloc: w must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(lambda) && lambda >= 0.0,
                   "pdst_lsqr_noalloc: lambda must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(tol) && tol >= 0.0,
                   "pdst_lsqr_noalloc: tol must be finite and >= 0");
    PDST_CHECK_ARG(h->m == 0 || d_dev, "pdst_lsqr_noalloc: d is NULL");
    PDST_CHECK_ARG(m_out_dev, "pdst_lsqr_noalloc: m_out is NULL");
    PDST_CHECK_ARG(opts.profile == 0, "pdst_lsqr_noalloc: profile mode is not available");
    PDST_CHECK_ARG(opts.refine == 0,
                   "pdst_lsqr_noalloc: refinement sweeps are not available (refine %d)",
                   opts.refine);
    PDST_CHECK_ARG(opts.precond == 0 || opts.precond == 1,
                   "pdst_lsqr_noalloc: unknown precond %d", opts.precond);
    if (!h->vals[dtype].present) {
        set_error("pdst_lsqr_noalloc: values of dtype %d were not kept by pdst_build_G", dtype);
        return PDST_ERR_STATE;
    }
    if (fmt == PDST_FMT_ELEMENT && !(h->formats & (1u << PDST_FMT_ELEMENT))) {
        set_error("pdst_lsqr_noalloc: element indices were not built");
        return PDST_ERR_STATE;
    }
    if (fmt == PDST_FMT_BLOCKED && !blocked_nz_ok(h->nz)) {
        set_error("pdst_lsqr_noalloc: the blocked layout needs nz <= 64 (nz <= 32 unless nz %% 4 == 0)");
        return PDST_ERR_LIMIT;
    }
    const bool scaled = opts.precond == 1;
    if (scaled && !h->has_colscale) {
        set_error("pdst_lsqr_noalloc: precond = 1 needs pdst_set_col_scaling first");
        return PDST_ERR_STATE;
    }
    int cur = -1;
    PDST_CUDA(cudaGetDevice(&cur));
    PDST_CHECK_ARG(cur == h->device,
                   "pdst_lsqr_noalloc: the handle's device (%d) must be current (is %d)",
                   h->device, cur);
    const bool lamrows = scaled && lambda > 0.0;
    const int kblock = opts.kblock > 0 ? opts.kblock : 16;
    PDST_CHECK_ARG(kblock <= 1024, "pdst_lsqr_noalloc: kblock must be <= 1024");
    const int64_t M = h->m + h->n + (lamrows ? h->n : 0);
    const size_t st = dtype == PDST_F64 ? sizeof(double) : sizeof(float);
    const size_t need = noalloc_need(M, h->n, st, h->n_adj * h->nz, h->H);
    if (need > NOALLOC_BYTES) {
        set_error("pdst_lsqr_noalloc: this system needs %zu bytes of scratch; the static "
                  "array holds %zu (use pdst_lsqr)", need, NOALLOC_BYTES);
        return PDST_ERR_LIMIT;
    }
    unsigned char *base = nullptr;
    PDST_TRY(noalloc_scratch(cur, &base));

    LsqrScalars init{};
    init.cs2 = -1.0;
    init.damp = scaled ? 0.0 : lambda;
    init.lam_rows = lamrows ? lambda : 0.0;
    init.atol = opts.atol >= 0.0 ? opts.atol : tol;
    init.btol = opts.btol >= 0.0 ? opts.btol : tol;
    init.ctol = 1.0 / (opts.conlim > 0.0 ? opts.conlim : 1e8);
    init.w_smooth = w;
    init.itmax = itmax;
    init.hist = opts.rnorm_hist_dev;

    cudaStream_t s = (cudaStream_t)stream;
    LsqrScalars fin{};
    int launches = 0;
    pdst_status st_;
    if (dtype == PDST_F64)
        st_ = fmt == PDST_FMT_ELEMENT
                  ? noalloc_run<double, double, FMT_ELEM>(h, base, dtype, scaled, lamrows, d_dev,
                                                          init, kblock, m_out_dev, s, fin, launches)
                  : noalloc_run<double, double, FMT_BLK>(h, base, dtype, scaled, lamrows, d_dev,
                                                         init, kblock, m_out_dev, s, fin, launches);
    else if (dtype == PDST_F32)
        st_ = fmt == PDST_FMT_ELEMENT
                  ? noalloc_run<float, float, FMT_ELEM>(h, base, dtype, scaled, lamrows, d_dev,
                                                        init, kblock, m_out_dev, s, fin, launches)
                  : noalloc_run<float, float, FMT_BLK>(h, base, dtype, scaled, lamrows, d_dev,
                                                       init, kblock, m_out_dev, s, fin, launches);
    else
        st_ = fmt == PDST_FMT_ELEMENT
                  ? noalloc_run<__nv_bfloat16, float, FMT_ELEM>(h, base, dtype, scaled, lamrows,
                                                                d_dev, init, kblock, m_out_dev, s,
                                                                fin, launches)
                  : noalloc_run<__nv_bfloat16, float, FMT_BLK>(h, base, dtype, scaled, lamrows,
                                                               d_dev, init, kblock, m_out_dev, s,
                                                               fin, launches);
    if (st_ != PDST_OK) return st_;
    if (info) {
        *info = pdst_lsqr_info{};
        info->iters = fin.itn;
        info->istop = fin.istop;
        info->rnorm = fin.rnorm;
        info->arnorm = fin.arnorm;
        info->anorm = fin.anorm;
        info->acond = fin.acond;
        info->xnorm = fin.xnorm;
        info->bnorm = fin.bnorm;
        info->kernel_launches = launches;
    }
    if (fin.err) {
        set_error("pdst_lsqr_noalloc: non-finite value in the LSQR recurrence (iteration %d)",
                  fin.itn);
        return PDST_ERR_BREAKDOWN;
    }
    return PDST_OK;
}
