// batched.cu -- batched LSQR: many independent systems (each its own handle,
// sizes may differ) with up to 16 right-hand sides each, solved together.
//
// Every phase of an iteration is one persistent launch over a work list that
// spans all systems (a "segmented" list: each system owns a contiguous range
// of items).  The right-hand sides of a system share its G: a half-warp holds
// the 16 right-hand sides in its lanes, so each matrix entry read from HBM is
// used for all of them (a sparse-times-dense product instead of 16 sparse
// products).  Each (system, right-hand side) pair keeps its own FP64 LSQR
// recurrence (Paige & Saunders 1982) with its own damping, and stops on its
// own; a system whose pairs have all stopped drops out of the work lists.
//
// Per iteration: k_bfwd (u-bar <- A v - alpha u, per-item partial norms),
// k_bred (beta per pair), k_badj (v-bar <- A^T u - beta v), k_bred (alpha and
// the recurrence per pair), k_bupd (x, w), k_bred (||w||^2).  Reductions sum
// per-item partials in item order, so results are bit-reproducible.
//
// The rows per forward work item are picked by a small autotuner that times
// the forward phase for a few candidates on the actual batch.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "lsqr_dev.cuh"

namespace pdst {
namespace {

constexpr int BT = 256;      // threads per block
constexpr int RMAX = 16;     // right-hand sides per system (lanes of a half-warp)
constexpr int LCOLS = 32;    // columns per stencil / update work item
constexpr int NB = 8;        // work buffers per system: U, V, X, W, chunk sums, chunk counters,
                             // cell sums, scaled V
//
// With the per-cell depth-block preconditioner (precond = 2) the adjoint
// leaves s = A^T u (stencil and lambda rows included) in Vs, and k_bblk, one
// half-warp per cell with lane j = right-hand side j, finishes each cell:
// t = P_h^T s, v-bar <- t / beta - (beta/alpha) v-bar, Vs <- P_h v-bar, and
// the cell's sums of squares (one launch more per iteration).

template <class VT, class ST> struct BSys {
    int64_t m;
    int32_t n, nx, ny, nz, R;
    int32_t RS;       // row stride of V: R rounded up to 4, 8 or 16
    int64_t n_adj;    // adjoint work items
    double w;
    const int64_t *row_cptr;
    const int32_t *row_cells;
    const VT *val;
    const int64_t *cell_rptr;
    const int32_t *cell_cnt;
    const int32_t *cell_rows;
    const int32_t *cell_order;
    const VT *valB;   // blocked CSC values
    const int32_t *adj_item;   // (cell, first row) per adjoint work item
    int32_t adj_chunk;         // rows per adjoint work item
    ST *chunk_part;   // adjoint work items x nz x RMAX partial sums
    unsigned *cell_done;       // H finished-chunk counters
    double *cell_ss;           // H x RMAX: sum of v^2 of cells finished across several items
    ST *U;            // (m + n [+ n]) x RS, right-hand side fastest (padding lanes stay 0)
    ST *V;            // n x RS, right-hand side fastest (padding lanes stay 0)
    ST *Vs;           // n x RS: D o V (or P V) with a right scaling, else V itself; with depth
                      // blocks it holds (A^T u) between the adjoint and k_bblk
    const double *D;  // right diagonal scaling D (n) or nullptr
    const ST *P;      // per-cell depth blocks P_h (H x nz x nz, upper triangular) or nullptr
    int32_t lamr;     // 1: the lambda_j D rows are appended (scaled form)
    double *X, *W;    // n x R
    const double *d;  // m x R
    LsqrScalars *sc;  // R
    int64_t nf;       // forward G-row tiles (then ceil(n / LCOLS) stencil tiles)
    int32_t active;   // pairs still iterating
};

enum { PH_INIT = 0, PH_FWD = 1, PH_ADJ_INIT = 2, PH_ADJ = 3, PH_UPD = 4 };

constexpr int WPB = BT / 32;   // warps per block

__device__ __forceinline__ int find_sys(const int64_t *__restrict__ beg, int nsys, int64_t it) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (beg[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-warp running sums of the per-pair partials.  Warp g (of NW = gridDim.x *
// WPB) takes warp items g, g + NW, ...; lane j (< RMAX, both half-warps already
// added) keeps the running sum of right-hand side j for the current system and
// writes it to slot (system, g) of `partial` when the warp moves on to a later
// system (systems skipped get 0).  Which items a warp takes, and so the order
// of every sum, depends only on the grid, so the totals are bit-reproducible
// for a given launch shape; no block-wide barrier is needed.
struct WarpSum {
    double run = 0.0;
    int cur = 0;
    __device__ __forceinline__ void put(double *partial, int sys, int64_t g, int64_t nw,
                                        double v) const {
        const int lane = threadIdx.x & 31;
        if (lane < RMAX) partial[((int64_t)sys * nw + g) * RMAX + lane] = v;
    }
    __device__ __forceinline__ void add(double ss, int s, double *partial, int64_t g, int64_t nw) {
        if (s != cur) {
            put(partial, cur, g, nw, run);
            for (int q = cur + 1; q < s; ++q) put(partial, q, g, nw, 0.0);
            run = 0.0;
            cur = s;
        }
        run += ss;
    }
    __device__ __forceinline__ void finish(double *partial, int nsys, int64_t g, int64_t nw) const {
        put(partial, cur, g, nw, run);
        for (int q = cur + 1; q < nsys; ++q) put(partial, q, g, nw, 0.0);
    }
};

// Per-lane column state: lane j of each half-warp owns right-hand side j.
struct Col {
    bool act;
    double alpha, beta;
    double lam;       // lambda of the appended lambda D rows (scaled form), else 0
};

__device__ __forceinline__ Col col_state(const LsqrScalars *sc, int j, int R) {
    Col c{false, 0.0, 0.0, 0.0};
    if (j < R) {
        const LsqrScalars &s = sc[j];
        c.act = !(s.done | s.istop);
        c.alpha = s.alpha;
        c.beta = s.beta;
        c.lam = s.lam_rows;
    }
    return c;
}

// Laplacian of column j of a strided (rows x R) block.
template <class AT, class ST>
__device__ __forceinline__ AT laplace_strided(const ST *__restrict__ x, int64_t jc, int R, int j,
                                              int nx, int ny, int nz) {
    const int k = (int)(jc % nz);
    const int64_t hh = jc / nz;
    const int ix = (int)(hh % nx), iy = (int)(hh / nx);
    const int64_t sy = (int64_t)nx * nz;
    const AT c = (AT)x[jc * R + j];
    AT s = 0;
    if (k > 0) s += c - (AT)x[(jc - 1) * R + j];
    if (k < nz - 1) s += c - (AT)x[(jc + 1) * R + j];
    if (ix > 0) s += c - (AT)x[(jc - nz) * R + j];
    if (ix < nx - 1) s += c - (AT)x[(jc + nz) * R + j];
    if (iy > 0) s += c - (AT)x[(jc - sy) * R + j];
    if (iy < ny - 1) s += c - (AT)x[(jc + sy) * R + j];
    return s;
}

// u-bar = [d; 0], v = x = w = 0; partials of ||d_j||^2.
template <class VT, class ST>
__global__ void __launch_bounds__(BT) k_binit(BSys<VT, ST> *sys, int nsys, const int64_t *beg,
                                              int64_t nitems, int TR, double *partial) {
    WarpSum ws;
    const int lane = threadIdx.x & 31, j = lane & 15, half = lane >> 4;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < nitems; it += nw) {
        const int s = find_sys(beg, nsys, it);
        BSys<VT, ST> &S = sys[s];
        const int64_t li = it - beg[s];
        const int R = S.R;
        double ss = 0.0;
        if (j < R) {
            if (li < S.nf) {
                const int64_t r0 = li * TR, r1 = r0 + TR < S.m ? r0 + TR : S.m;
                for (int64_t r = r0 + half; r < r1; r += 2) {
                    const double v = S.d[r * R + j];
                    S.U[r * S.RS + j] = (ST)v;
                    ss += v * v;
                }
            } else {
                const int64_t c0 = (li - S.nf) * LCOLS;
                const int64_t c1 = c0 + LCOLS < S.n ? c0 + LCOLS : S.n;
                for (int64_t c = c0 + half; c < c1; c += 2) {
                    S.U[(S.m + c) * S.RS + j] = (ST)0;
                    if (S.lamr) S.U[(S.m + S.n + c) * S.RS + j] = (ST)0;
                    S.V[c * S.RS + j] = (ST)0;
                    S.Vs[c * S.RS + j] = (ST)0;
                    S.X[c * R + j] = 0.0;
                    S.W[c * R + j] = 0.0;
                }
            }
        }
        ss += __shfl_xor_sync(FULL, ss, 16);
        ws.add(ss, s, partial, gw, nw);
    }
    ws.finish(partial, nsys, gw, nw);
}

__device__ __forceinline__ int pick4(const int cc[4], int ci) {
    return ci == 0 ? cc[0] : ci == 1 ? cc[1] : ci == 2 ? cc[2] : cc[3];
}

// The G rows of one forward work item (half-warp per row; lane j of each half
// ends with right-hand side j's (G v)_r).  V is stored right-hand side fastest
// with a row stride RS of 4, 8 or 16, so a run's block of V (nz depths x RS
// right-hand sides, contiguous) is read as 16-byte vectors: lane t of a
// half-warp takes the group g = t mod (RS/4) of four right-hand sides at
// depths t div (RS/4), + 16/(RS/4), ..., and each of its loads meets the other
// lanes' in one contiguous 256-byte span.  The run's value at that depth is
// loaded by the RS/4 lanes that share it.  At the row end the lanes of one
// group are summed by shuffles (fixed order) and lane j takes right-hand side
// j.  The row's first 64 cells are read into registers once and broadcast by
// shuffle.  NZC > 0 (with RS = 16) fixes nz at compile time: each lane's
// depths unroll and two runs are loaded before their products are summed.
template <int NZC, class VT, class ST>
__device__ __forceinline__ void fwd_g_item(const BSys<VT, ST> &S, int64_t li, int TR, const Col &c,
                                           ST ia, ST cu, int j, int half, double &ss) {
    using AT = ST;
    const int R = S.R, RS = NZC ? 16 : S.RS, nz = NZC ? NZC : S.nz;
    const int G4 = RS >> 2, lg = G4 >> 1;   // groups of 4; log2(G4)
    const int g = j & (G4 - 1), k0 = j >> lg, kst = 16 >> lg;
    const int64_t r0 = li * TR, r1 = r0 + TR < S.m ? r0 + TR : S.m;
    // both halves iterate the same number of times (shuffles below)
    const int64_t nrows = (r1 - r0 + 1) / 2;
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t r = r0 + 2 * t + half;
        const bool live = r < r1;
        int64_t e0 = 0, e1 = 0;
        if (live) {
            e0 = __ldg(S.row_cptr + r);
            e1 = __ldg(S.row_cptr + r + 1);
        }
        const int nrun = (int)(e1 - e0);
        int cc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            cc[i] = (j + 16 * i < nrun) ? __ldg(S.row_cells + e0 + j + 16 * i) : 0;
        // the two halves may have different run counts: loop to the max
        int nmax = nrun;
        nmax = max(nmax, __shfl_xor_sync(FULL, nmax, 16));
        AT a4[4] = {0, 0, 0, 0};
        if constexpr (NZC > 0) {
            constexpr int NI = NZC / 4;   // depths per lane (k0, k0 + 4, ...)
            const VT *vrow = S.val + e0 * NZC + k0;
            const ST *vb = S.Vs + 4 * g + k0 * 16;
            for (int e = 0; e < nmax; e += 2) {
                const int h0 = __shfl_sync(FULL, pick4(cc, e >> 4), (half << 4) | (e & 15));
                const int h1 =
                    __shfl_sync(FULL, pick4(cc, (e + 1) >> 4), (half << 4) | ((e + 1) & 15));
                if (e >= nrun) continue;
                const bool two = e + 1 < nrun;
                const int c0 = e < 64 ? h0 : __ldg(S.row_cells + e0 + e);
                const int c1 = !two ? c0 : (e + 1 < 64 ? h1 : __ldg(S.row_cells + e0 + e + 1));
                AT va[2][NI];
                ST xv[2][NI][4];
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    va[0][i] = (AT)ldval(vrow + (int64_t)e * NZC + 4 * i);
                    ldx4<ST>(vb + (int64_t)c0 * (NZC * 16) + 64 * i, xv[0][i]);
                }
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    va[1][i] = two ? (AT)ldval(vrow + (int64_t)(e + 1) * NZC + 4 * i) : (AT)0;
                    ldx4<ST>(vb + (int64_t)c1 * (NZC * 16) + 64 * i, xv[1][i]);
                }
#pragma unroll
                for (int i = 0; i < NI; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) a4[q] += va[0][i] * (AT)xv[0][i][q];
                if (two) {
#pragma unroll
                    for (int i = 0; i < NI; ++i)
#pragma unroll
                        for (int q = 0; q < 4; ++q) a4[q] += va[1][i] * (AT)xv[1][i][q];
                }
            }
        } else {
            for (int e = 0; e < nmax; ++e) {
                int h = __shfl_sync(FULL, pick4(cc, e >> 4), (half << 4) | (e & 15));
                if (e >= nrun) continue;
                if (e >= 64) h = __ldg(S.row_cells + e0 + e);
                const VT *v = S.val + (e0 + e) * nz;
                const ST *xb = S.Vs + (int64_t)h * nz * RS + 4 * g;
                for (int k = k0; k < nz; k += kst) {
                    const AT a = (AT)ldval(v + k);
                    ST xv[4];
                    ldx4<ST>(xb + (int64_t)k * RS, xv);
                    a4[0] += a * (AT)xv[0];
                    a4[1] += a * (AT)xv[1];
                    a4[2] += a * (AT)xv[2];
                    a4[3] += a * (AT)xv[3];
                }
            }
        }
        for (int off = G4; off < 16; off <<= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) a4[i] += __shfl_xor_sync(FULL, a4[i], off);
        // lane j takes component j mod 4 of group j div 4 (held by lane j div 4)
        const int sl = (half << 4) | (j >> 2);
        AT q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = __shfl_sync(FULL, a4[i], sl);
        const int cpt = j & 3;
        const AT acc = cpt == 0 ? q[0] : cpt == 1 ? q[1] : cpt == 2 ? q[2] : q[3];
        if (live && c.act) {
            const AT u = acc * ia - cu * S.U[r * RS + j];
            S.U[r * RS + j] = u;
            ss += (double)u * (double)u;
        }
    }
}

// Forward phase: G rows (fwd_g_item) and the w L rows (column tiles).
template <class VT, class ST>
__global__ void __launch_bounds__(BT, 4) k_bfwd(BSys<VT, ST> *sys, int nsys, const int64_t *beg,
                                             int64_t nitems, int TR, double *partial) {
    using AT = ST;
    WarpSum ws;
    const int lane = threadIdx.x & 31, j = lane & 15, half = lane >> 4;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < nitems; it += nw) {
        const int s = find_sys(beg, nsys, it);
        const BSys<VT, ST> &S = sys[s];
        const int64_t li = it - beg[s];
        double ss = 0.0;
        if (S.active > 0) {
            const int R = S.R, RS = S.RS, nz = S.nz;
            const int jj = j < R ? j : 0;
            const Col c = col_state(S.sc, j, R);
            const AT ia = c.alpha > 0.0 ? (AT)(1.0 / c.alpha) : (AT)0;
            const AT cu = c.beta > 0.0 ? (AT)(c.alpha / c.beta) : (AT)0;
            if (li < S.nf) {
                if (RS == 16 && nz == 16)
                    fwd_g_item<16>(S, li, TR, c, ia, cu, j, half, ss);
                else if (RS == 16 && nz == 8)
                    fwd_g_item<8>(S, li, TR, c, ia, cu, j, half, ss);
                else
                    fwd_g_item<0>(S, li, TR, c, ia, cu, j, half, ss);
            } else {
                const int64_t c0 = (li - S.nf) * LCOLS;
                const int64_t c1 = c0 + LCOLS < S.n ? c0 + LCOLS : S.n;
                const AT wsm = (AT)S.w;
                for (int64_t jc = c0 + half; jc < c1; jc += 2) {
                    const AT lap = laplace_strided<AT, ST>(S.Vs, jc, RS, jj, S.nx, S.ny, nz);
                    if (c.act) {
                        ST *up = S.U + (S.m + jc) * RS + j;
                        const AT u = wsm * lap * ia - cu * *up;
                        *up = u;
                        ss += (double)u * (double)u;
                        if (S.lamr) {   // lambda_j D v rows (the same order as the single solve)
                            ST *ul = S.U + (S.m + S.n + jc) * RS + j;
                            const AT u2 = (AT)c.lam * (AT)S.Vs[jc * RS + j] * ia - cu * *ul;
                            *ul = u2;
                            ss += (double)u2 * (double)u2;
                        }
                    }
                }
            }
        }
        ss += __shfl_xor_sync(FULL, ss, 16);
        ws.add(ss, s, partial, gw, nw);
    }
    ws.finish(partial, nsys, gw, nw);
}

constexpr int BNZ = 16;   // depths per cell held in registers by the adjoint's generic path
constexpr int BNZ_WIDE = 32;   // the same in the kernels of batches with deeper systems

// Laplacian of column jc for right-hand sides 4g..4g+3 of a block stored with
// row stride 16 (same neighbour order as laplace_strided).
template <class AT, class ST>
__device__ __forceinline__ void laplace4(const ST *__restrict__ x, int64_t jc, int g, int nx, int ny,
                                         int nz, AT out[4]) {
    const int k = (int)(jc % nz);
    const int64_t hh = jc / nz;
    const int ix = (int)(hh % nx), iy = (int)(hh / nx);
    const int64_t sy = (int64_t)nx * nz;
    const ST *p = x + jc * 16 + 4 * g;
    ST c[4];
    ldx4<ST>(p, c);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = 0;
    auto nb = [&](int64_t o) {
        ST t[4];
        ldx4<ST>(p + o * 16, t);
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] += (AT)c[q] - (AT)t[q];
    };
    if (k > 0) nb(-1);
    if (k < nz - 1) nb(1);
    if (ix > 0) nb(-nz);
    if (ix < nx - 1) nb(nz);
    if (iy > 0) nb(-sy);
    if (iy < ny - 1) nb(sy);
}

// Chunk bookkeeping shared by both adjoint paths: store this chunk's sums,
// count the finished chunks of the cell, and tell whether this warp holds the
// cell's last chunk (which then sums all chunks in chunk order).
__device__ __forceinline__ bool adj_last_chunk(unsigned *cell_done, int h, int nch, int lane,
                                               int *flag) {
    // the lanes' partial writes reach lane 0 through __syncwarp; its
    // acquire-release add publishes them and orders the last item's reads
    // of the other items' partials (from L2) after their writers' adds
    __syncwarp();
    if (lane == 0) {
        unsigned prev;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;"
                     : "=r"(prev) : "l"(cell_done + h) : "memory");
        *flag = prev == (unsigned)(nch - 1);
    }
    __syncwarp();
    const bool last = *flag != 0;
    if (last && lane == 0) cell_done[h] = 0u;
    return last;
}

// Adjoint work item with RS = 16 and nz = NZC (8 or 16): NZC lanes per row,
// lane t of a row owning right-hand sides 4g..4g+3 (g = t mod 4) at depths
// 4kq..4kq+3 (kq = t div 4); a row's u block (64 bytes) and nz values are
// read as 16-byte vectors and each lane does a 4 x 4 outer product.  The
// 32 / NZC row slots of the warp take rows q, q + 32/NZC, ... (two per step)
// and are summed by shuffles (fixed order).  Lanes 0..15 return the sum of
// squares of the new v for right-hand side = lane.
template <int NZC, class VT, class ST>
__device__ __forceinline__ double adj_item16(const BSys<VT, ST> &S, int64_t li, int init, int lane,
                                             int *flag) {
    using AT = ST;
    using WT = typename Wide<VT>::T;
    constexpr int LPR = NZC, RPW = 32 / LPR;
    const int sub = lane / LPR, t = lane % LPR, g = t & 3, kq = t >> 2;
    const int h = __ldg(S.adj_item + 2 * li);
    const int q0 = __ldg(S.adj_item + 2 * li + 1);
    const int64_t c0 = __ldg(S.cell_rptr + h);
    const int cnt = __ldg(S.cell_cnt + h);
    const int q1 = q0 + S.adj_chunk < cnt ? q0 + S.adj_chunk : cnt;
    const int32_t *rows = S.cell_rows + c0;
    const VT *vb = S.valB + c0 * NZC + 4 * kq;
    const ST *ub = S.U + 4 * g;
    AT acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    int ra = q0 + sub < q1 ? __ldg(rows + q0 + sub) : 0;
    int rb = q0 + sub + RPW < q1 ? __ldg(rows + q0 + sub + RPW) : 0;
    for (int q = q0 + sub; q < q1; q += 2 * RPW) {
        const bool two = q + RPW < q1;
        const int na = q + 2 * RPW < q1 ? __ldg(rows + q + 2 * RPW) : 0;
        const int nb = q + 3 * RPW < q1 ? __ldg(rows + q + 3 * RPW) : 0;
        ST u0[4], u1[4] = {0, 0, 0, 0};
        WT w0[4], w1[4] = {0, 0, 0, 0};
        ldx4<ST>(ub + (int64_t)ra * 16, u0);
        Pack4<VT>::ld(vb + (int64_t)q * NZC, w0);
        if (two) {
            ldx4<ST>(ub + (int64_t)rb * 16, u1);
            Pack4<VT>::ld(vb + (int64_t)(q + RPW) * NZC, w1);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += (AT)w0[a] * (AT)u0[b];
        if (two) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += (AT)w1[a] * (AT)u1[b];
        }
        ra = na;
        rb = nb;
    }
    for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += __shfl_xor_sync(FULL, acc[a][b], off);
    const int nch = cnt > S.adj_chunk ? (cnt + S.adj_chunk - 1) / S.adj_chunk : 1;
    bool finish = true;
    if (nch > 1) {
        ST *cp = S.chunk_part;
        if (sub == 0)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    cp[(li * NZC + 4 * kq + a) * RMAX + 4 * g + b] = acc[a][b];
        finish = adj_last_chunk(S.cell_done, h, nch, lane, flag);
        if (finish) {
            const int64_t first = li - q0 / S.adj_chunk;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    AT sum = 0;
                    for (int cch = 0; cch < nch; ++cch)
                        sum += (AT)__ldcg(cp + ((first + cch) * NZC + 4 * kq + a) * RMAX + 4 * g + b);
                    acc[a][b] = sum;
                }
        }
    }
    double ss4[4] = {0.0, 0.0, 0.0, 0.0};
    if (finish && sub == 0) {
        bool upd[4];
        AT ib[4], cv[4], lr[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const Col c = col_state(S.sc, 4 * g + b, S.R);
            upd[b] = c.act && (init || c.beta > 0.0);
            ib[b] = c.beta > 0.0 ? (AT)(1.0 / c.beta) : (AT)0;
            cv[b] = init ? (AT)0 : (c.alpha > 0.0 ? (AT)(c.beta / c.alpha) : (AT)0);
            lr[b] = (AT)c.lam;
        }
        const AT wsm = (AT)S.w;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t jc = (int64_t)h * NZC + 4 * kq + a;
            AT lap[4];
            laplace4<AT, ST>(S.U + S.m * 16, jc, g, S.nx, S.ny, NZC, lap);
            ST *vp = S.V + jc * 16 + 4 * g;
            const AT dj = S.D ? (AT)S.D[jc] : (AT)1;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (!upd[b]) continue;
                AT sv = acc[a][b] + wsm * lap[b];
                if (S.lamr) sv += lr[b] * (AT)S.U[(S.m + S.n + jc) * 16 + 4 * g + b];
                if (S.P) {   // finished by k_bblk
                    S.Vs[jc * 16 + 4 * g + b] = sv;
                    continue;
                }
                if (S.D) sv *= dj;
                const AT v = init ? sv * ib[b] : sv * ib[b] - cv[b] * vp[b];
                vp[b] = v;
                if (S.D) S.Vs[jc * 16 + 4 * g + b] = dj * v;
                ss4[b] += (double)v * (double)v;
            }
        }
    }
    // per right-hand side: lanes with equal g (xor 4, 8, 16), then lane j takes j
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        ss4[b] += __shfl_xor_sync(FULL, ss4[b], 4);
        ss4[b] += __shfl_xor_sync(FULL, ss4[b], 8);
        ss4[b] += __shfl_xor_sync(FULL, ss4[b], 16);
    }
    const int j = lane & 15;
    double q[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) q[b] = __shfl_sync(FULL, ss4[b], j >> 2);
    const int cpt = j & 3;
    const double r = cpt == 0 ? q[0] : cpt == 1 ? q[1] : cpt == 2 ? q[2] : q[3];
    // the cell's sums go to its slots, added in cell order by k_bred (which
    // warp, and which item of a split cell, finishes the cell varies)
    if (finish && lane < 16 && !S.P) S.cell_ss[(int64_t)h * RMAX + j] = r;
    return 0.0;
}

// Adjoint work item, any RS and nz <= BNZ: lane j = right-hand side j, the two
// half-warps take alternate rows; each row's index and u are read once and its
// nz values as nz/4 16-byte vectors (blocked CSC).  Lanes j of the first half
// return the sum of squares of the new v for right-hand side j.
template <int W, class VT, class ST>
__device__ __forceinline__ double adj_item_any(const BSys<VT, ST> &S, int64_t li, int init, int lane,
                                               int *flag) {
    constexpr int BNZ = W;
    using AT = ST;
    const int j = lane & 15, half = lane >> 4;
    const int R = S.R, RS = S.RS, nz = S.nz;
    const int jj = j < R ? j : 0;
    const Col c = col_state(S.sc, j, R);
    const bool upd = c.act && (init || c.beta > 0.0);
    const AT ib = c.beta > 0.0 ? (AT)(1.0 / c.beta) : (AT)0;
    const AT cv = init ? (AT)0 : (c.alpha > 0.0 ? (AT)(c.beta / c.alpha) : (AT)0);
    const int h = __ldg(S.adj_item + 2 * li);
    const int q0 = __ldg(S.adj_item + 2 * li + 1);
    const int64_t c0 = __ldg(S.cell_rptr + h);
    const int cnt = __ldg(S.cell_cnt + h);
    const int q1 = q0 + S.adj_chunk < cnt ? q0 + S.adj_chunk : cnt;
    const int32_t *rows = S.cell_rows + c0;
    const VT *vb = S.valB + c0 * nz;
    AT acc[BNZ];
#pragma unroll
    for (int k = 0; k < BNZ; ++k) acc[k] = 0;
    int rnext = (q0 + half < q1) ? __ldg(rows + q0 + half) : -1;
    for (int q = q0 + half; q < q1; q += 2) {
        const int r = rnext;
        rnext = (q + 2 < q1) ? __ldg(rows + q + 2) : -1;
        const AT ur = (AT)S.U[(int64_t)r * RS + jj];
        const VT *v = vb + (int64_t)q * nz;
        if ((nz & 3) == 0) {
#pragma unroll
            for (int k = 0; k < BNZ; k += 4) {
                if (k < nz) {
                    typename Wide<VT>::T w4[4];
                    Pack4<VT>::ld(v + k, w4);
                    acc[k] += (AT)w4[0] * ur;
                    acc[k + 1] += (AT)w4[1] * ur;
                    acc[k + 2] += (AT)w4[2] * ur;
                    acc[k + 3] += (AT)w4[3] * ur;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < BNZ; ++k)
                if (k < nz) acc[k] += (AT)widen(v[k]) * ur;
        }
    }
#pragma unroll
    for (int k = 0; k < BNZ; ++k) acc[k] += __shfl_xor_sync(FULL, acc[k], 16);
    const int nch = cnt > S.adj_chunk ? (cnt + S.adj_chunk - 1) / S.adj_chunk : 1;
    bool finish = true;
    if (nch > 1) {
        ST *cp = S.chunk_part;
        if (half == 0 && j < R)
#pragma unroll
            for (int k = 0; k < BNZ; ++k)
                if (k < nz) cp[(li * nz + k) * RMAX + j] = acc[k];
        finish = adj_last_chunk(S.cell_done, h, nch, lane, flag);
        if (finish) {
            const int64_t first = li - q0 / S.adj_chunk;
#pragma unroll
            for (int k = 0; k < BNZ; ++k) {
                if (k >= nz) continue;
                AT sum = 0;
                for (int cch = 0; cch < nch; ++cch)
                    sum += (AT)__ldcg(cp + ((first + cch) * nz + k) * RMAX + jj);
                acc[k] = sum;
            }
        }
    }
    double ss = 0.0;
    if (finish && half == 0 && upd) {
        const AT wsm = (AT)S.w;
#pragma unroll
        for (int k = 0; k < BNZ; ++k) {
            if (k >= nz) continue;
            const int64_t jc = (int64_t)h * nz + k;
            AT sv = acc[k] + wsm * laplace_strided<AT, ST>(S.U + S.m * RS, jc, RS, j, S.nx,
                                                           S.ny, nz);
            if (S.lamr) sv += (AT)c.lam * (AT)S.U[(S.m + S.n + jc) * RS + j];
            if (S.P) {   // finished by k_bblk
                S.Vs[jc * RS + j] = sv;
                continue;
            }
            const AT dj = S.D ? (AT)S.D[jc] : (AT)1;
            if (S.D) sv *= dj;
            ST *vp = S.V + jc * RS + j;
            const AT v = init ? sv * ib : sv * ib - cv * *vp;
            *vp = v;
            if (S.D) S.Vs[jc * RS + j] = dj * v;
            ss += (double)v * (double)v;
        }
    }
    if (finish && half == 0 && j < R && !S.P) S.cell_ss[(int64_t)h * RMAX + j] = ss;
    return 0.0;
}

// Adjoint phase: work item = a chunk of up to adj_chunk rows of one cell of
// one system (the handle's adjoint work list).  A cell split over several
// chunks is finished by its last chunk (chunk order sums).
// Items are drawn dynamically from a counter (reset by k_bred), one ahead;
// every cell's sums go to its slots, so the result does not depend on which
// warp took which item.  The per-warp partial slots stay zero.
// W = BNZ_WIDE: the kernel of batches with a system of more than BNZ depths
// (its generic path holds 32 depths per lane, two blocks per SM).
template <class VT, class ST, int W = BNZ>
__global__ void __launch_bounds__(BT, W == BNZ ? 4 : 2)
    k_badj(BSys<VT, ST> *sys, int nsys, const int64_t *beg, int64_t nitems, int init,
           double *partial, unsigned *next_item) {
    __shared__ int last_flag[WPB];
    WarpSum ws;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned nxt = 0;
    if (lane == 0) nxt = atomicAdd(next_item, 1u);
    for (int64_t it = __shfl_sync(FULL, nxt, 0); it < nitems; it = __shfl_sync(FULL, nxt, 0)) {
        if (lane == 0) nxt = atomicAdd(next_item, 1u);
        const int s = find_sys(beg, nsys, it);
        const BSys<VT, ST> &S = sys[s];
        const int64_t li = it - beg[s];
        if (S.active > 0 && li < S.n_adj) {
            if (S.RS == 16 && S.nz == 16)
                adj_item16<16>(S, li, init, lane, last_flag + warp);
            else if (S.RS == 16 && S.nz == 8)
                adj_item16<8>(S, li, init, lane, last_flag + warp);
            else if (W == BNZ || S.nz <= BNZ)
                adj_item_any<BNZ>(S, li, init, lane, last_flag + warp);
            else
                adj_item_any<W>(S, li, init, lane, last_flag + warp);
        }
    }
    ws.finish(partial, nsys, gw, nw);
}

// x += t1 w, w = v + t2 w (FP64) for pairs with a pending update; ||w||^2.
template <class VT, class ST>
__global__ void __launch_bounds__(BT) k_bupd(BSys<VT, ST> *sys, int nsys, const int64_t *beg,
                                             int64_t nitems, double *partial) {
    WarpSum ws;
    const int lane = threadIdx.x & 31, j = lane & 15, half = lane >> 4;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < nitems; it += nw) {
        const int s = find_sys(beg, nsys, it);
        const BSys<VT, ST> &S = sys[s];
        const int64_t li = it - beg[s];
        double ss = 0.0;
        if (j < S.R) {
            const LsqrScalars &sc = S.sc[j];
            const int pend = sc.pending;
            if (pend) {
                const double ia = sc.alpha > 0.0 ? 1.0 / sc.alpha : 0.0;
                const double t1 = sc.t1, t2 = sc.t2;
                const int64_t c0 = li * LCOLS, c1 = c0 + LCOLS < S.n ? c0 + LCOLS : S.n;
                for (int64_t c = c0 + half; c < c1; c += 2) {
                    const int64_t i = c * S.R + j;
                    const double v = (double)S.V[c * S.RS + j] * ia;
                    double w = S.W[i];
                    if (pend == 2) {
                        w = v;
                    } else {
                        S.X[i] += t1 * w;
                        w = v + t2 * w;
                    }
                    S.W[i] = w;
                    ss += w * w;
                }
            }
        }
        ss += __shfl_xor_sync(FULL, ss, 16);
        ws.add(ss, s, partial, gw, nw);
    }
    ws.finish(partial, nsys, gw, nw);
}

// m = D o x (scaled form) or x, n x R per system.
__global__ void k_bfinal(int64_t n, int R, const double *__restrict__ D, const double *__restrict__ X,
                         double *m_out) {
    const int64_t total = n * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        m_out[i] = D ? D[i / R] * X[i] : X[i];
}

// m = P x with the depth blocks: m[(h nz + k) R + j] = sum_{i >= k} P_h[k][i] x[(h nz + i) R + j].
template <class ST>
__global__ void k_bfinal_blk(int64_t n, int nz, int R, const ST *__restrict__ P,
                             const double *__restrict__ X, double *m_out) {
    const int64_t total = n * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / R;
        const int j = (int)(e - col * R);
        const int64_t h = col / nz;
        const int k = (int)(col - h * nz);
        const ST *Pr = P + (h * nz + k) * nz;
        double sum = 0.0;
        for (int i = k; i < nz; ++i) sum += (double)Pr[i] * X[(h * nz + i) * R + j];
        m_out[e] = sum;
    }
}

// The depth-block finish of the adjoint (precond = 2): half-warp per cell (two
// cells per warp item), lane j = right-hand side j.  Reads s = A^T u from Vs,
// t = P_h^T s (in place, depths descending), v-bar = t / beta - (beta/alpha)
// v-bar (start step: t / beta), Vs = P_h v-bar; the cell's sum of v-bar^2 per
// right-hand side goes to its slot (added in cell order by k_bred).  The
// blocks are read once per cell and broadcast to the lanes.
template <class VT, class ST, int BNZ = pdst::BNZ>
__global__ void __launch_bounds__(BT) k_bblk(BSys<VT, ST> *sys, int nsys, const int64_t *beg,
                                             int64_t nitems, int init) {
    using AT = ST;
    const int lane = threadIdx.x & 31, j = lane & 15, half = lane >> 4;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < nitems; it += nw) {
        const int s = find_sys(beg, nsys, it);
        const BSys<VT, ST> &S = sys[s];
        const int nz = S.nz;
        const int64_t H = S.n / nz;
        const int64_t h = 2 * (it - beg[s]) + half;
        if (S.active == 0 || h >= H || j >= S.R) continue;
        const Col c = col_state(S.sc, j, S.R);
        const bool upd = c.act && (init || c.beta > 0.0);
        double ss = 0.0;
        if (upd) {
            const AT ib = c.beta > 0.0 ? (AT)(1.0 / c.beta) : (AT)0;
            const AT cv = init ? (AT)0 : (c.alpha > 0.0 ? (AT)(c.beta / c.alpha) : (AT)0);
            const ST *P = S.P + h * nz * nz;
            const int64_t c0 = h * nz;
            AT a[BNZ];
#pragma unroll
            for (int k = 0; k < BNZ; ++k) a[k] = k < nz ? (AT)S.Vs[(c0 + k) * S.RS + j] : (AT)0;
#pragma unroll
            for (int k = BNZ - 1; k >= 0; --k) {
                if (k >= nz) continue;
                AT t = 0;
#pragma unroll
                for (int i = 0; i <= k; ++i) t += (AT)P[i * nz + k] * a[i];
                a[k] = t;
            }
#pragma unroll
            for (int k = 0; k < BNZ; ++k) {
                if (k >= nz) continue;
                ST *vp = S.V + (c0 + k) * S.RS + j;
                const AT v = init ? a[k] * ib : a[k] * ib - cv * *vp;
                *vp = v;
                a[k] = v;
                ss += (double)v * (double)v;
            }
#pragma unroll
            for (int k = 0; k < BNZ; ++k) {
                if (k >= nz) continue;
                AT q = 0;
#pragma unroll
                for (int i = k; i < BNZ; ++i)
                    if (i < nz) q += (AT)P[k * nz + i] * a[i];
                S.Vs[(c0 + k) * S.RS + j] = q;
            }
        }
        S.cell_ss[h * RMAX + j] = ss;
    }
}

// One block of 256 threads per system: thread (l, j) sums the partials of the
// producing kernel's warps l, l + 16, ... (G warps) for right-hand side j, then thread j adds the 16 sums in
// order (deterministic) and advances that pair's scalars; thread 0 finally
// counts the pairs still iterating.
constexpr int RED_T = 256;

template <class VT, class ST>
__global__ void __launch_bounds__(RED_T) k_bred(BSys<VT, ST> *sys, int G, const double *partial,
                                                int phase, int *active_out,
                                                unsigned *adj_counter) {
    __shared__ double part[RED_T / RMAX][RMAX];
    const int s = blockIdx.x, t = threadIdx.x, j = t % RMAX, l = t / RMAX;
    BSys<VT, ST> &S = sys[s];
    // both sums take their terms in index order, the loads issued eight at a
    // time (one L2 round trip per eight terms); slots past the end add +0.0,
    // which leaves these sums of squares unchanged bit for bit
    constexpr int LS = RED_T / RMAX;
    double acc = 0.0;
    for (int b = l; b < G; b += 8 * LS) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = b + u * LS < G ? partial[((int64_t)s * G + b + u * LS) * RMAX + j] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    if (phase == PH_ADJ_INIT || phase == PH_ADJ) {
        if (s == 0 && t == 0) *adj_counter = 0u;   // for the next adjoint launch
        const int H = S.n / S.nz;
        for (int hh = l; hh < H; hh += 8 * LS) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = hh + u * LS < H ? __ldcg(S.cell_ss + (int64_t)(hh + u * LS) * RMAX + j) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
        }
    }
    part[l][j] = acc;
    __syncthreads();
    if (t < RMAX && j < S.R) {
        LsqrScalars *sc = S.sc + j;
        const bool frozen = (phase == PH_UPD) ? !sc->pending : (sc->done | sc->istop) != 0;
        if (!frozen) {
            double tsum = 0.0;
            for (int k = 0; k < RED_T / RMAX; ++k) tsum += part[k][j];
            if (phase == PH_INIT) {
                const double b = sqrt(tsum);
                sc->beta = b;
                sc->bnorm = b;
                sc->rnorm = b;
                sc->phibar = b;
                if (!isfinite(b)) sc->err = 1;
                if (!(b > 0.0) || !isfinite(b)) sc->done = 1;
            } else if (phase == PH_FWD) {
                const double b = sqrt(tsum);
                if (!isfinite(b)) {
                    sc->err = 1;
                    sc->done = 1;
                }
                sc->beta = b;
            } else if (phase == PH_ADJ_INIT || phase == PH_ADJ) {
                const double an = (phase == PH_ADJ && !(sc->beta > 0.0)) ? sc->alpha : sqrt(tsum);
                if (!isfinite(an)) {
                    sc->err = 1;
                    sc->done = 1;
                } else if (phase == PH_ADJ_INIT) {
                    sc->alpha = an;
                    sc->rhobar = an;
                    sc->arnorm = an * sc->beta;
                    sc->pending = 2;
                    if (!(sc->arnorm > 0.0)) sc->done = 1;
                } else {
                    lsqr_step(sc, an);
                }
            } else {
                sc->wnorm2 = tsum;
                sc->pending = 0;
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        int a = 0;
        for (int k = 0; k < S.R; ++k) a += !(S.sc[k].done | S.sc[k].istop);
        S.active = a;
        active_out[s] = a;
    }
}

// ------------------------------------------------------------------ driver

struct BatchKey {
    std::vector<uint64_t> hs;   // handle uids
    std::vector<int32_t> nrhs;
    int dtype;
    int precond;
    bool operator<(const BatchKey &o) const {
        return std::tie(hs, nrhs, dtype, precond) < std::tie(o.hs, o.nrhs, o.dtype, o.precond);
    }
};

struct BatchWork {
    BatchKey key;
    int TR = 0;
    bool tuned = false;
    bool wide = false;   // a system has more than BNZ depths: the W = BNZ_WIDE kernels
    std::vector<DevBuf *> bufs;
    DevBuf desc, scal, partial, fbeg, abeg, ubeg, bbeg, active, adj_ctr;
    int *h_active = nullptr;
    LsqrScalars *h_scal = nullptr;
    int64_t nf_items = 0, na_items = 0, nu_items = 0, nb_items = 0;
    unsigned gi = 1, gf = 1, ga = 1, gu = 1, gb = 1;   // grids of init / forward / adjoint /
                                                       // update / depth-block finish
    std::vector<int64_t> hf, ha, hu, hb;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<double> tune_ms;
    ~BatchWork() {
        for (auto *b : bufs) delete b;
        for (auto &g : graphs)
            if (g.second) cudaGraphExecDestroy(g.second);
        if (h_active) cudaFreeHost(h_active);
        if (h_scal) cudaFreeHost(h_scal);
    }
};

static std::mutex g_batch_mutex;
static BatchWork *g_batch = nullptr;   // the most recent batch (reused when identical)

template <class K> static unsigned bgrid(K kernel, int device, int64_t items) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BT, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)num_sms(device) * per_sm;
    int64_t need = (items + (BT / 32) - 1) / (BT / 32);
    if (need < 1) need = 1;
    return (unsigned)(g < need ? g : need);
}

static int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// V row stride: R rounded up to 4, 8 or 16 (16-byte groups that divide 16 lanes).
static int v_stride(int R) { return R <= 4 ? 4 : R <= 8 ? 8 : 16; }

template <class VT, class ST> struct Batched {
    using Sys = BSys<VT, ST>;

    // Forward item layout for TR rows per item.
    static void layout_fwd(const std::vector<pdst_handle *> &hs, int TR, std::vector<int64_t> &beg,
                           std::vector<int64_t> &nf) {
        beg.assign(hs.size() + 1, 0);
        nf.resize(hs.size());
        for (size_t s = 0; s < hs.size(); ++s) {
            nf[s] = (hs[s]->m + TR - 1) / TR;
            const int64_t nl = ((int64_t)hs[s]->n + LCOLS - 1) / LCOLS;
            beg[s + 1] = beg[s] + round_up(nf[s] + nl, WPB);
        }
    }

    static pdst_status prepare(BatchWork *bw, const std::vector<pdst_handle *> &hs,
                               const int32_t *nrhs, int dtype, int TR, cudaStream_t s) {
        const bool scaled = bw->key.precond != 0;
        const bool blk = bw->key.precond == 2;
        const int nsys = (int)hs.size();
        std::vector<Sys> d(nsys);
        std::vector<int64_t> nf;
        layout_fwd(hs, TR, bw->hf, nf);
        bw->ha.assign(nsys + 1, 0);
        bw->hu.assign(nsys + 1, 0);
        bw->hb.assign(nsys + 1, 0);
        for (int i = 0; i < nsys; ++i) {
            pdst_handle *h = hs[i];
            bw->ha[i + 1] = bw->ha[i] + round_up(h->n_adj, WPB);
            bw->hu[i + 1] = bw->hu[i] + round_up(((int64_t)h->n + LCOLS - 1) / LCOLS, WPB);
            bw->hb[i + 1] = bw->hb[i] + ((int64_t)h->H + 1) / 2;   // two cells per warp item
        }
        bw->nf_items = bw->hf[nsys];
        bw->na_items = bw->ha[nsys];
        bw->nu_items = bw->hu[nsys];
        bw->nb_items = bw->hb[nsys];
        const int device = hs[0]->device;
        bw->gi = bgrid(k_binit<VT, ST>, device, bw->nf_items);
        bw->gf = bgrid(k_bfwd<VT, ST>, device, bw->nf_items);
        int maxnz = 0;
        for (auto *h : hs) maxnz = std::max(maxnz, (int)h->nz);
        bw->wide = maxnz > BNZ;
        bw->ga = bw->wide ? bgrid(k_badj<VT, ST, BNZ_WIDE>, device, bw->na_items)
                          : bgrid(k_badj<VT, ST>, device, bw->na_items);
        bw->gu = bgrid(k_bupd<VT, ST>, device, bw->nu_items);
        bw->gb = bw->wide ? bgrid(k_bblk<VT, ST, BNZ_WIDE>, device, std::max<int64_t>(bw->nb_items, 1))
                          : bgrid(k_bblk<VT, ST>, device, std::max<int64_t>(bw->nb_items, 1));
        const int64_t maxg = std::max(std::max(bw->gi, bw->gf), std::max(bw->ga, bw->gu));
        // (re)allocate vectors only on a new batch
        if (bw->bufs.empty()) {
            for (int i = 0; i < nsys; ++i) {
                pdst_handle *h = hs[i];
                const int R = nrhs[i];
                DevBuf *U = new DevBuf, *V = new DevBuf, *X = new DevBuf, *W = new DevBuf;
                DevBuf *CP = new DevBuf, *CD = new DevBuf, *CS = new DevBuf, *VS = new DevBuf;
                bw->bufs.insert(bw->bufs.end(), {U, V, X, W, CP, CD, CS, VS});
                const int64_t csb = sizeof(double) * std::max<int64_t>((int64_t)h->H * RMAX, 1);
                PDST_TRY(CS->alloc(csb));
                PDST_CUDA(cudaMemsetAsync(CS->p, 0, csb, s));
                PDST_TRY(CP->alloc(sizeof(ST) * std::max<int64_t>(h->n_adj * h->nz * RMAX, 1)));
                PDST_TRY(CD->alloc(sizeof(unsigned) * std::max<int32_t>(h->H, 1)));
                PDST_CUDA(cudaMemsetAsync(CD->p, 0, sizeof(unsigned) * std::max<int32_t>(h->H, 1), s));
                const int64_t ubytes =
                    sizeof(ST) * (h->m + h->n + (scaled ? h->n : 0)) * v_stride(R);
                PDST_TRY(U->alloc(ubytes));
                PDST_CUDA(cudaMemsetAsync(U->p, 0, ubytes, s));
                const int64_t vbytes = sizeof(ST) * std::max<int64_t>((int64_t)h->n * v_stride(R), 1);
                PDST_TRY(V->alloc(vbytes));
                PDST_CUDA(cudaMemsetAsync(V->p, 0, vbytes, s));
                if (scaled) {
                    PDST_TRY(VS->alloc(vbytes));
                    PDST_CUDA(cudaMemsetAsync(VS->p, 0, vbytes, s));
                }
                PDST_TRY(X->alloc(sizeof(double) * (int64_t)h->n * R));
                PDST_TRY(W->alloc(sizeof(double) * (int64_t)h->n * R));
            }
            PDST_TRY(bw->scal.alloc(sizeof(LsqrScalars) * nsys * RMAX));
            PDST_TRY(bw->desc.alloc(sizeof(Sys) * nsys));
            PDST_TRY(bw->active.alloc(sizeof(int) * nsys));
            PDST_TRY(bw->adj_ctr.alloc(sizeof(unsigned)));
            PDST_TRY(bw->abeg.alloc(sizeof(int64_t) * (nsys + 1)));
            PDST_TRY(bw->ubeg.alloc(sizeof(int64_t) * (nsys + 1)));
            PDST_TRY(bw->bbeg.alloc(sizeof(int64_t) * (nsys + 1)));
            PDST_CUDA(cudaMallocHost(&bw->h_active, sizeof(int) * nsys));
            PDST_CUDA(cudaMallocHost(&bw->h_scal, sizeof(LsqrScalars) * nsys * RMAX));
        }
        PDST_TRY(bw->partial.alloc(sizeof(double) * RMAX * nsys * maxg * WPB));
        PDST_TRY(bw->fbeg.alloc(sizeof(int64_t) * (nsys + 1)));
        LsqrScalars *scd = bw->scal.as<LsqrScalars>();
        for (int i = 0; i < nsys; ++i) {
            pdst_handle *h = hs[i];
            Sys &q = d[i];
            q.m = h->m;
            q.n = h->n;
            q.nx = h->grid.nx;
            q.ny = h->grid.ny;
            q.nz = h->nz;
            q.R = nrhs[i];
            q.RS = v_stride(nrhs[i]);
            q.n_adj = h->n_adj;
            q.row_cptr = h->row_cptr.as<int64_t>();
            q.row_cells = h->row_cells.as<int32_t>();
            q.val = h->vals[dtype].csr.as<VT>();
            q.cell_rptr = h->cell_rptr.as<int64_t>();
            q.cell_cnt = h->cell_cnt.as<int32_t>();
            q.cell_rows = h->cell_rows.as<int32_t>();
            q.cell_order = h->cell_order.as<int32_t>();
            q.valB = h->vals[dtype].bcsc.as<VT>();
            q.U = bw->bufs[NB * i]->as<ST>();
            q.V = bw->bufs[NB * i + 1]->as<ST>();
            q.Vs = scaled ? bw->bufs[NB * i + 7]->as<ST>() : q.V;
            q.D = (scaled && !blk) ? h->colscale.as<double>() : nullptr;
            q.P = !blk ? nullptr
                       : static_cast<const ST *>(sizeof(ST) == sizeof(double) ? h->blkP64.p
                                                                              : h->blkP32.p);
            q.lamr = scaled ? 1 : 0;
            q.X = bw->bufs[NB * i + 2]->as<double>();
            q.W = bw->bufs[NB * i + 3]->as<double>();
            q.chunk_part = bw->bufs[NB * i + 4]->as<ST>();
            q.cell_done = bw->bufs[NB * i + 5]->as<unsigned>();
            q.cell_ss = bw->bufs[NB * i + 6]->as<double>();
            q.adj_item = h->adj_item.as<int32_t>();
            q.adj_chunk = h->adj_chunk;
            q.sc = scd + (size_t)i * RMAX;
            q.nf = nf[i];
            q.active = 0;
        }
        bw->TR = TR;
        PDST_CUDA(cudaMemcpyAsync(bw->desc.p, d.data(), sizeof(Sys) * nsys, cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaMemcpyAsync(bw->fbeg.p, bw->hf.data(), sizeof(int64_t) * (nsys + 1),
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaMemcpyAsync(bw->abeg.p, bw->ha.data(), sizeof(int64_t) * (nsys + 1),
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaMemcpyAsync(bw->ubeg.p, bw->hu.data(), sizeof(int64_t) * (nsys + 1),
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaMemcpyAsync(bw->bbeg.p, bw->hb.data(), sizeof(int64_t) * (nsys + 1),
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        return PDST_OK;
    }

    // per-call inputs: right-hand sides and scalars
    static pdst_status load_inputs(BatchWork *bw, int nsys, const double *const *d_dev,
                                   const std::vector<LsqrScalars> &init, cudaStream_t s) {
        std::vector<Sys> d(nsys);
        PDST_CUDA(cudaMemcpyAsync(d.data(), bw->desc.p, sizeof(Sys) * nsys, cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nsys; ++i) {
            d[i].d = d_dev[i];
            d[i].w = init[(size_t)i * RMAX].w_smooth;
            d[i].active = d[i].R;
        }
        PDST_CUDA(cudaMemcpyAsync(bw->desc.p, d.data(), sizeof(Sys) * nsys, cudaMemcpyHostToDevice, s));
        for (int i = 0; i < nsys; ++i)
            PDST_CUDA(cudaMemsetAsync(bw->bufs[NB * i + 5]->p, 0, bw->bufs[NB * i + 5]->bytes, s));
        PDST_CUDA(cudaMemsetAsync(bw->adj_ctr.p, 0, sizeof(unsigned), s));
        std::copy(init.begin(), init.end(), bw->h_scal);
        PDST_CUDA(cudaMemcpyAsync(bw->scal.p, bw->h_scal, sizeof(LsqrScalars) * nsys * RMAX,
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        return PDST_OK;
    }

    // The adjoint phase (and, with depth blocks, the cells' finish) in the
    // kernels of the batch's width.
    static void launch_adj(BatchWork *bw, int nsys, int init, cudaStream_t s) {
        Sys *sys = bw->desc.as<Sys>();
        double *part = bw->partial.as<double>();
        unsigned *ctr = bw->adj_ctr.as<unsigned>();
        const int64_t *ab = bw->abeg.as<int64_t>(), *bb = bw->bbeg.as<int64_t>();
        if (bw->wide)
            k_badj<VT, ST, BNZ_WIDE><<<bw->ga, BT, 0, s>>>(sys, nsys, ab, bw->na_items, init, part,
                                                          ctr);
        else
            k_badj<VT, ST><<<bw->ga, BT, 0, s>>>(sys, nsys, ab, bw->na_items, init, part, ctr);
        if (bw->key.precond == 2) {
            if (bw->wide)
                k_bblk<VT, ST, BNZ_WIDE><<<bw->gb, BT, 0, s>>>(sys, nsys, bb, bw->nb_items, init);
            else
                k_bblk<VT, ST><<<bw->gb, BT, 0, s>>>(sys, nsys, bb, bw->nb_items, init);
        }
    }

    static void launch_iter(BatchWork *bw, int nsys, cudaStream_t s) {
        Sys *sys = bw->desc.as<Sys>();
        double *part = bw->partial.as<double>();
        int *act = bw->active.as<int>();
        unsigned *ctr = bw->adj_ctr.as<unsigned>();
        k_bfwd<VT, ST><<<bw->gf, BT, 0, s>>>(sys, nsys, bw->fbeg.as<int64_t>(), bw->nf_items, bw->TR,
                                             part);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->gf * WPB), part, PH_FWD, act, ctr);
        launch_adj(bw, nsys, 0, s);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->ga * WPB), part, PH_ADJ, act, ctr);
        k_bupd<VT, ST><<<bw->gu, BT, 0, s>>>(sys, nsys, bw->ubeg.as<int64_t>(), bw->nu_items, part);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->gu * WPB), part, PH_UPD, act, ctr);
    }

    static pdst_status start(BatchWork *bw, int nsys, cudaStream_t s) {
        Sys *sys = bw->desc.as<Sys>();
        double *part = bw->partial.as<double>();
        int *act = bw->active.as<int>();
        unsigned *ctr = bw->adj_ctr.as<unsigned>();
        k_binit<VT, ST><<<bw->gi, BT, 0, s>>>(sys, nsys, bw->fbeg.as<int64_t>(), bw->nf_items, bw->TR,
                                              part);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->gi * WPB), part, PH_INIT, act, ctr);
        launch_adj(bw, nsys, 1, s);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->ga * WPB), part, PH_ADJ_INIT, act, ctr);
        k_bupd<VT, ST><<<bw->gu, BT, 0, s>>>(sys, nsys, bw->ubeg.as<int64_t>(), bw->nu_items, part);
        k_bred<VT, ST><<<nsys, RED_T, 0, s>>>(sys, (int)(bw->gu * WPB), part, PH_UPD, act, ctr);
        PDST_CUDA(cudaGetLastError());
        return PDST_OK;
    }

    // Time one whole iteration for each candidate tile and keep the fastest
    // (the start-up phase runs first, so the iterations do real work).
    static pdst_status autotune(BatchWork *bw, const std::vector<pdst_handle *> &hs,
                                const int32_t *nrhs, int dtype, const double *const *d_dev,
                                const std::vector<LsqrScalars> &init, int device, cudaStream_t s) {
        const int cands[] = {2, 8, 32};
        double best = 1e300;
        int best_tr = 8;
        bw->tune_ms.clear();
        const int nsys = (int)hs.size();
        cudaEvent_t e0, e1;
        PDST_CUDA(cudaEventCreate(&e0));
        PDST_CUDA(cudaEventCreate(&e1));
        for (int tr : cands) {
            PDST_TRY(prepare(bw, hs, nrhs, dtype, tr, s));
            PDST_TRY(load_inputs(bw, nsys, d_dev, init, s));
            PDST_TRY(start(bw, nsys, s));
            Sys *sys = bw->desc.as<Sys>();
            float ms = 0.f, tot = 0.f;
            (void)sys;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                launch_iter(bw, nsys, s);
                cudaEventRecord(e1, s);
                PDST_CUDA(cudaEventSynchronize(e1));
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;
            }
            bw->tune_ms.push_back(tot / 2);
            if (tot / 2 < best) {
                best = tot / 2;
                best_tr = tr;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return prepare(bw, hs, nrhs, dtype, best_tr, s);
    }

    static pdst_status run(BatchWork *bw, const std::vector<pdst_handle *> &hs, const int32_t *nrhs,
                           int dtype, const double *const *d_dev, const std::vector<LsqrScalars> &init,
                           int kblock, int tile_rows, double *const *m_out, cudaStream_t s,
                           int &launches) {
        const int nsys = (int)hs.size();
        const int device = hs[0]->device;
        // tile_rows > 0: use it; 0: use the autotuned tile (tune once per batch)
        const bool want_tune = tile_rows == 0 && !bw->tuned;
        const bool want_fixed = tile_rows > 0 && (tile_rows != bw->TR || bw->tuned);
        if (want_tune || want_fixed || bw->TR == 0) {
            for (auto &g : bw->graphs)
                if (g.second) cudaGraphExecDestroy(g.second);
            bw->graphs.clear();
            if (tile_rows > 0) {
                PDST_TRY(prepare(bw, hs, nrhs, dtype, tile_rows, s));
                bw->tuned = false;
            } else {
                PDST_TRY(autotune(bw, hs, nrhs, dtype, d_dev, init, device, s));
                bw->tuned = true;
            }
        }
        PDST_TRY(load_inputs(bw, nsys, d_dev, init, s));
        PDST_TRY(start(bw, nsys, s));
        const int per_iter = bw->key.precond == 2 ? 7 : 6;
        launches += per_iter;
        cudaGraphExec_t exec = nullptr;
        auto it = bw->graphs.find(kblock);
        if (it != bw->graphs.end()) {
            exec = it->second;
        } else {
            cudaStream_t cs;
            PDST_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int i = 0; i < kblock; ++i) launch_iter(bw, nsys, cs);
                e = cudaStreamEndCapture(cs, &g);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                set_error("batched LSQR graph capture: %s", cudaGetErrorString(e));
                return PDST_ERR_CUDA;
            }
            bw->graphs[kblock] = exec;
        }
        for (;;) {
            PDST_CUDA(cudaMemcpyAsync(bw->h_active, bw->active.p, sizeof(int) * nsys,
                                      cudaMemcpyDeviceToHost, s));
            PDST_CUDA(cudaStreamSynchronize(s));
            int any = 0;
            for (int i = 0; i < nsys; ++i) any += bw->h_active[i];
            if (!any) break;
            PDST_CUDA(cudaGraphLaunch(exec, s));
            launches += per_iter * kblock;
        }
        for (int i = 0; i < nsys; ++i) {
            const int64_t n = hs[i]->n;
            const unsigned g = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>((n * nrhs[i] + BT - 1) / BT, (int64_t)num_sms(device) * 8));
            if (bw->key.precond == 2)
                k_bfinal_blk<ST><<<g, BT, 0, s>>>(
                    n, hs[i]->nz, nrhs[i],
                    static_cast<const ST *>(sizeof(ST) == sizeof(double) ? hs[i]->blkP64.p
                                                                         : hs[i]->blkP32.p),
                    bw->bufs[NB * i + 2]->as<double>(), m_out[i]);
            else
                k_bfinal<<<g, BT, 0, s>>>(n, nrhs[i],
                                          bw->key.precond ? hs[i]->colscale.as<double>() : nullptr,
                                          bw->bufs[NB * i + 2]->as<double>(), m_out[i]);
        }
        PDST_CUDA(cudaGetLastError());
        launches += nsys;
        PDST_CUDA(cudaMemcpyAsync(bw->h_scal, bw->scal.p, sizeof(LsqrScalars) * nsys * RMAX,
                                  cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        return PDST_OK;
    }
};

}  // namespace
}  // namespace pdst

using namespace pdst;

extern "C" void pdst_batched_opts_default(pdst_batched_opts *o) {
    if (!o) return;
    o->tile_rows = 0;
    o->kblock = 8;
    o->chosen_tile_rows = 0;
    o->kernel_launches = 0;
    for (int i = 0; i < 4; ++i) o->tune_ms[i] = 0.0;
    o->precond = 0;
    o->reserved = 0;
}

extern "C" pdst_status pdst_lsqr_batched(int32_t nsys, const pdst_handle_t *hs, const int32_t *nrhs,
                                         const double *const *d_dev, const double *w,
                                         const double *const *lambda, int32_t itmax, double tol,
                                         int32_t dtype, double *const *m_out_dev,
                                         pdst_lsqr_info *infos, pdst_batched_opts *opts,
                                         void *stream) {
    PDST_CHECK_ARG(nsys >= 1 && hs && nrhs && d_dev && w && lambda && m_out_dev,
                   "pdst_lsqr_batched: NULL argument or nsys < 1");
    PDST_CHECK_ARG(dtype >= 0 && dtype <= 2, "pdst_lsqr_batched: unknown dtype");
    PDST_CHECK_ARG(itmax >= 0, "pdst_lsqr_batched: itmax must be >= 0");
    PDST_CHECK_ARG(std::isfinite(tol) && tol >= 0.0, "pdst_lsqr_batched: tol must be >= 0");
    std::vector<pdst_handle *> H(nsys);
    for (int i = 0; i < nsys; ++i) {
        PDST_CHECK_ARG(hs[i] != nullptr, "pdst_lsqr_batched: handle %d is NULL", i);
        PDST_CHECK_ARG(nrhs[i] >= 1 && nrhs[i] <= RMAX,
                       "pdst_lsqr_batched: nrhs[%d] must be in 1..%d", i, RMAX);
        PDST_CHECK_ARG(hs[i]->device == hs[0]->device,
                       "pdst_lsqr_batched: all handles must be on one device");
        PDST_CHECK_ARG(hs[i]->m == 0 || d_dev[i], "pdst_lsqr_batched: d[%d] is NULL", i);
        PDST_CHECK_ARG(m_out_dev[i] && lambda[i], "pdst_lsqr_batched: NULL output or lambda");
        PDST_CHECK_ARG(std::isfinite(w[i]) && w[i] >= 0.0, "pdst_lsqr_batched: bad w[%d]", i);
        for (int j = 0; j < nrhs[i]; ++j)
            PDST_CHECK_ARG(std::isfinite(lambda[i][j]) && lambda[i][j] >= 0.0,
                           "pdst_lsqr_batched: bad lambda[%d][%d]", i, j);
        if (!hs[i]->vals[dtype].present) {
            set_error("pdst_lsqr_batched: values of dtype %d were not kept in handle %d", dtype, i);
            return PDST_ERR_STATE;
        }
        if (hs[i]->nz > BNZ_WIDE) {
            set_error("pdst_lsqr_batched: nz = %d in handle %d; the batched form supports nz <= %d",
                      hs[i]->nz, i, BNZ_WIDE);
            return PDST_ERR_LIMIT;
        }
        H[i] = hs[i];
    }
    pdst_batched_opts local;
    pdst_batched_opts_default(&local);
    if (opts) local = *opts;
    const int kblock = local.kblock > 0 ? local.kblock : 8;
    PDST_CHECK_ARG(local.precond >= 0 && local.precond <= 2,
                   "pdst_lsqr_batched: unknown precond %d", local.precond);
    for (int i = 0; i < nsys; ++i) {
        if (local.precond == 1 && !hs[i]->has_colscale) {
            set_error("pdst_lsqr_batched: precond = 1 needs pdst_set_col_scaling on handle %d", i);
            return PDST_ERR_STATE;
        }
        if (local.precond == 2 && !hs[i]->has_blkprec) {
            set_error("pdst_lsqr_batched: precond = 2 needs pdst_set_block_precond on handle %d",
                      i);
            return PDST_ERR_STATE;
        }
    }
    PDST_CHECK_ARG(kblock <= 256, "pdst_lsqr_batched: kblock must be <= 256");
    PDST_CHECK_ARG(local.tile_rows >= 0 && local.tile_rows <= 4096,
                   "pdst_lsqr_batched: tile_rows out of range");

    std::vector<LsqrScalars> init((size_t)nsys * RMAX);
    for (int i = 0; i < nsys; ++i)
        for (int j = 0; j < RMAX; ++j) {
            LsqrScalars &q = init[(size_t)i * RMAX + j];
            q = LsqrScalars{};
            q.cs2 = -1.0;
            const double lam = j < nrhs[i] ? lambda[i][j] : 0.0;
            // scaled form: lambda_j D rows in the operator, no recurrence damping
            q.damp = local.precond ? 0.0 : lam;
            q.lam_rows = local.precond ? lam : 0.0;
            q.atol = tol;
            q.btol = tol;
            q.ctol = 1e-8;
            q.w_smooth = w[i];
            q.itmax = itmax;
            if (j >= nrhs[i] || itmax == 0) q.done = 1;
        }

    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchKey key{std::vector<uint64_t>(nsys), std::vector<int32_t>(nrhs, nrhs + nsys), dtype,
                 local.precond};
    for (int i = 0; i < nsys; ++i) key.hs[i] = hs[i]->uid;
    if (!g_batch || g_batch->key < key || key < g_batch->key) {
        delete g_batch;
        g_batch = new BatchWork();
        g_batch->key = key;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    pdst_status st;
    if (dtype == PDST_F64)
        st = Batched<double, double>::run(g_batch, H, nrhs, dtype, d_dev, init, kblock,
                                          local.tile_rows, m_out_dev, s, launches);
    else if (dtype == PDST_F32)
        st = Batched<float, float>::run(g_batch, H, nrhs, dtype, d_dev, init, kblock,
                                        local.tile_rows, m_out_dev, s, launches);
    else
        st = Batched<__nv_bfloat16, float>::run(g_batch, H, nrhs, dtype, d_dev, init, kblock,
                                                local.tile_rows, m_out_dev, s, launches);
    if (st != PDST_OK) {
        delete g_batch;
        g_batch = nullptr;
        return st;
    }
    if (opts) {
        opts->chosen_tile_rows = g_batch->TR;
        opts->kernel_launches = launches;
        for (size_t i = 0; i < 4; ++i)
            opts->tune_ms[i] = i < g_batch->tune_ms.size() ? g_batch->tune_ms[i] : 0.0;
    }
    bool err = false;
    size_t k = 0;
    for (int i = 0; i < nsys; ++i)
        for (int j = 0; j < nrhs[i]; ++j) {
            const LsqrScalars &c = g_batch->h_scal[(size_t)i * RMAX + j];
            err |= c.err != 0;
            if (infos) {
                pdst_lsqr_info &f = infos[k++];
                f = pdst_lsqr_info{};
                f.iters = c.itn;
                f.istop = c.istop;
                f.rnorm = c.rnorm;
                f.arnorm = c.arnorm;
                f.anorm = c.anorm;
                f.acond = c.acond;
                f.xnorm = c.xnorm;
                f.bnorm = c.bnorm;
            }
        }
    if (err) {
        set_error("pdst_lsqr_batched: non-finite value in a recurrence");
        return PDST_ERR_BREAKDOWN;
    }
    return PDST_OK;
}
