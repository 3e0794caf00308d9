// build_g.cu -- on-device assembly of the sensitivity matrix G (Eq. 5-7,
// synthetic form) and of its transpose.
//
// G[r, h*nz + k] = l_h(r) * Kdz[t(r)][k]: every horizontal cell h that ray r
// crosses contributes all nz depth columns (Eq. 5), columns ordered depth
// fastest (Eq. 7).  l_h(r) comes from cutting the quadratic Bezier ray into
// N = max(1, ceil(4 * polygon_length / dx)) equal-parameter chords, giving
// each chord to the cell of its midpoint (clamped into the grid) and summing
// the chord lengths of a cell in chord order.
//
// Every floating-point operation of that recipe is written with an explicit
// round-to-nearest intrinsic (no fused multiply-add), so the FP64 values are
// reproducible bit for bit by any IEEE implementation of the same recipe.
//
// Layout produced (all device memory owned by the handle):
//   row_cptr[m+1] int64, row_cells[U] int32   cell-level CSR (runs of nz entries)
//   cell_rptr[H+1] int64, cell_rows[U] int32  cell-level transpose, rows ascending
//   vals[d].csr[nnz], vals[d].csc[nnz]         values in CSR / CSC order per dtype
//   row_ptr, col, col_ptr, row_idx             element indices (PDST_FMT_ELEMENT)
// with nnz = nz * U and the CSC of column j = h*nz + k starting at
// nz*cell_rptr[h] + k*cnt[h].
#include <atomic>
#include <cmath>

#include "common.cuh"

namespace pdst {

namespace {

struct Ray {
    double x0, y0, x1, y1, x2, y2;
};

__device__ __forceinline__ void bezier_pt(const Ray &c, double tau, double &x, double &y) {
    double a = __dsub_rn(1.0, tau);
    double b0 = __dmul_rn(a, a);
    double b1 = __dmul_rn(__dmul_rn(2.0, tau), a);
    double b2 = __dmul_rn(tau, tau);
    x = __dadd_rn(__dadd_rn(__dmul_rn(b0, c.x0), __dmul_rn(b1, c.x1)), __dmul_rn(b2, c.x2));
    y = __dadd_rn(__dadd_rn(__dmul_rn(b0, c.y0), __dmul_rn(b1, c.y1)), __dmul_rn(b2, c.y2));
}

__device__ __forceinline__ double hyp(double ex, double ey) {
    return __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
}

__device__ __forceinline__ int64_t chord_count_dev(const Ray &c, double dx) {
    double lp = __dadd_rn(hyp(__dsub_rn(c.x1, c.x0), __dsub_rn(c.y1, c.y0)),
                          hyp(__dsub_rn(c.x2, c.x1), __dsub_rn(c.y2, c.y1)));
    if (!(lp > 0.0)) return 0;
    double nf = ceil(__ddiv_rn(__dmul_rn(4.0, lp), dx));
    if (nf < 1.0) nf = 1.0;
    return (int64_t)nf;
}

__device__ __forceinline__ int cell_of(double coord, double dx, int ncell) {
    double f = floor(__ddiv_rn(coord, dx));
    if (f < 0.0) f = 0.0;
    if (f > (double)(ncell - 1)) f = (double)(ncell - 1);
    return (int)f;
}

// Lower node and fraction of the bilinear interpolation along one axis:
// nodes at (i + 1/2) dx; i0 = floor(coord/dx - 1/2) clamped to [0, n-2],
// t = coord/dx - 1/2 - i0 clamped to [0, 1].
__device__ __forceinline__ int bilin_axis(double coord, double dx, int n, double &t) {
    const double f = __dsub_rn(__ddiv_rn(coord, dx), 0.5);
    double i0 = floor(f);
    if (i0 < 0.0) i0 = 0.0;
    if (i0 > (double)(n - 2)) i0 = (double)(n - 2);
    double tt = __dsub_rn(f, i0);
    if (tt < 0.0) tt = 0.0;
    if (tt > 1.0) tt = 1.0;
    t = tt;
    return (int)i0;
}

// One warp walks one ray.  The 32 lanes evaluate 32 consecutive chords at a
// time; the per-cell sums are then advanced in chord order (every lane holds
// the same running sum, so the result does not depend on the lane).  With
// interp 1 a chord gives len * w to the four nodes around its midpoint
// (bilinear weights w, Eq. 1's coefficients), in the order (i0, j0),
// (i0+1, j0), (i0, j0+1), (i0+1, j0+1).  The distinct cells (nodes) live in a
// per-warp shared-memory list of capacity `cap`.  Returns the number of
// distinct cells (> cap means the list overflowed).
__device__ int walk_ray_warp(const Ray &c, int nx, int ny, double dx, int interp, int cap,
                             int *lc, double *la) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int64_t N = chord_count_dev(c, dx);
    int u = 0, cur_slot = -1, cur_cell = -1;
    double cur = 0.0;
    double cx, cy;
    bezier_pt(c, 0.0, cx, cy);
    for (int64_t base = 0; base < N; base += 32) {
        int64_t s = base + lane + 1;
        bool valid = s <= N;
        double qx = 0.0, qy = 0.0;
        if (valid) bezier_pt(c, __ddiv_rn((double)s, (double)N), qx, qy);
        double px = __shfl_up_sync(full, qx, 1), py = __shfl_up_sync(full, qy, 1);
        if (lane == 0) {
            px = cx;
            py = cy;
        }
        const int np = interp ? 4 : 1;   // contributions per chord
        double len[4] = {0.0, 0.0, 0.0, 0.0};
        int cell[4] = {0, 0, 0, 0};
        if (valid) {
            const double l = hyp(__dsub_rn(qx, px), __dsub_rn(qy, py));
            double mx = __dmul_rn(0.5, __dadd_rn(px, qx));
            double my = __dmul_rn(0.5, __dadd_rn(py, qy));
            if (!interp) {
                len[0] = l;
                cell[0] = cell_of(my, dx, ny) * nx + cell_of(mx, dx, nx);
            } else {
                double tx, ty;
                const int ix = bilin_axis(mx, dx, nx, tx), iy = bilin_axis(my, dx, ny, ty);
                const double a = __dsub_rn(1.0, tx), b = __dsub_rn(1.0, ty);
                cell[0] = iy * nx + ix;
                cell[1] = iy * nx + ix + 1;
                cell[2] = (iy + 1) * nx + ix;
                cell[3] = (iy + 1) * nx + ix + 1;
                len[0] = __dmul_rn(l, __dmul_rn(a, b));
                len[1] = __dmul_rn(l, __dmul_rn(tx, b));
                len[2] = __dmul_rn(l, __dmul_rn(a, ty));
                len[3] = __dmul_rn(l, __dmul_rn(tx, ty));
            }
        }
        cx = __shfl_sync(full, qx, 31);
        cy = __shfl_sync(full, qy, 31);
        int nvalid = (int)((N - base) < 32 ? (N - base) : 32);
        for (int jj = 0; jj < nvalid * np; ++jj) {
            const int j = jj / np, q = jj - j * np;
            const int mine = q == 0 ? cell[0] : q == 1 ? cell[1] : q == 2 ? cell[2] : cell[3];
            const double lmine = q == 0 ? len[0] : q == 1 ? len[1] : q == 2 ? len[2] : len[3];
            int cj = __shfl_sync(full, mine, j);
            double lj = __shfl_sync(full, lmine, j);
            if (cj != cur_cell) {
                if (lane == 0 && cur_slot >= 0 && cur_slot < cap) la[cur_slot] = cur;
                __syncwarp();
                int found = -1;
                int lim = u < cap ? u : cap;
                for (int q0 = 0; q0 < lim; q0 += 32) {
                    int q = q0 + lane;
                    unsigned b = __ballot_sync(full, q < lim && lc[q] == cj);
                    if (b) {
                        found = q0 + __ffs(b) - 1;
                        break;
                    }
                }
                if (found >= 0) {
                    cur = la[found];
                    cur_slot = found;
                } else {
                    if (lane == 0 && u < cap) lc[u] = cj;
                    cur_slot = u;
                    ++u;
                    cur = 0.0;
                }
                cur_cell = cj;
                __syncwarp();
            }
            cur = __dadd_rn(cur, lj);
        }
    }
    if (lane == 0 && cur_slot >= 0 && cur_slot < cap) la[cur_slot] = cur;
    __syncwarp();
    return u;
}

__device__ __forceinline__ Ray load_ray(const double *ctrl, int64_t r) {
    const double *p = ctrl + 6 * r;
    return Ray{p[0], p[1], p[2], p[3], p[4], p[5]};
}

// Pass 1: distinct cells per row.
__global__ void k_count_cells(int64_t m, const double *__restrict__ ctrl, int nx, int ny,
                              double dx, int interp, int cap, int32_t *__restrict__ cnt,
                              int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
    double *la = reinterpret_cast<double *>(smem) + (size_t)warp * cap;
    int *lc = reinterpret_cast<int *>(smem + (size_t)wpb * cap * sizeof(double)) + (size_t)warp * cap;
    for (int64_t r = (int64_t)blockIdx.x * wpb + warp; r < m; r += (int64_t)gridDim.x * wpb) {
        int u = walk_ray_warp(load_ray(ctrl, r), nx, ny, dx, interp, cap, lc, la);
        if ((threadIdx.x & 31) == 0) {
            cnt[r] = u;
            if (u > cap) atomicExch(err, 1);
        }
    }
}

// Pass 2: walk again, sort the row's cells ascending (rank of unique keys)
// and write cells, per-cell lengths and the owning row of every run.
__global__ void k_fill_cells(int64_t m, const double *__restrict__ ctrl, int nx, int ny,
                             double dx, int interp, int cap, const int64_t *__restrict__ cptr,
                             int32_t *__restrict__ cells, double *__restrict__ lens,
                             int32_t *__restrict__ run_row, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *la = reinterpret_cast<double *>(smem) + (size_t)warp * cap;
    int *lc = reinterpret_cast<int *>(smem + (size_t)wpb * cap * sizeof(double)) + (size_t)warp * cap;
    for (int64_t r = (int64_t)blockIdx.x * wpb + warp; r < m; r += (int64_t)gridDim.x * wpb) {
        int u = walk_ray_warp(load_ray(ctrl, r), nx, ny, dx, interp, cap, lc, la);
        int64_t base = cptr[r];
        if (u > cap || (int64_t)u != cptr[r + 1] - base) {
            if (lane == 0) atomicExch(err, 2);
            continue;
        }
        for (int q = lane; q < u; q += 32) {
            int key = lc[q];
            int rank = 0;
            for (int j = 0; j < u; ++j) rank += lc[j] < key;
            cells[base + rank] = key;
            lens[base + rank] = la[q];
            run_row[base + rank] = (int32_t)r;
        }
        __syncwarp();
    }
}

// vals[nz*e + k] = l_e * K in FP64, plus narrower copies, with K = Kdz[t][k]
// (t the period of run e's row) or, given a per-cell table, Kc[h][t][k] (h
// the run's cell).
__global__ void k_expand_values(int64_t U, int nz, const double *__restrict__ lens,
                                const int32_t *__restrict__ run_row,
                                const int32_t *__restrict__ row_period,
                                const double *__restrict__ kdz,
                                const int32_t *__restrict__ run_cell,
                                const double *__restrict__ kdz_cells, int n_periods,
                                double *v64, float *v32, __nv_bfloat16 *vbf) {
    int64_t total = U * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i / nz;
        int k = (int)(i - e * nz);
        int t = row_period[run_row[e]];
        const double kv = kdz_cells
                              ? kdz_cells[((int64_t)run_cell[e] * n_periods + t) * nz + k]
                              : kdz[(int64_t)t * nz + k];
        double v = __dmul_rn(lens[e], kv);
        if (v64) v64[i] = v;
        if (v32) v32[i] = __double2float_rn(v);
        if (vbf) vbf[i] = __double2bfloat16(v);
    }
}

__global__ void k_cell_count(int64_t U, const int32_t *__restrict__ cells, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < U;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[cells[e]], 1);
}

// Histogram of cells per chunk of `ch` consecutive rows.
__global__ void k_chunk_count(int64_t U, int ch, int H, const int32_t *__restrict__ cells,
                              const int32_t *__restrict__ run_row, int32_t *chunk_cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < U;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&chunk_cnt[(int64_t)(run_row[e] / ch) * H + cells[e]], 1);
}

// Turn per-chunk counts into absolute start positions, chunk by chunk.
__global__ void k_chunk_scan(int64_t nchunk, int H, const int64_t *__restrict__ cell_rptr,
                             const int32_t *__restrict__ chunk_cnt, int64_t *chunk_base) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    int64_t run = cell_rptr[h];
    for (int64_t c = 0; c < nchunk; ++c) {
        int64_t idx = c * H + h;
        int32_t t = chunk_cnt[idx];
        chunk_base[idx] = run;
        run += t;
    }
}

// One block per chunk places its rows in order: rows of a chunk are visited
// one after another, the runs of one row in parallel (distinct cells).
__global__ void k_chunk_place(int64_t m, int ch, int H, const int64_t *__restrict__ row_cptr,
                              const int32_t *__restrict__ cells, int64_t *chunk_base,
                              int32_t *__restrict__ cell_rows, int64_t *__restrict__ run_pos) {
    int64_t c = blockIdx.x;
    int64_t r0 = c * ch, r1 = r0 + ch < m ? r0 + ch : m;
    int64_t *base = chunk_base + c * H;
    for (int64_t r = r0; r < r1; ++r) {
        for (int64_t e = row_cptr[r] + threadIdx.x; e < row_cptr[r + 1]; e += blockDim.x) {
            int h = cells[e];
            int64_t pos = base[h];
            base[h] = pos + 1;
            cell_rows[pos] = (int32_t)r;
            run_pos[e] = pos;
        }
        __syncthreads();
    }
}

// Blocked CSC copy: the nz values of run e (row r, cell h) go to the run's
// position in the cell's row list, depth fastest.
template <class T>
__global__ void k_bcsc_values(int64_t U, int nz, const int64_t *__restrict__ run_pos,
                              const T *__restrict__ csr, T *__restrict__ bcsc) {
    int64_t total = U * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i / nz;
        int k = (int)(i - e * nz);
        bcsc[run_pos[e] * nz + k] = csr[i];
    }
}

// Rows per adjoint work item.  A cell split over several items pays for its
// partial sums, a fence and a counter per item, which costs about as much as
// streaming a few hundred rows, so items are made as long as the load balance
// allows: the largest power of two in [ADJ_CHUNK_MIN, ADJ_CHUNK_MAX] that still
// gives at least ITEMS_PER_WARP items to each resident warp of the adjoint
// sweep (32 per SM; the warps draw items dynamically, so a few items each are
// enough to balance them).  Measured on B300 (FP32 sweep): 256-512 rows best
// on the 64 x 64 x 16 system, 1024 on the 100 x 100 x 20 one; this rule picks
// 256 and 1024.
constexpr int ITEMS_PER_WARP = 8;

static int choose_adj_chunk(const std::vector<int32_t> &cnt, int sms) {
    const int64_t target = (int64_t)sms * 32 * ITEMS_PER_WARP;
    int chunk = ADJ_CHUNK_MIN;
    while (chunk < ADJ_CHUNK_MAX) {
        const int64_t next = 2 * (int64_t)chunk;
        int64_t items = 0;
        for (int32_t c : cnt) items += std::max<int64_t>(1, (c + next - 1) / next);
        if (items < target) break;
        chunk *= 2;
    }
    return chunk;
}

// Double-float copy: each FP64 value as its nearest float plus the rest.
__global__ void k_split_values(int64_t nnz, const double *__restrict__ v, dfl *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dfl(v[i]);
}

template <class T>
__global__ void k_csc_values(int64_t U, int nz, const int32_t *__restrict__ cells,
                             const int64_t *__restrict__ run_pos,
                             const int64_t *__restrict__ cell_rptr,
                             const int32_t *__restrict__ cell_cnt, const T *__restrict__ csr,
                             T *__restrict__ csc) {
    int64_t total = U * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = i / nz;
        int k = (int)(i - e * nz);
        int h = cells[e];
        int64_t start = cell_rptr[h];
        csc[(int64_t)nz * start + (int64_t)k * cell_cnt[h] + (run_pos[e] - start)] = csr[i];
    }
}

__global__ void k_elem_csr(int64_t m, int64_t U, int nz, const int64_t *__restrict__ row_cptr,
                           const int32_t *__restrict__ cells, int64_t *row_ptr, int32_t *col) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = tid; r <= m; r += stride) row_ptr[r] = (int64_t)nz * row_cptr[r];
    for (int64_t i = tid; i < U * nz; i += stride) {
        int64_t e = i / nz;
        col[i] = cells[e] * nz + (int)(i - e * nz);
    }
}

__global__ void k_elem_csc(int64_t U, int H, int nz, const int32_t *__restrict__ cells,
                           const int32_t *__restrict__ run_row,
                           const int64_t *__restrict__ run_pos,
                           const int64_t *__restrict__ cell_rptr,
                           const int32_t *__restrict__ cell_cnt, int64_t *col_ptr,
                           int32_t *row_idx) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t n = (int64_t)H * nz;
    for (int64_t j = tid; j <= n; j += stride) {
        if (j == n) {
            col_ptr[j] = (int64_t)nz * cell_rptr[H];
        } else {
            int64_t h = j / nz;
            int k = (int)(j - h * nz);
            col_ptr[j] = (int64_t)nz * cell_rptr[h] + (int64_t)k * cell_cnt[h];
        }
    }
    for (int64_t i = tid; i < U * nz; i += stride) {
        int64_t e = i / nz;
        int k = (int)(i - e * nz);
        int h = cells[e];
        int64_t start = cell_rptr[h];
        row_idx[(int64_t)nz * start + (int64_t)k * cell_cnt[h] + (run_pos[e] - start)] = run_row[e];
    }
}

// ------------------------------------------------------------- prefix sum

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

// out[i+1] = in[0] + ... + in[i] within each tile; bsum[b] = tile total.
template <class Tin>
__global__ void k_scan_tiles(const Tin *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                             int64_t *__restrict__ bsum) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    int64_t v[SCAN_PER];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        v[i] = base + i < n ? (int64_t)in[base + i] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < SCAN_THREADS / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t run = incl - s + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        run += v[i];
        if (base + i < n) out[base + i + 1] = run;
    }
    if (threadIdx.x == SCAN_THREADS - 1) bsum[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t n, int64_t *__restrict__ out, const int64_t *__restrict__ bex) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i + 1] += bex[i / SCAN_TILE];
}

}  // namespace

// Exclusive prefix sum: out[0] = 0, out[i+1] = sum of in[0..i].
template <class Tin>
static pdst_status scan_exclusive(const Tin *in, int64_t n, int64_t *out, cudaStream_t s) {
    PDST_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    if (n == 0) return PDST_OK;
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf bsum, bex;
    PDST_TRY(bsum.alloc(sizeof(int64_t) * nb));
    PDST_TRY(bex.alloc(sizeof(int64_t) * (nb + 1)));
    k_scan_tiles<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, out, bsum.as<int64_t>());
    PDST_CUDA(cudaGetLastError());
    if (nb > 1) {
        PDST_TRY(scan_exclusive<int64_t>(bsum.as<int64_t>(), nb, bex.as<int64_t>(), s));
        k_scan_add<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(
            n, out, bex.as<int64_t>());
        PDST_CUDA(cudaGetLastError());
    }
    PDST_CUDA(cudaStreamSynchronize(s));   // bsum/bex are released on return
    return PDST_OK;
}

// Host mirror of the chord count, used only to size the per-warp cell list.
static int64_t host_chord_count(const double *c, double dx) {
    double ax = c[2] - c[0], ay = c[3] - c[1], bx = c[4] - c[2], by = c[5] - c[3];
    double lp = std::sqrt(ax * ax + ay * ay) + std::sqrt(bx * bx + by * by);
    if (!(lp > 0.0)) return 0;
    double nf = std::ceil(4.0 * lp / dx);
    return nf < 1.0 ? 1 : (int64_t)nf;
}

static unsigned grid_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Blocked-CSC copies of every kept value set (and element-CSC copies with the
// element layout) from its CSR-order values; rp = each run's position in the
// blocked CSC layout.  Asynchronous.
static pdst_status transposed_value_copies(pdst_handle *h, const int64_t *rp, cudaStream_t s) {
    const int64_t U = h->U, nnz = h->nnz;
    const int nz = h->nz;
    if (!nnz) return PDST_OK;
    unsigned g = grid_for(nnz, 256, h->device);
    const bool elem = (h->formats & (1u << PDST_FMT_ELEMENT)) != 0;
    if (h->vals[0].present) {
        k_bcsc_values<double><<<g, 256, 0, s>>>(U, nz, rp, h->vals[0].csr.as<double>(),
                                               h->vals[0].bcsc.as<double>());
        if (elem)
            k_csc_values<double><<<g, 256, 0, s>>>(U, nz, h->row_cells.as<int32_t>(), rp,
                                                  h->cell_rptr.as<int64_t>(),
                                                  h->cell_cnt.as<int32_t>(),
                                                  h->vals[0].csr.as<double>(),
                                                  h->vals[0].csc.as<double>());
    }
    if (h->vals[1].present) {
        k_bcsc_values<float><<<g, 256, 0, s>>>(U, nz, rp, h->vals[1].csr.as<float>(),
                                              h->vals[1].bcsc.as<float>());
        if (elem)
            k_csc_values<float><<<g, 256, 0, s>>>(U, nz, h->row_cells.as<int32_t>(), rp,
                                                 h->cell_rptr.as<int64_t>(),
                                                 h->cell_cnt.as<int32_t>(),
                                                 h->vals[1].csr.as<float>(),
                                                 h->vals[1].csc.as<float>());
    }
    if (h->vals[PDST_DF64].present)
        k_bcsc_values<dfl><<<g, 256, 0, s>>>(U, nz, rp, h->vals[PDST_DF64].csr.as<dfl>(),
                                            h->vals[PDST_DF64].bcsc.as<dfl>());
    if (h->vals[2].present) {
        k_bcsc_values<__nv_bfloat16><<<g, 256, 0, s>>>(U, nz, rp,
                                                      h->vals[2].csr.as<__nv_bfloat16>(),
                                                      h->vals[2].bcsc.as<__nv_bfloat16>());
        if (elem)
            k_csc_values<__nv_bfloat16><<<g, 256, 0, s>>>(
                U, nz, h->row_cells.as<int32_t>(), rp, h->cell_rptr.as<int64_t>(),
                h->cell_cnt.as<int32_t>(), h->vals[2].csr.as<__nv_bfloat16>(),
                h->vals[2].csc.as<__nv_bfloat16>());
    }
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}

static pdst_status build_impl(pdst_handle *h, const double *ctrl_host, const int32_t *per_host,
                              const double *kdz_host, const double *kdz_cells_host,
                              uint32_t dtypes, bool keep_lengths, cudaStream_t s) {
    const int nx = h->grid.nx, ny = h->grid.ny, nz = h->nz, H = h->H;
    const double dx = h->grid.dx_km;
    const int64_t m = h->m;

    // capacity of the per-warp distinct-cell list (distinct cells <= chords)
    int64_t maxN = 0;
    for (int64_t r = 0; r < m; ++r) maxN = std::max(maxN, host_chord_count(ctrl_host + 6 * r, dx));
    // distinct cells a ray can touch: one per chord (four nodes per chord
    // with bilinear coefficients)
    int64_t cap64 = std::min<int64_t>((h->interp ? 4 : 1) * maxN + 64, H);
    cap64 = (cap64 + 31) / 32 * 32;
    if (cap64 < 32) cap64 = 32;
    const int64_t smem_budget = 200 * 1024;
    if (cap64 * 12 > smem_budget) {
        set_error("a ray may cross up to %lld distinct cells; the per-warp list holds %lld",
                  (long long)cap64, (long long)(smem_budget / 12));
        return PDST_ERR_LIMIT;
    }
    const int cap = (int)cap64;
    int wpb = (int)std::min<int64_t>(8, smem_budget / (cap64 * 12));
    size_t smem = (size_t)wpb * cap * 12;
    PDST_CUDA(cudaFuncSetAttribute(k_count_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    PDST_CUDA(cudaFuncSetAttribute(k_fill_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));

    DevBuf d_ctrl, d_kdz, d_cnt, d_err, d_lens, d_runrow, d_runpos;
    PDST_TRY(d_ctrl.alloc(sizeof(double) * 6 * std::max<int64_t>(m, 1)));
    PDST_TRY(d_kdz.alloc(sizeof(double) * (size_t)h->n_periods * nz));
    DevBuf d_kcells;
    if (kdz_cells_host) {
        const size_t kb = sizeof(double) * (size_t)H * h->n_periods * nz;
        PDST_TRY(d_kcells.alloc(kb));
        PDST_CUDA(cudaMemcpyAsync(d_kcells.p, kdz_cells_host, kb, cudaMemcpyHostToDevice, s));
    }
    PDST_TRY(h->row_period.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1)));
    PDST_TRY(d_cnt.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1)));
    PDST_TRY(d_err.alloc(sizeof(int)));
    if (m) {
        PDST_CUDA(cudaMemcpyAsync(d_ctrl.p, ctrl_host, sizeof(double) * 6 * m,
                                  cudaMemcpyHostToDevice, s));
        PDST_CUDA(cudaMemcpyAsync(h->row_period.p, per_host, sizeof(int32_t) * m,
                                  cudaMemcpyHostToDevice, s));
    }
    PDST_CUDA(cudaMemcpyAsync(d_kdz.p, kdz_host, sizeof(double) * h->n_periods * nz,
                              cudaMemcpyHostToDevice, s));
    PDST_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), s));

    int sms = num_sms(h->device);
    unsigned wgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + wpb - 1) / wpb,
                                                                      (int64_t)sms * 8));
    if (m) {
        k_count_cells<<<wgrid, wpb * 32, smem, s>>>(m, d_ctrl.as<double>(), nx, ny, dx,
                                                   h->interp, cap,
                                                   d_cnt.as<int32_t>(), d_err.as<int>());
        PDST_CUDA(cudaGetLastError());
    }
    PDST_TRY(h->row_cptr.alloc(sizeof(int64_t) * (m + 1)));
    PDST_TRY(scan_exclusive<int32_t>(d_cnt.as<int32_t>(), m, h->row_cptr.as<int64_t>(), s));
    int herr = 0;
    PDST_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaMemcpyAsync(&h->U, h->row_cptr.as<int64_t>() + m, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("a ray crossed more distinct cells than the per-warp list holds (%d)", cap);
        return PDST_ERR_LIMIT;
    }
    const int64_t U = h->U;
    h->nnz = U * nz;
    d_cnt.release();

    PDST_TRY(h->row_cells.alloc(sizeof(int32_t) * std::max<int64_t>(U, 1)));
    PDST_TRY(d_lens.alloc(sizeof(double) * std::max<int64_t>(U, 1)));
    PDST_TRY(d_runrow.alloc(sizeof(int32_t) * std::max<int64_t>(U, 1)));
    if (m) {
        k_fill_cells<<<wgrid, wpb * 32, smem, s>>>(m, d_ctrl.as<double>(), nx, ny, dx,
                                                  h->interp, cap,
                                                  h->row_cptr.as<int64_t>(),
                                                  h->row_cells.as<int32_t>(), d_lens.as<double>(),
                                                  d_runrow.as<int32_t>(), d_err.as<int>());
        PDST_CUDA(cudaGetLastError());
    }

    // values in CSR order
    const int64_t nnz = h->nnz;
    for (int d = 0; d < 4; ++d) {
        if (!(dtypes & (1u << d))) continue;
        size_t es = d == PDST_F64 ? 8 : d == PDST_F32 ? 4 : d == PDST_BF16 ? 2 : sizeof(dfl);
        PDST_TRY(h->vals[d].csr.alloc(es * std::max<int64_t>(nnz, 1)));
        PDST_TRY(h->vals[d].bcsc.alloc(es * std::max<int64_t>(nnz, 1)));
        if ((h->formats & (1u << PDST_FMT_ELEMENT)) && d != PDST_DF64)
            PDST_TRY(h->vals[d].csc.alloc(es * std::max<int64_t>(nnz, 1)));
        h->vals[d].present = true;
    }
    // the float pairs are split from the FP64 values (kept or temporary)
    DevBuf v64_tmp;
    double *v64 = h->vals[PDST_F64].present ? h->vals[PDST_F64].csr.as<double>() : nullptr;
    if (h->vals[PDST_DF64].present && !v64 && nnz) {
        PDST_TRY(v64_tmp.alloc(sizeof(double) * nnz));
        v64 = v64_tmp.as<double>();
    }
    if (nnz) {
        k_expand_values<<<grid_for(nnz, 256, h->device), 256, 0, s>>>(
            U, nz, d_lens.as<double>(), d_runrow.as<int32_t>(), h->row_period.as<int32_t>(),
            d_kdz.as<double>(), h->row_cells.as<int32_t>(),
            kdz_cells_host ? d_kcells.as<double>() : nullptr, h->n_periods, v64,
            h->vals[1].present ? h->vals[1].csr.as<float>() : nullptr,
            h->vals[2].present ? h->vals[2].csr.as<__nv_bfloat16>() : nullptr);
        PDST_CUDA(cudaGetLastError());
        if (h->vals[PDST_DF64].present) {
            k_split_values<<<grid_for(nnz, 256, h->device), 256, 0, s>>>(
                nnz, v64, h->vals[PDST_DF64].csr.as<dfl>());
            PDST_CUDA(cudaGetLastError());
        }
        PDST_CUDA(cudaStreamSynchronize(s));   // the temporary is released on scope exit
    }

    // cell-level transpose
    PDST_TRY(h->cell_cnt.alloc(sizeof(int32_t) * H));
    PDST_TRY(h->cell_rptr.alloc(sizeof(int64_t) * (H + 1)));
    PDST_TRY(h->cell_rows.alloc(sizeof(int32_t) * std::max<int64_t>(U, 1)));
    PDST_TRY(d_runpos.alloc(sizeof(int64_t) * std::max<int64_t>(U, 1)));
    PDST_CUDA(cudaMemsetAsync(h->cell_cnt.p, 0, sizeof(int32_t) * H, s));
    if (U) {
        k_cell_count<<<grid_for(U, 256, h->device), 256, 0, s>>>(U, h->row_cells.as<int32_t>(),
                                                                 h->cell_cnt.as<int32_t>());
        PDST_CUDA(cudaGetLastError());
    }
    PDST_TRY(scan_exclusive<int32_t>(h->cell_cnt.as<int32_t>(), H, h->cell_rptr.as<int64_t>(), s));
    if (U) {
        const int ch = 256;
        int64_t nchunk = (m + ch - 1) / ch;
        DevBuf ccnt, cbase;
        PDST_TRY(ccnt.alloc(sizeof(int32_t) * nchunk * H));
        PDST_TRY(cbase.alloc(sizeof(int64_t) * nchunk * H));
        PDST_CUDA(cudaMemsetAsync(ccnt.p, 0, sizeof(int32_t) * nchunk * H, s));
        k_chunk_count<<<grid_for(U, 256, h->device), 256, 0, s>>>(
            U, ch, H, h->row_cells.as<int32_t>(), d_runrow.as<int32_t>(), ccnt.as<int32_t>());
        PDST_CUDA(cudaGetLastError());
        k_chunk_scan<<<(H + 127) / 128, 128, 0, s>>>(nchunk, H, h->cell_rptr.as<int64_t>(),
                                                      ccnt.as<int32_t>(), cbase.as<int64_t>());
        PDST_CUDA(cudaGetLastError());
        k_chunk_place<<<(unsigned)nchunk, 128, 0, s>>>(m, ch, H, h->row_cptr.as<int64_t>(),
                                                       h->row_cells.as<int32_t>(),
                                                       cbase.as<int64_t>(),
                                                       h->cell_rows.as<int32_t>(),
                                                       d_runpos.as<int64_t>());
        PDST_CUDA(cudaGetLastError());
        PDST_TRY(transposed_value_copies(h, d_runpos.as<int64_t>(), s));
        PDST_CUDA(cudaGetLastError());
        PDST_CUDA(cudaStreamSynchronize(s));   // chunk tables are released on scope exit
    }

    if (h->formats & (1u << PDST_FMT_ELEMENT)) {
        PDST_TRY(h->row_ptr.alloc(sizeof(int64_t) * (m + 1)));
        PDST_TRY(h->col.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
        PDST_TRY(h->col_ptr.alloc(sizeof(int64_t) * ((int64_t)h->n + 1)));
        PDST_TRY(h->row_idx.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
        k_elem_csr<<<grid_for(std::max<int64_t>(nnz, m + 1), 256, h->device), 256, 0, s>>>(
            m, U, nz, h->row_cptr.as<int64_t>(), h->row_cells.as<int32_t>(),
            h->row_ptr.as<int64_t>(), h->col.as<int32_t>());
        PDST_CUDA(cudaGetLastError());
        k_elem_csc<<<grid_for(std::max<int64_t>(nnz, (int64_t)h->n + 1), 256, h->device), 256, 0,
                     s>>>(U, H, nz, h->row_cells.as<int32_t>(), d_runrow.as<int32_t>(),
                          d_runpos.as<int64_t>(), h->cell_rptr.as<int64_t>(),
                          h->cell_cnt.as<int32_t>(), h->col_ptr.as<int64_t>(),
                          h->row_idx.as<int32_t>());
        PDST_CUDA(cudaGetLastError());
    }
    PDST_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("G assembly: per-row cell list inconsistent between passes (code %d)", herr);
        return PDST_ERR_CUDA;
    }
    // work order of the transpose products: longest cells first, so that the
    // last work items of a launch are the short ones
    {
        std::vector<int32_t> cnt(H), order(H);
        PDST_CUDA(cudaMemcpy(cnt.data(), h->cell_cnt.p, sizeof(int32_t) * H,
                             cudaMemcpyDeviceToHost));
        for (int i = 0; i < H; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return cnt[a] > cnt[b]; });
        PDST_TRY(h->cell_order.alloc(sizeof(int32_t) * H));
        PDST_CUDA(cudaMemcpy(h->cell_order.p, order.data(), sizeof(int32_t) * H,
                             cudaMemcpyHostToDevice));
        // adjoint work items: every cell (empty ones too) in chunks of
        // adj_chunk rows, cells longest first, chunks of a cell consecutive
        h->adj_chunk = choose_adj_chunk(cnt, num_sms(h->device));
        std::vector<int32_t> items;
        for (int i = 0; i < H; ++i) {
            const int c = order[i];
            for (int q0 = 0; q0 < std::max(cnt[c], 1); q0 += h->adj_chunk) {
                items.push_back(c);
                items.push_back(q0);
            }
        }
        h->n_adj = (int64_t)items.size() / 2;
        PDST_TRY(h->adj_item.alloc(sizeof(int32_t) * items.size()));
        PDST_CUDA(cudaMemcpy(h->adj_item.p, items.data(), sizeof(int32_t) * items.size(),
                             cudaMemcpyHostToDevice));
    }
    if (keep_lengths) {
        h->run_len.take(d_lens);
        h->run_row.take(d_runrow);
        h->run_pos.take(d_runpos);
        h->has_lengths = true;
    }
    return PDST_OK;
}

}  // namespace pdst

using namespace pdst;

extern "C" pdst_status pdst_build_G(const pdst_grid *grid, int64_t n_paths,
                                    const double *ctrl_host, const int32_t *path_period_host,
                                    int32_t n_periods, const double *kdz_host,
                                    const pdst_build_opts *opts, void *stream,
                                    pdst_handle_t *out) {
    PDST_CHECK_ARG(out != nullptr, "pdst_build_G: out is NULL");
    *out = nullptr;
    PDST_CHECK_ARG(grid != nullptr, "pdst_build_G: grid is NULL");
    PDST_CHECK_ARG(grid->nx > 0 && grid->ny > 0 && grid->nz > 0,
                   "pdst_build_G: grid dimensions must be positive");
    PDST_CHECK_ARG(std::isfinite(grid->dx_km) && grid->dx_km > 0.0,
                   "pdst_build_G: dx_km must be positive and finite");
    PDST_CHECK_ARG(n_paths >= 0 && n_paths < INT32_MAX, "pdst_build_G: n_paths out of range");
    PDST_CHECK_ARG(n_periods > 0, "pdst_build_G: n_periods must be positive");
    PDST_CHECK_ARG(kdz_host != nullptr, "pdst_build_G: kdz is NULL");
    PDST_CHECK_ARG(n_paths == 0 || (ctrl_host && path_period_host),
                   "pdst_build_G: ctrl / path_period is NULL");
    int64_t H = (int64_t)grid->nx * grid->ny, n = H * grid->nz;
    PDST_CHECK_ARG(n < INT32_MAX, "pdst_build_G: nx*ny*nz must fit in int32");
    for (int64_t i = 0; i < 6 * n_paths; ++i)
        PDST_CHECK_ARG(std::isfinite(ctrl_host[i]), "pdst_build_G: non-finite ray coordinate %lld",
                       (long long)i);
    for (int64_t r = 0; r < n_paths; ++r)
        PDST_CHECK_ARG(path_period_host[r] >= 0 && path_period_host[r] < n_periods,
                       "pdst_build_G: period index of path %lld out of range", (long long)r);
    for (int64_t i = 0; i < (int64_t)n_periods * grid->nz; ++i)
        PDST_CHECK_ARG(std::isfinite(kdz_host[i]), "pdst_build_G: non-finite kdz entry");
    const double *kdz_cells = opts ? opts->kdz_cells : nullptr;
    if (kdz_cells)
        for (int64_t i = 0; i < H * n_periods * grid->nz; ++i)
            PDST_CHECK_ARG(std::isfinite(kdz_cells[i]), "pdst_build_G: non-finite kdz_cells entry");
    uint32_t dtypes = opts && opts->value_dtypes ? opts->value_dtypes
                                                 : (1u << PDST_F64) | (1u << PDST_F32);
    uint32_t formats = opts && opts->formats ? opts->formats
                                             : (1u << PDST_FMT_ELEMENT) | (1u << PDST_FMT_BLOCKED);
    PDST_CHECK_ARG((dtypes & ~15u) == 0, "pdst_build_G: unknown value dtype bits");
    PDST_CHECK_ARG((formats & ~3u) == 0, "pdst_build_G: unknown format bits");
    const int interp = opts ? opts->interp : 0;
    PDST_CHECK_ARG(interp == 0 || (interp == 1 && grid->nx >= 2 && grid->ny >= 2),
                   "pdst_build_G: interp must be 0, or 1 on a grid of at least 2 x 2 nodes");

    static std::atomic<uint64_t> next_uid{1};
    pdst_handle *h = new pdst_handle();
    h->uid = next_uid.fetch_add(1);
    cudaGetDevice(&h->device);
    h->grid = *grid;
    h->m = n_paths;
    h->n = (int32_t)n;
    h->H = (int32_t)H;
    h->nz = grid->nz;
    h->n_periods = n_periods;
    h->formats = formats;
    h->interp = interp;
    pdst_status st = build_impl(h, ctrl_host, path_period_host, kdz_host, kdz_cells, dtypes,
                                opts && opts->keep_lengths, (cudaStream_t)stream);
    if (st != PDST_OK) {
        delete h;
        return st;
    }
    *out = h;
    return PDST_OK;
}

// ------------------------------------------------ depth kernels from a model
//
// The synthetic kernel module of the outer loop (the paragraph after Eq. 6:
// G is rebuilt from the updated model): under cell h the kernel depth follows
// the column's mean relative velocity s_h = (1/nz) sum_k (1 + m[h*nz + k]),
// z0 = z0_factor * T * s_h^a, K[h][t][k] = (z_k / z0) exp(1 - z_k / z0) dz.
// One rounding per written operation (this file has no FMA contraction).

namespace pdst {

__global__ void k_kernels_from_model(int32_t H, int nz, int T, const double *__restrict__ periods,
                                     double z0f, double kp, double dz,
                                     const double *__restrict__ mv, double *__restrict__ K) {
    const int64_t total = (int64_t)H * T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = i / T;
        const int t = (int)(i - h * T);
        const double *col = mv + h * nz;
        double s = 0.0;
        for (int k = 0; k < nz; ++k) s = s + (1.0 + col[k]);   // depth order
        s = s / (double)nz;
        if (kp != 1.0) s = pow(s, kp);
        const double z0 = (z0f * periods[t]) * s;
        double *out = K + i * nz;
        for (int k = 0; k < nz; ++k) {
            const double z = ((double)k + 0.5) * dz;
            const double q = z / z0;
            out[k] = (q * exp(1.0 - q)) * dz;
        }
    }
}

}  // namespace pdst

extern "C" pdst_status pdst_depth_kernels_from_model(pdst_handle_t h, const double *periods_host,
                                                     double z0_factor, double kernel_power,
                                                     const double *m_dev, double *kdz_cells_dev,
                                                     void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_depth_kernels_from_model: handle is NULL");
    PDST_CHECK_ARG(periods_host && m_dev && kdz_cells_dev,
                   "pdst_depth_kernels_from_model: NULL pointer argument");
    PDST_CHECK_ARG(std::isfinite(z0_factor) && z0_factor > 0.0,
                   "pdst_depth_kernels_from_model: z0_factor must be positive and finite");
    PDST_CHECK_ARG(std::isfinite(kernel_power),
                   "pdst_depth_kernels_from_model: kernel_power must be finite");
    PDST_CHECK_ARG(std::isfinite(h->grid.dz_km) && h->grid.dz_km > 0.0,
                   "pdst_depth_kernels_from_model: the grid's dz_km must be positive");
    for (int t = 0; t < h->n_periods; ++t)
        PDST_CHECK_ARG(std::isfinite(periods_host[t]) && periods_host[t] > 0.0,
                       "pdst_depth_kernels_from_model: period %d must be positive and finite", t);
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf per;
    PDST_TRY(per.alloc(sizeof(double) * h->n_periods));
    PDST_CUDA(cudaMemcpyAsync(per.p, periods_host, sizeof(double) * h->n_periods,
                              cudaMemcpyHostToDevice, s));
    const int64_t work = (int64_t)h->H * h->n_periods;
    k_kernels_from_model<<<grid_for(work, 128, h->device), 128, 0, s>>>(
        h->H, h->nz, h->n_periods, per.as<double>(), z0_factor, kernel_power, h->grid.dz_km,
        m_dev, kdz_cells_dev);
    PDST_CUDA(cudaGetLastError());
    PDST_CUDA(cudaStreamSynchronize(s));   // the period copy is released on return
    return PDST_OK;
}

extern "C" pdst_status pdst_set_depth_kernels(pdst_handle_t h, const double *kdz_cells_dev,
                                              void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_set_depth_kernels: handle is NULL");
    PDST_CHECK_ARG(kdz_cells_dev != nullptr, "pdst_set_depth_kernels: kdz_cells is NULL");
    if (!h->has_lengths) {
        set_error("pdst_set_depth_kernels: the handle was built without keep_lengths");
        return PDST_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nnz = h->nnz;
    if (!nnz) return PDST_OK;
    DevBuf v64_tmp;
    double *v64 = h->vals[PDST_F64].present ? h->vals[PDST_F64].csr.as<double>() : nullptr;
    if (h->vals[PDST_DF64].present && !v64) {
        PDST_TRY(v64_tmp.alloc(sizeof(double) * nnz));
        v64 = v64_tmp.as<double>();
    }
    k_expand_values<<<grid_for(nnz, 256, h->device), 256, 0, s>>>(
        h->U, h->nz, h->run_len.as<double>(), h->run_row.as<int32_t>(),
        h->row_period.as<int32_t>(), nullptr, h->row_cells.as<int32_t>(), kdz_cells_dev,
        h->n_periods, v64, h->vals[1].present ? h->vals[1].csr.as<float>() : nullptr,
        h->vals[2].present ? h->vals[2].csr.as<__nv_bfloat16>() : nullptr);
    PDST_CUDA(cudaGetLastError());
    if (h->vals[PDST_DF64].present) {
        k_split_values<<<grid_for(nnz, 256, h->device), 256, 0, s>>>(
            nnz, v64, h->vals[PDST_DF64].csr.as<dfl>());
        PDST_CUDA(cudaGetLastError());
    }
    PDST_TRY(transposed_value_copies(h, h->run_pos.as<int64_t>(), s));
    PDST_CUDA(cudaStreamSynchronize(s));
    return PDST_OK;
}
