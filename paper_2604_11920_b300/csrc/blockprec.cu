// blockprec.cu -- per-cell depth-block right preconditioner for LSQR on
// A = [G; w L; lambda I] (pdst_lsqr with precond = 2).
//
// The nz columns of a horizontal cell h (depth fastest, Eq. 7) are coupled by
// every row of G that crosses the cell (Eq. 5: one path coefficient times a
// depth kernel over all nz depths) and by the depth terms of L.  Their block
// of the normal matrix, B_h = A_h^T A_h, is
//     sum over the cell's rows r of g_r g_r^T       (g_r: the row's nz values)
//   + w^2 (L^T L)_hh + lambda^2 I,
// where, for the 7-point graph Laplacian (L x)_j = sum_i (x_j - x_i) over the
// existing neighbours i of j (deg_j of them), (L^T L)_hh is pentadiagonal in
// depth: deg_a^2 + deg_a on the diagonal (the column's own entry squared plus
// one per neighbour), -(deg_a + deg_b) for vertically adjacent depths a, b
// (the grid graph has no triangles, so only the two diagonal entries meet),
// and +1 for depths two apart (their common neighbour in between).
//
// k_depth_gram forms B_h in FP64, one block per cell, from the cell's rows in
// the blocked CSC layout (contiguous: the cell's rows, nz values each);
// k_inv_chol factors each block (Cholesky, one warp per cell, lane = row) and
// inverts the factor column by column (lane c solves R p = e_c).  The LSQR
// kernels apply P_h^T and P_h in the adjoint's per-cell finish.
#include <cmath>

#include "common.cuh"

namespace pdst {
namespace {

constexpr int GT_THREADS = 256;
constexpr int GT_ROWS = 64;          // rows of one cell staged in shared memory at a time
constexpr int MAXNZ = 32;
constexpr int MAXPAIRS = MAXNZ * (MAXNZ + 1) / 2;
constexpr int PAIRS_PER_THREAD = (MAXPAIRS + GT_THREADS - 1) / GT_THREADS;   // 3

__device__ __forceinline__ int lap_degree(int ix, int iy, int k, int nx, int ny, int nz) {
    return (k > 0) + (k < nz - 1) + (ix > 0) + (ix < nx - 1) + (iy > 0) + (iy < ny - 1);
}

template <class VT>
__global__ void __launch_bounds__(GT_THREADS)
    k_depth_gram(const int64_t *__restrict__ cell_rptr, const int32_t *__restrict__ cell_cnt,
                 const VT *__restrict__ valB, int nx, int ny, int nz, double w, double lam,
                 double *B) {
    __shared__ double tile[GT_ROWS * MAXNZ];
    const int h = blockIdx.x;
    const int t = threadIdx.x;
    const int np = nz * (nz + 1) / 2;
    // this thread's (i, k) pairs of the upper triangle, enumerated row by row
    int pi[PAIRS_PER_THREAD], pk[PAIRS_PER_THREAD];
    double acc[PAIRS_PER_THREAD];
#pragma unroll
    for (int q = 0; q < PAIRS_PER_THREAD; ++q) {
        int p = t + GT_THREADS * q, i = 0;
        pi[q] = -1;
        pk[q] = 0;
        acc[q] = 0.0;
        if (p < np) {
            while (p >= nz - i) {
                p -= nz - i;
                ++i;
            }
            pi[q] = i;
            pk[q] = i + p;
        }
    }
    const int64_t c0 = cell_rptr[h];
    const int cnt = cell_cnt[h];
    const VT *v = valB + c0 * nz;
    for (int r0 = 0; r0 < cnt; r0 += GT_ROWS) {
        const int nr = cnt - r0 < GT_ROWS ? cnt - r0 : GT_ROWS;
        __syncthreads();
        for (int e = t; e < nr * nz; e += GT_THREADS)
            tile[e] = (double)widen(v[(int64_t)r0 * nz + e]);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PAIRS_PER_THREAD; ++q) {
            if (pi[q] < 0) continue;
            const double *a = tile + pi[q], *b = tile + pk[q];
            double s = acc[q];
            for (int r = 0; r < nr; ++r) s = fma(a[r * nz], b[r * nz], s);
            acc[q] = s;
        }
    }
    const int ix = h % nx, iy = h / nx;
    const double w2 = w * w;
    double *Bh = B + (int64_t)h * nz * nz;
#pragma unroll
    for (int q = 0; q < PAIRS_PER_THREAD; ++q) {
        if (pi[q] < 0) continue;
        const int i = pi[q], k = pk[q];
        const int di = lap_degree(ix, iy, i, nx, ny, nz);
        double lap = 0.0;
        if (k == i) lap = (double)(di * di + di);
        else if (k == i + 1) lap = -(double)(di + lap_degree(ix, iy, k, nx, ny, nz));
        else if (k == i + 2) lap = 1.0;
        double b = acc[q] + w2 * lap;
        if (k == i) b += lam * lam;
        Bh[i * nz + k] = b;
        Bh[k * nz + i] = b;
    }
}

constexpr int IC_WARPS = 2;

// P_h = R_h^{-1}, B_h = R_h^T R_h.  A block whose pivot is not positive (or not
// finite) gets P_h = I and its cell index in *bad (the smallest such index).
__global__ void __launch_bounds__(32 * IC_WARPS)
    k_inv_chol(int32_t H, int nz, const double *__restrict__ B, double *P64, float *P32,
               double *P64T, float *P32T, int *bad) {
    __shared__ double S[IC_WARPS][MAXNZ][MAXNZ + 1];
    __shared__ double Q[IC_WARPS][MAXNZ][MAXNZ + 1];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t h = (int64_t)blockIdx.x * IC_WARPS + wq;
    if (h >= H) return;
    const double *Bh = B + h * nz * nz;
    double(*R)[MAXNZ + 1] = S[wq];
    double(*X)[MAXNZ + 1] = Q[wq];
    for (int e = lane; e < nz * nz; e += 32) R[e / nz][e % nz] = Bh[e];
    __syncwarp();
    // right-looking Cholesky on the upper triangle: row c of R is finished at step c
    bool ok = true;
    for (int c = 0; c < nz; ++c) {
        const double d = R[c][c];
        ok = ok && (d > 0.0) && isfinite(d);
        const double rc = ok ? sqrt(d) : 1.0;
        __syncwarp();
        if (lane > c && lane < nz) R[c][lane] = R[c][lane] / rc;
        __syncwarp();
        if (lane > c && lane < nz) {
            const double ri = R[c][lane];
            for (int k = lane; k < nz; ++k) R[lane][k] -= ri * R[c][k];
        }
        if (lane == 0) R[c][c] = rc;
        __syncwarp();
    }
    // lane c: column c of R^{-1} by back substitution (R x = e_c, x_i = 0 for i > c)
    if (ok && lane < nz) {
        const int c = lane;
        for (int i = 0; i < nz; ++i) X[i][c] = 0.0;
        X[c][c] = 1.0 / R[c][c];
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k) s += R[i][k] * X[k][c];
            X[i][c] = -s / R[i][i];
        }
    }
    __syncwarp();
    if (!ok && lane == 0) atomicMin(bad, (int)h);
    double *P = P64 + h * nz * nz, *PT = P64T + h * nz * nz;
    float *Pf = P32 + h * nz * nz, *PfT = P32T + h * nz * nz;
    for (int e = lane; e < nz * nz; e += 32) {
        const int i = e / nz, k = e % nz;
        const double p = ok ? X[i][k] : (i == k ? 1.0 : 0.0);
        const double pt = ok ? X[k][i] : (i == k ? 1.0 : 0.0);
        P[e] = p;
        Pf[e] = (float)p;
        PT[e] = pt;
        PfT[e] = (float)pt;
    }
}

// Caller-supplied blocks: the upper triangle, the lower one zeroed, FP32 and
// transposed copies.
__global__ void k_copy_upper(int64_t total, int nz, const double *__restrict__ Pin, double *P64,
                             float *P32, double *P64T, float *P32T) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nn = (int64_t)nz * nz;
        const int64_t r = e % nn, base = e - r;
        const int i = (int)(r / nz), k = (int)(r % nz);
        const double p = k >= i ? Pin[e] : 0.0;
        const double pt = i >= k ? Pin[base + (int64_t)k * nz + i] : 0.0;
        P64[e] = p;
        P32[e] = (float)p;
        P64T[e] = pt;
        P32T[e] = (float)pt;
    }
}

pdst_status gram_blocks(pdst_handle *h, double w, double lam, double *B, cudaStream_t s) {
    if (h->H == 0) return PDST_OK;
    const unsigned g = (unsigned)h->H;
    const int64_t *rp = h->cell_rptr.as<int64_t>();
    const int32_t *cnt = h->cell_cnt.as<int32_t>();
    if (h->vals[PDST_F64].present)
        k_depth_gram<double><<<g, GT_THREADS, 0, s>>>(rp, cnt, h->vals[PDST_F64].bcsc.as<double>(),
                                                      h->grid.nx, h->grid.ny, h->nz, w, lam, B);
    else if (h->vals[PDST_F32].present)
        k_depth_gram<float><<<g, GT_THREADS, 0, s>>>(rp, cnt, h->vals[PDST_F32].bcsc.as<float>(),
                                                     h->grid.nx, h->grid.ny, h->nz, w, lam, B);
    else if (h->vals[PDST_BF16].present)
        k_depth_gram<__nv_bfloat16><<<g, GT_THREADS, 0, s>>>(
            rp, cnt, h->vals[PDST_BF16].bcsc.as<__nv_bfloat16>(), h->grid.nx, h->grid.ny, h->nz, w,
            lam, B);
    else {
        set_error("depth blocks: the handle keeps no FP64, FP32 or BF16 values");
        return PDST_ERR_STATE;
    }
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}

pdst_status check_common(pdst_handle *h, double w, double lam, const char *fn) {
    PDST_CHECK_ARG(h != nullptr, "%s: handle is NULL", fn);
    PDST_CHECK_ARG(std::isfinite(w) && std::isfinite(lam) && w >= 0 && lam >= 0,
                   "%s: w and lambda must be finite and >= 0", fn);
    if (h->nz > MAXNZ) {
        set_error("%s: the depth-block preconditioner needs nz <= %d (nz = %d)", fn, MAXNZ, h->nz);
        return PDST_ERR_LIMIT;
    }
    return PDST_OK;
}

}  // namespace
}  // namespace pdst

using namespace pdst;

extern "C" pdst_status pdst_depth_blocks(pdst_handle_t h, double w, double lambda, double *B_dev,
                                         void *stream) {
    PDST_TRY(check_common(h, w, lambda, "pdst_depth_blocks"));
    PDST_CHECK_ARG(B_dev != nullptr || h->H == 0, "pdst_depth_blocks: B_dev is NULL");
    return gram_blocks(h, w, lambda, B_dev, (cudaStream_t)stream);
}

extern "C" pdst_status pdst_set_block_precond(pdst_handle_t h, const double *P_dev, double w,
                                              double lambda, void *stream) {
    PDST_TRY(check_common(h, w, lambda, "pdst_set_block_precond"));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = (int64_t)h->H * h->nz * h->nz;
    h->has_blkprec = false;
    PDST_TRY(h->blkP64.alloc(sizeof(double) * std::max<int64_t>(total, 1)));
    PDST_TRY(h->blkP32.alloc(sizeof(float) * std::max<int64_t>(total, 1)));
    PDST_TRY(h->blkP64T.alloc(sizeof(double) * std::max<int64_t>(total, 1)));
    PDST_TRY(h->blkP32T.alloc(sizeof(float) * std::max<int64_t>(total, 1)));
    if (total == 0) {
        h->has_blkprec = true;
        return PDST_OK;
    }
    const unsigned gv = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    if (P_dev) {
        k_copy_upper<<<gv, 256, 0, s>>>(total, h->nz, P_dev, h->blkP64.as<double>(),
                                         h->blkP32.as<float>(), h->blkP64T.as<double>(),
                                         h->blkP32T.as<float>());
        PDST_CUDA(cudaGetLastError());
        PDST_CUDA(cudaStreamSynchronize(s));
        h->has_blkprec = true;
        return PDST_OK;
    }
    DevBuf B, bad;
    PDST_TRY(B.alloc(sizeof(double) * total));
    PDST_TRY(bad.alloc(sizeof(int)));
    PDST_TRY(gram_blocks(h, w, lambda, B.as<double>(), s));
    const int big = 0x7fffffff;
    PDST_CUDA(cudaMemcpyAsync(bad.p, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    const unsigned gb = (unsigned)((h->H + IC_WARPS - 1) / IC_WARPS);
    k_inv_chol<<<gb, 32 * IC_WARPS, 0, s>>>(h->H, h->nz, B.as<double>(), h->blkP64.as<double>(),
                                              h->blkP32.as<float>(), h->blkP64T.as<double>(),
                                              h->blkP32T.as<float>(), bad.as<int>());
    PDST_CUDA(cudaGetLastError());
    int first_bad = big;
    PDST_CUDA(cudaMemcpyAsync(&first_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    if (first_bad != big) {
        set_error("pdst_set_block_precond: the depth block of cell %d is not positive definite "
                  "(no ray crosses it and w = lambda = 0?)", first_bad);
        return PDST_ERR_BREAKDOWN;
    }
    h->has_blkprec = true;
    return PDST_OK;
}

extern "C" pdst_status pdst_get_block_precond(pdst_handle_t h, double *P_dev_out, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_get_block_precond: handle is NULL");
    if (!h->has_blkprec) {
        set_error("pdst_get_block_precond: no block preconditioner is set");
        return PDST_ERR_STATE;
    }
    const int64_t total = (int64_t)h->H * h->nz * h->nz;
    PDST_CHECK_ARG(P_dev_out != nullptr || total == 0, "pdst_get_block_precond: P_dev_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (total > 0)
        PDST_CUDA(cudaMemcpyAsync(P_dev_out, h->blkP64.p, sizeof(double) * total,
                                  cudaMemcpyDeviceToDevice, s));
    PDST_CUDA(cudaStreamSynchronize(s));
    return PDST_OK;
}
