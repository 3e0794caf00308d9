// common.cuh -- internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/pdst.h"

namespace pdst {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);

// Evaluate a CUDA call; on failure record the message and return the status.
#define PDST_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::pdst::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                              cudaGetErrorString(e_));                               \
            return e_ == cudaErrorMemoryAllocation ? PDST_ERR_OOM : PDST_ERR_CUDA;   \
        }                                                                            \
    } while (0)

#define PDST_TRY(expr)                                                               \
    do {                                                                             \
        pdst_status s_ = (expr);                                                     \
        if (s_ != PDST_OK) return s_;                                                \
    } while (0)

#define PDST_CHECK_ARG(cond, ...)                                                    \
    do {                                                                             \
        if (!(cond)) {                                                               \
            ::pdst::set_error(__VA_ARGS__);                                          \
            return PDST_ERR_ARG;                                                     \
        }                                                                            \
    } while (0)

// ------------------------------------------------------------ device memory

// Owning device buffer (cudaMalloc / cudaFree).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    pdst_status alloc(size_t nbytes) {
        if (p && bytes >= nbytes) return PDST_OK;
        release();
        if (nbytes == 0) nbytes = 16;
        cudaError_t e = cudaMalloc(&p, nbytes);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            set_error("cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? PDST_ERR_OOM : PDST_ERR_CUDA;
        }
        bytes = nbytes;
        return PDST_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    // take over o's memory (o ends empty)
    void take(DevBuf &o) {
        release();
        p = o.p;
        bytes = o.bytes;
        o.p = nullptr;
        o.bytes = 0;
    }
};

// ------------------------------------------------------------- LSQR state

// Scalars of one LSQR recurrence (Paige & Saunders 1982 notation), kept in
// device memory and advanced by the last block of the adjoint kernel.
struct LsqrScalars {
    double alpha, beta;            // alpha_i (||v-bar||) and beta (||u-bar||)
    double rhobar, phibar;
    double anorm, acond, ddnorm, res2, xnorm, xxnorm, z, cs2, sn2;
    double rnorm, arnorm, bnorm;
    double t1, t2;                 // pending update x += t1 w, w = v + t2 w
    double wnorm2;                 // ||w||^2 of the current w
    double damp, atol, btol, ctol;
    double w_smooth;               // smoothing weight w
    double lam_rows;               // lambda of the appended lambda*D rows (scaled form)
    double *hist;                  // optional ||r|| history (device)
    // LSMR (Fong & Saunders 2011): rotation state, ||r|| estimate state,
    // ||A|| and cond(A) accumulators, third update coefficient
    double alphabar, zetabar, cbar, sbar, rho_prev, rhobar_prev;
    double betadd, betad, rhod_prev, tautilde_prev, thetatilde, zeta_prev, dsum;
    double anorm2, rbar_max, rbar_min;
    double t3;                     // LSMR: h = v - t3 h (t1: h-bar, t2: x)
    double alpha_next;             // alpha_{i+1} from the adjoint sweep (the forward's scale)
    double beta_next;              // beta_{i+2} from a forward that ran beside a pending step
    int32_t itn, itmax, istop, pending, done, err;
    int32_t method;                // 0 LSQR, 1 LSMR
    int32_t step_pending;          // 1: the adjoint left its scalar step to k_step
};

// "Last block" counters of the reduction kernels.
struct LsqrSync {
    unsigned int count[8];
};

// Double-float number hi + lo (two floats; arithmetic in dfloat.cuh).  Trivial
// default constructor, so it can live in shared memory and in device arrays.
struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr dfl(float v) : hi(v), lo(0.f) {}
    // nearest float, then the rest (v - hi is exact in FP64)
    __host__ __device__ dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct ValueSet {
    DevBuf csr;   // values in CSR order (row-major, cells ascending, depth fastest)
    DevBuf csc;   // element CSC order: column j = h*nz+k at nz*cell_rptr[h] + k*cnt[h]
                  // (kept with the element layout only)
    DevBuf bcsc;  // blocked CSC order: entry (cell h, row q, depth k) at
                  // (cell_rptr[h] + q)*nz + k, depth fastest (always kept)
    bool present = false;
};

// Rows of one cell per adjoint work item: chosen per handle at assembly
// (adj_chunk_rows) between these bounds.
constexpr int ADJ_CHUNK_MIN = 256;
constexpr int ADJ_CHUNK_MAX = 2048;

struct LsqrWork;   // lsqr.cu

void destroy_work(LsqrWork *w);

inline int num_sms(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 148;
}

}  // namespace pdst

struct pdst_handle {
    uint64_t uid = 0;       // unique per handle in this process (never reused)
    int device = 0;
    pdst_grid grid{};
    int64_t m = 0;          // rows of G
    int32_t n = 0;          // columns
    int32_t H = 0;          // horizontal cells nx*ny
    int32_t nz = 0;
    int64_t U = 0;          // (row, cell) runs = nnz / nz
    int64_t nnz = 0;
    int32_t n_periods = 0;
    uint32_t formats = 0;

    pdst::DevBuf row_period;   // int32 [m]
    // blocked (cell-level) indices, always built
    pdst::DevBuf row_cptr;     // int64 [m+1]  run pointer per row
    pdst::DevBuf row_cells;    // int32 [U]    cell of each run (ascending in a row)
    pdst::DevBuf cell_rptr;    // int64 [H+1]  run pointer per cell (transpose)
    pdst::DevBuf cell_rows;    // int32 [U]    rows of each cell (ascending)
    pdst::DevBuf cell_cnt;     // int32 [H]    rows per cell
    pdst::DevBuf cell_order;   // int32 [H]    cells by descending row count (work order)
    pdst::DevBuf adj_item;     // int32 [2*n_adj]  (cell, first row) of each adjoint work item
    int32_t adj_chunk = 256;   // rows of one cell per adjoint work item
    int32_t interp = 0;        // 0 cell lengths, 1 bilinear node coefficients
    int64_t n_adj = 0;         // adjoint work items: chunks of ADJ_CHUNK rows, longest cells first
    // element indices (PDST_FMT_ELEMENT)
    pdst::DevBuf row_ptr;      // int64 [m+1]
    pdst::DevBuf col;          // int32 [nnz]
    pdst::DevBuf col_ptr;      // int64 [n+1]
    pdst::DevBuf row_idx;      // int32 [nnz]
    pdst::ValueSet vals[4];    // by pdst_dtype

    // kept with pdst_build_opts.keep_lengths, for pdst_set_depth_kernels
    pdst::DevBuf run_len;      // double [U]  ray length (or node coefficient) of each run
    pdst::DevBuf run_row;      // int32 [U]   row of each run
    pdst::DevBuf run_pos;      // int64 [U]   position of each run in the blocked CSC layout
    bool has_lengths = false;

    pdst::DevBuf colscale;     // double [n] right diagonal scaling D
    bool has_colscale = false;
    pdst::DevBuf blkP64;       // double [H*nz*nz] per-cell depth blocks P_h (upper triangular)
    pdst::DevBuf blkP32;       // float  [H*nz*nz] the same, rounded (F32 and BF16 forms)
    pdst::DevBuf blkP64T;      // double [H*nz*nz] P_h^T per cell (row-major), for coalesced
    pdst::DevBuf blkP32T;      // float  [H*nz*nz]   reads of the rows of P_h
    bool has_blkprec = false;

    pdst::LsqrWork *work = nullptr;
    ~pdst_handle() { pdst::destroy_work(work); }
};

// ----------------------------------------------------------- device helpers

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T> __device__ __forceinline__ T cvt(double v);
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float>(double v) { return (float)v; }

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
