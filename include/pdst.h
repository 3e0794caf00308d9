/*
 * pdst.h -- C ABI of the B300 library for the regularised traveltime
 * least-squares solve of direct surface-wave tomography (pDSurfTomo,
 * arXiv 2604.11920).
 *
 * The library builds the sensitivity matrix G of Eq. 5-6 on the GPU from ray
 * geometry and a period depth-kernel table, and solves
 *
 *     min_m ||G m - d||^2 + w^2 ||L m||^2 + lambda^2 ||m||^2          (*)
 *
 * (the least-squares problem of Eq. 6, "Solver for the Large-scale Linear
 * System", with a smoothing term w L, L the 3-D 7-point Laplacian, and
 * damping lambda) by LSQR (Paige & Saunders 1982, the solver the paper cites
 * beside LSMR), entirely in hand-written sm_103a kernels.
 *
 * Conventions
 *  - Grid nx x ny x nz, cell size dx_km, layer thickness dz_km.  Model column
 *    j = (iy*nx + ix)*nz + k (depth fastest, Eq. 7).  Data rows follow the
 *    order of the paths passed to pdst_build_G.
 *  - Pointers named *_host are host memory; *_dev are device memory on the
 *    handle's device.  All device buffers passed in stay owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that return results to the host synchronise that stream.
 *  - Every function returns a pdst_status; on error, pdst_last_error_string()
 *    returns a message for the calling thread.  Arguments are checked on the
 *    host before any launch; no function aborts the process.
 *  - A handle may be used by one host thread at a time; solves on the same
 *    handle must not overlap (they share the handle's workspace).
 */
#ifndef PDST_H
#define PDST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdst_handle *pdst_handle_t;

typedef enum {
    PDST_OK = 0,
    PDST_ERR_ARG = 1,           /* invalid argument (checked on the host) */
    PDST_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    PDST_ERR_OOM = 3,           /* device allocation failed */
    PDST_ERR_BREAKDOWN = 4,     /* NaN/Inf met in the LSQR recurrence */
    PDST_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    PDST_ERR_NOT_CONVERGED = 6, /* reserved: a solve reports istop = 7 instead */
    PDST_ERR_LIMIT = 7,         /* a documented size limit was exceeded */
    PDST_ERR_STATE = 8          /* the requested form was not built into the handle */
} pdst_status;

/* Precision of stored G values and of the LSQR vectors u, v. */
typedef enum {
    PDST_F64 = 0,   /* FP64 values, FP64 vectors (the plain form) */
    PDST_F32 = 1,   /* FP32 values, FP32 vectors, FP32 accumulation */
    PDST_BF16 = 2,  /* BF16 values, FP32 vectors, FP32 accumulation */
    PDST_DF64 = 3   /* double-float: each FP64 value kept as a float pair hi + lo
                       (about 48 significant bits), vectors and accumulation in
                       the same form, all arithmetic on the FP32 pipe.  Blocked
                       layout and pdst_lsqr / pdst_lsqr_host only (no counterpart
                       in the paper: B300's FP64 pipe bounds the PDST_F64 sweeps) */
} pdst_dtype;

/* Index layout used by the sparse products. */
typedef enum {
    PDST_FMT_ELEMENT = 0, /* CSR + CSC, one int32 index per stored entry */
    PDST_FMT_BLOCKED = 1  /* one int32 index per (row, cell) run of nz entries */
} pdst_format;

typedef struct {
    int32_t nx, ny, nz;
    double dx_km;     /* horizontal cell size (km) */
    double dz_km;     /* layer thickness (km); not used by the assembly itself */
} pdst_grid;

typedef struct {
    uint32_t value_dtypes; /* bit mask of (1u << pdst_dtype) value copies to keep; 0 = F64|F32 */
    uint32_t formats;      /* bit mask of (1u << pdst_format) index layouts; 0 = both */
    const double *kdz_cells; /* optional host table (nx*ny x n_periods x nz, cell h = iy*nx+ix
                                slowest, depth fastest): a depth kernel per horizontal cell,
                                value (r, h, k) = l_h(r) * kdz_cells[h][t(r)][k] (laterally
                                varying 1-D models under Eq. 5); NULL: kdz for every cell.
                                Copied; must be finite. */
    int32_t interp;        /* 0 (default): each chord's length goes to the cell holding its
                              midpoint; 1: Eq. 1's bilinear interpolation coefficients v_ik,
                              each chord's length split over the four grid nodes around its
                              midpoint (nodes at cell centres, so the columns keep the cell
                              numbering; needs nx, ny >= 2) */
    int32_t keep_lengths;  /* 1: keep each (row, cell) run's ray length and its place in the
                              transposed layout, so that pdst_set_depth_kernels can replace
                              the depth kernels later (20 bytes per run); 0 (default): free
                              them after assembly */
} pdst_build_opts;

/*
 * Build G on the device (Eq. 5-7, synthetic form).
 *
 * Row r of G is the ray of path r at period path_period[r]:
 *   G[r, h*nz + k] = l_h(r) * kdz[path_period[r]*nz + k]
 * for every horizontal cell h = iy*nx + ix the ray crosses, where l_h(r) is
 * the ray length inside h.  The ray is the quadratic Bezier curve with
 * control points ctrl_host[6r .. 6r+5] = (P0x, P0y, P1x, P1y, P2x, P2y) in km;
 * it is cut into N = max(1, ceil(4 * (|P1-P0| + |P2-P1|) / dx)) chords of
 * equal parameter step, each chord's length goes to the cell holding its
 * midpoint (clamped into the grid), and lengths are summed per cell in chord
 * order.  A ray of zero length gives an empty row.  Every hit cell stores all
 * nz depth entries (explicit zeros included), cells ascending within a row.
 * The FP64 values equal, bit for bit, the same recipe evaluated with one
 * rounding per written operation (no fused multiply-add).
 *
 * Inputs are host arrays, copied to the device; n_paths may be 0.  The call
 * is synchronous.  Errors: PDST_ERR_ARG (bad sizes, non-finite coordinates,
 * period index out of range), PDST_ERR_LIMIT (a ray that may cross more
 * distinct cells than the per-warp list holds, about 17,000), PDST_ERR_OOM,
 * PDST_ERR_CUDA.  On success *out owns all device memory of G; release it
 * with pdst_destroy.
 */
pdst_status pdst_build_G(const pdst_grid *grid, int64_t n_paths, const double *ctrl_host,
                         const int32_t *path_period_host, int32_t n_periods,
                         const double *kdz_host, const pdst_build_opts *opts,
                         void *stream, pdst_handle_t *out);

/* Release a handle and all device memory it owns.  NULL is accepted. */
pdst_status pdst_destroy(pdst_handle_t h);

/* Sizes: rows m, columns n, stored entries nnz (any pointer may be NULL). */
pdst_status pdst_G_info(pdst_handle_t h, int64_t *m, int32_t *n, int64_t *nnz);

/*
 * Copy G (CSR) or G^T (CSR of the transpose, i.e. CSC of G; rows ascending
 * within each column) to caller-allocated host arrays: ptr (m+1 or n+1),
 * idx (nnz), val (nnz, the stored values of `dtype` widened to FP64).  Any
 * output pointer may be NULL.  PDST_ERR_STATE if that dtype was not kept.
 * The index arrays are built from the blocked layout when the element layout
 * was not kept.  Synchronous.
 */
pdst_status pdst_G_export_csr(pdst_handle_t h, int32_t dtype, int64_t *row_ptr_host,
                              int32_t *col_host, double *val_host);
pdst_status pdst_G_export_csc(pdst_handle_t h, int32_t dtype, int64_t *col_ptr_host,
                              int32_t *row_host, double *val_host);

/*
 * y = G x (trans = 0; x has n entries, y has m) or y = G^T x (trans = 1),
 * with the stored values of `dtype`, FP64 input/output vectors (device) and
 * FP64 accumulation.  Gather-only kernels (CSR for G, CSC for G^T), no
 * atomics.  Asynchronous on `stream`.
 */
pdst_status pdst_apply_G(pdst_handle_t h, int32_t dtype, int32_t trans, const double *x_dev,
                         double *y_dev, void *stream);

typedef struct {
    int32_t dtype;     /* pdst_dtype of values and u/v vectors (default PDST_F64) */
    int32_t format;    /* pdst_format (default PDST_FMT_ELEMENT) */
    double atol;       /* < 0: use tol */
    double btol;       /* < 0: use tol */
    double conlim;     /* <= 0: 1e8 */
    int32_t precond;   /* 0 none; 1 right diagonal scaling set by pdst_set_col_scaling;
                          2 right block-diagonal preconditioner (one nz x nz block per
                          horizontal cell) set by pdst_set_block_precond: blocked format,
                          nz <= 32, dtype F64, F32 or BF16 (refine_dtype likewise) */
    int32_t kblock;    /* iterations per graph launch (<= 0: 16) */
    int32_t use_graph; /* 1 (default): CUDA graph replay; 0: plain launches */
    int32_t profile;   /* per-kernel device time in pdst_lsqr_info: 1, one iteration per
                          launch group, each kernel bracketed by CUDA events (k_step in line);
                          2, the CUDA-graph replay itself with event nodes around the forward,
                          the update and the adjoint of every iteration (k_step on its branch
                          beside the forward); 0 (default) none */
    double *rnorm_hist_dev; /* optional device array (itmax): ||r|| after each iteration */
    int32_t refine;    /* > 0: refinement with up to `refine` sweeps:
                          m <- m + D argmin ||A_D dy - r(m)||, the residual r(m) of the
                          augmented system computed in FP64 with the FP64 values of G (keep
                          PDST_F64 in pdst_build_G).  Sweep 0 solves in `dtype` to tol;
                          later sweeps solve in refine_dtype with atol = btol = refine_tol
                          (the stopping rules then hold for the full problem at m).  Stops
                          early when a sweep needs no iteration.  0 (default): one solve. */
    int32_t refine_dtype; /* pdst_dtype of sweeps 1.. (-1, default: dtype) */
    double refine_tol; /* tolerance of sweeps 1.. (default 1e-5) */
    int32_t method;    /* PDST_LSQR (default) or PDST_LSMR: the same Golub-Kahan sweeps,
                          the recurrence and x update of LSQR (Paige & Saunders 1982) or
                          of LSMR (Fong & Saunders 2011, the solver pDSurfTomo uses).  LSMR
                          reports ||r|| and ||A^T r|| from its own recurrences, ||x|| from
                          x, cond(A) as max/min of its second rotation's diagonal; same
                          stopping tests and istop numbering.  Not available in
                          pdst_lsqr_noalloc. */
    int32_t reserved0;
} pdst_lsqr_opts;

/* Krylov method of pdst_lsqr (pdst_lsqr_opts.method). */
typedef enum { PDST_LSQR = 0, PDST_LSMR = 1 } pdst_method;

/* Fill *o with the defaults listed above. */
void pdst_lsqr_opts_default(pdst_lsqr_opts *o);

typedef struct {
    int32_t iters;   /* iterations performed */
    int32_t istop;   /* 0 x = 0 is exact; 1 ||r|| <= btol||b|| + atol||A||||x||;
                        2 ||A^T r|| <= atol ||A|| ||r||; 3 cond(A) >= conlim;
                        4-6 the same at machine precision; 7 itmax reached */
    double rnorm;    /* estimate of ||[d; 0; 0] - [G; w L; lambda I] m|| (or scaled form) */
    double arnorm;   /* estimate of ||A^T r|| */
    double anorm;    /* estimate of ||A||_F */
    double acond;    /* estimate of cond(A) */
    double xnorm;    /* estimate of ||x|| (of y when scaled) */
    double bnorm;    /* ||d|| */
    int32_t kernel_launches; /* kernels this call launched (graph nodes included) */
    int32_t profiled_iters;  /* iterations covered by the *_ms fields (profile = 1) */
    double fwd_ms;   /* total device time of the forward kernel A v (profile = 1) */
    double adj_ms;   /* total device time of the adjoint kernel A^T u (+ its norm) */
    double upd_ms;   /* total device time of the x/w update and the scalar step of the
                        recurrence (one-warp kernel; in graph replay it runs beside the
                        forward) */
    int32_t sweeps;  /* refinement sweeps performed (0 without refinement); iters is the
                        total over all sweeps and the other fields describe the last one */
    int32_t reserved;
    double correction; /* ||last correction|| / ||m|| (refinement) */
} pdst_lsqr_info;

/*
 * Solve (*) by LSQR (Paige & Saunders 1982) on the augmented operator
 * A = [G; w L] with damping lambda in the recurrence, or, with
 * opts->precond = 1 and a scaling D set by pdst_set_col_scaling, on
 * A_D = [G D; w L D; lambda D] with no recurrence damping and m = D y (the
 * same minimiser), or, with opts->precond = 2 and the blocks P set by
 * pdst_set_block_precond, on A_P = [G P; w L P; lambda P] and m = P y.
 * d_dev: m_rows FP64 (device, caller-owned).  m_out_dev: n FP64 (device,
 * caller-owned).  tol sets atol = btol unless opts overrides;
 * conlim defaults to 1e8.  The Golub-Kahan scalars, the rotations, the norm
 * estimates and the x/w update are FP64 in every dtype.  info (host) may be
 * NULL.  The call is synchronous on `stream`.
 * Errors: PDST_ERR_ARG, PDST_ERR_STATE (dtype/format not built, or precond
 * requested without a scaling), PDST_ERR_BREAKDOWN, PDST_ERR_CUDA.
 */
pdst_status pdst_lsqr(pdst_handle_t h, const double *d_dev, double w, double lambda,
                      int32_t itmax, double tol, double *m_out_dev, pdst_lsqr_info *info,
                      const pdst_lsqr_opts *opts, void *stream);

/*
 * Allocation-free variant of pdst_lsqr.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory while
 * they solve.  Examples are a serving or plugin host that owns all device
 * memory through its own pool and forbids allocation once it is running, a
 * process under a hard device-memory cap where a late cudaMalloc may fail, and
 * a latency-sensitive loop that cannot afford the device-wide synchronisation
 * cudaFree brings.  pdst_lsqr allocates its workspace (and pinned host
 * memory, and a CUDA graph) on first use; this function allocates nothing:
 * all solve scratch (scalars, reduction partials, u-bar, v-bar, x, w) lives in
 * one file-scope device array of 16 MiB that every GPU which loads the
 * library holds until the process exits.
 *
 * Arguments and results are those of pdst_lsqr (same kernels in the same
 * order, same answer bit for bit); the iterations are plain kernel launches
 * (opts->use_graph is ignored), opts->profile and opts->refine must be 0,
 * opts->precond 0 or 1 and opts->method PDST_LSQR (PDST_ERR_ARG otherwise).  The handle's device must
 * be the current device.  The first call on a device looks up the array's
 * device address there (cudaGetSymbolAddress) and keeps it for later calls;
 * make that first call before any stream capture, and do not call this
 * function again on a device after cudaDeviceReset there (the module, and
 * with it the array, may then live at another address).
 * Every call on a device shares the one array, which keeps the previous
 * call's contents (the function clears what must start at zero): calls that
 * overlap on the GPU -- from two host threads or on two streams -- race and
 * give wrong results.  Synchronous on `stream`.
 * Errors: as pdst_lsqr, plus PDST_ERR_LIMIT when the system's scratch exceeds
 * 16 MiB: s (m + 3n) + 16 n bytes (s = 8 in FP64, 4 in FP32/BF16), plus
 * s (nnz / 256 + n) for the adjoint's per-chunk sums, plus about 100 KiB,
 * plus n more vector entries when lambda rows are appended (e.g. the
 * 64 x 64 x 16 system with 171,360 rows needs about 8.5 MB in FP64).
 */
pdst_status pdst_lsqr_noalloc(pdst_handle_t h, const double *d_dev, double w, double lambda,
                              int32_t itmax, double tol, double *m_out_dev,
                              pdst_lsqr_info *info, const pdst_lsqr_opts *opts, void *stream);

/* Damping sweep (no counterpart in the paper's solver module): the solutions of
 *     min_m ||G m - d||^2 + w^2 ||L m||^2 + lambda_l^2 ||m||^2,   l = 0..nlam-1,
 * from ONE Golub-Kahan bidiagonalisation of A = [G; w L].  The vectors u, v
 * (and alpha, beta) of LSQR do not depend on the damping, which enters only
 * the scalar recurrence (Paige & Saunders 1982), so each damping value costs
 * one recurrence and one x/w update per iteration instead of a full solve.
 * Every value stops on its own tests (atol = btol = tol unless opts set them);
 * the sweeps run until all have stopped or itmax.  Results are identical to
 * nlam separate pdst_lsqr calls with the same options.
 *   lambda_host  nlam damping values (host, copied), 1 <= nlam <= 64
 *   m_out_dev    nlam caller-owned device arrays of n doubles
 *   infos        nlam entries (iters, istop and estimates per value), or NULL
 *   opts         dtype / format / kblock / atol / btol / conlim as pdst_lsqr;
 *                precond, refine, profile must be 0 and method PDST_LSQR
 * Errors as pdst_lsqr.  Synchronous on return. */
pdst_status pdst_lsqr_damping_sweep(pdst_handle_t h, const double *d_dev, double w, int32_t nlam,
                                    const double *lambda_host, int32_t itmax, double tol,
                                    double *const *m_out_dev, pdst_lsqr_info *infos,
                                    const pdst_lsqr_opts *opts, void *stream);

/* Same as pdst_lsqr with host d and m (pinned or pageable): copies d in and
 * m out inside the call (the end-to-end path). */
pdst_status pdst_lsqr_host(pdst_handle_t h, const double *d_host, double w, double lambda,
                           int32_t itmax, double tol, double *m_out_host,
                           pdst_lsqr_info *info, const pdst_lsqr_opts *opts, void *stream);

/*
 * Right diagonal scaling m = D y for pdst_lsqr with precond = 1.
 * D_dev: n FP64 positive entries (device, copied into the handle), or NULL to
 * use the column-norm scaling D_j = 1 / ||[G; w L; lambda I]_{:,j}|| of the
 * augmented operator for the given w, lambda.  Synchronous.
 */
pdst_status pdst_set_col_scaling(pdst_handle_t h, const double *D_dev, double w, double lambda,
                                 void *stream);

/*
 * Per-cell depth-block right preconditioner (precond = 2).  The nz columns of
 * one horizontal cell h (Eq. 7's depth-fastest order: j = h*nz + k) are
 * strongly coupled: each row of G (Eq. 5) touches all of them through one
 * depth kernel, and L couples neighbouring depths.  Let A = [G; w L; lambda I]
 * and A_h its nz columns of cell h; the preconditioner factors the diagonal
 * block B_h = A_h^T A_h of the normal matrix as B_h = R_h^T R_h (Cholesky,
 * R_h upper triangular with a positive diagonal) and runs LSQR on A P with
 * P = blockdiag(P_h), P_h = R_h^{-1}, so that every cell's column group of
 * A P is orthonormal (the block form of column-norm scaling).  m = P y.
 *
 * pdst_depth_blocks: B_h for every cell into B_dev, (nx*ny) x nz x nz FP64,
 *   row-major per cell (entry (h, i, k) at (h*nz + i)*nz + k), from the FP64
 *   values of G when kept, else the FP32 or BF16 ones widened; device,
 *   caller-owned.  Asynchronous on `stream`.
 * pdst_set_block_precond: P_dev NULL computes B_h as above and P_h = R_h^{-1}
 *   in FP64 on the device for the given w, lambda; otherwise P_dev holds the
 *   blocks in the same layout (device, copied; only the upper triangle is
 *   read, the lower one is taken as zero).  The handle keeps P in FP64 and an
 *   FP32 copy (used by the F32 and BF16 forms).  Needs nz <= 32.
 *   Synchronous.  PDST_ERR_BREAKDOWN when a block is not positive definite
 *   (a cell no ray crosses with w = lambda = 0); the handle then keeps no
 *   preconditioner.
 * pdst_get_block_precond: copies the FP64 blocks P into P_dev_out (same
 *   layout).  PDST_ERR_STATE if none is set.  Synchronous.
 * Errors: PDST_ERR_ARG (NULL handle or output, non-finite or negative w or
 * lambda), PDST_ERR_LIMIT (nz > 32), PDST_ERR_OOM, PDST_ERR_CUDA.
 */
pdst_status pdst_depth_blocks(pdst_handle_t h, double w, double lambda, double *B_dev,
                              void *stream);
pdst_status pdst_set_block_precond(pdst_handle_t h, const double *P_dev, double w, double lambda,
                                   void *stream);
pdst_status pdst_get_block_precond(pdst_handle_t h, double *P_dev_out, void *stream);

typedef struct {
    int32_t tile_rows;        /* G rows per forward work item; 0 = chosen by the autotuner,
                                 which times one whole iteration for 2, 8 and 32 rows */
    int32_t kblock;           /* iterations per graph launch (<= 0: 8) */
    int32_t chosen_tile_rows; /* out: the tile used by the call */
    int32_t kernel_launches;  /* out: kernels launched by the call (graph nodes included) */
    double tune_ms[4];        /* out: iteration time per autotuner candidate (ms) */
    int32_t precond;          /* 0 none; 1 each system's right diagonal scaling set by
                                 pdst_set_col_scaling on its handle: pair (s, j) solves
                                 A_D = [G D; w L D; lambda_j D] with no recurrence damping and
                                 returns m = D y (the same minimiser); 2 each system's
                                 depth blocks P set by pdst_set_block_precond on its handle
                                 (A_P = [G P; w L P; lambda_j P], m = P y; one kernel more
                                 per iteration finishes each cell) */
    int32_t reserved;
} pdst_batched_opts;

/* Fill *o with the defaults listed above. */
void pdst_batched_opts_default(pdst_batched_opts *o);

/*
 * Batched LSQR: nsys independent systems (each its own handle; grid sizes,
 * row counts and nnz may differ) with nrhs[s] right-hand sides each (1..16),
 * solved together.  Each phase of an iteration is one persistent launch over a
 * work list spanning all systems, and each matrix entry read from HBM serves
 * all right-hand sides of its system.  Each (system, right-hand side) pair runs
 * its own LSQR recurrence (Paige & Saunders 1982; FP64 scalars) on
 * A_s = [G_s; w_s L] with damping lambda[s][j], and stops on its own
 * (atol = btol = tol, conlim = 1e8, itmax iterations at most).
 *
 * d_dev[s]: m_s x nrhs[s] FP64 (device), right-hand side fastest.
 * w[s]: smoothing weight per system.  lambda[s]: nrhs[s] damping values (host).
 * m_out_dev[s]: n_s x nrhs[s] FP64 (device, caller-owned), right-hand side
 * fastest.  infos: sum(nrhs) entries, system-major (may be NULL).  Each
 * system needs nz <= 32 (PDST_ERR_LIMIT otherwise); a batch with a system of
 * more than 16 depth nodes runs its adjoint in kernels that hold 32 depths
 * per lane (two blocks per SM) for all of its systems.  dtype:
 * values and u/v vectors (PDST_F32 / PDST_BF16 use FP32 vectors).  opts may be
 * NULL (autotuned tile, kblock 8); its out fields are filled when given.
 * Work space for the batch is allocated on the first call and reused while the
 * same handles, right-hand-side counts and dtype are passed again.
 * Synchronous on `stream`.  Errors: PDST_ERR_ARG, PDST_ERR_STATE (dtype not
 * kept), PDST_ERR_BREAKDOWN, PDST_ERR_OOM, PDST_ERR_CUDA.
 */
pdst_status pdst_lsqr_batched(int32_t nsys, const pdst_handle_t *hs, const int32_t *nrhs,
                              const double *const *d_dev, const double *w,
                              const double *const *lambda, int32_t itmax, double tol,
                              int32_t dtype, double *const *m_out_dev, pdst_lsqr_info *infos,
                              pdst_batched_opts *opts, void *stream);

/*
 * Column norms c_j = ||[G; w L; lambda I]_{:,j}||_2 of the augmented operator
 * (c_dev: n FP64, device).  Asynchronous on `stream`.
 */
pdst_status pdst_col_norms(pdst_handle_t h, double w, double lambda, double *c_dev, void *stream);

/* Set the handle's right scaling to D_j = c_j^(-p) (p = 1: column-norm
 * scaling; p = 0: no scaling).  Synchronous. */
pdst_status pdst_set_col_scaling_power(pdst_handle_t h, double w, double lambda, double p,
                                       void *stream);

/* ---- learned right-diagonal preconditioner --------------------------------
 * A small MLP maps 8 per-column features of G to the scaling D of
 * pdst_set_col_scaling: xh = (f - mu) / sigma, h1 = tanh(W1 xh + b1),
 * h2 = tanh(W2 h1 + b2), z = w3 . h2 + b3, D = softplus(z).  Parameters are
 * one FP32 device vector in the order mu[8], sigma[8], W1[64][8], b1[64],
 * W2[64][64], b2[64], w3[64], b3 (PDST_MLP_NPARAM floats); the last
 * PDST_MLP_NTRAIN of them (from W1) are trained. */
#define PDST_MLP_NFEAT 8
#define PDST_MLP_HIDDEN 64
#define PDST_MLP_NPARAM (2 * PDST_MLP_NFEAT + PDST_MLP_HIDDEN * PDST_MLP_NFEAT + \
                         PDST_MLP_HIDDEN + PDST_MLP_HIDDEN * PDST_MLP_HIDDEN + \
                         2 * PDST_MLP_HIDDEN + 1)
#define PDST_MLP_NTRAIN (PDST_MLP_NPARAM - 2 * PDST_MLP_NFEAT)

/*
 * Per-column features of G (feat_dev: n x 8 FP32, device, row = column j):
 *  f0 log(||G_:j|| + 1e-8)        f1 log(1 + number of rows in column j)
 *  f2 (k + 1/2) / nz (depth)       f3 sum_r G_rj^2 log T(r) / sum_r G_rj^2 (0 if empty)
 *  f4, f5, f6 log of the mean, min, max of (||G_:i|| + 1e-8) over the 7-point
 *             neighbours i of j    f7 log(max_r |G_rj| + 1e-8)
 * log_periods_host: n_periods values log T (host), T in the units of the
 * depth-kernel table.  Uses the FP64 values when kept.  Synchronous.
 */
pdst_status pdst_precond_features(pdst_handle_t h, const double *log_periods_host, float *feat_dev,
                                  void *stream);

/* D = softplus(MLP(features)) for n columns: D_dev (FP64) and/or logD_dev
 * (FP32, log D) may be NULL.  Asynchronous. */
pdst_status pdst_mlp_forward(const float *params_dev, const float *feat_dev, int64_t n,
                             double *D_dev, float *logD_dev, void *stream);

/*
 * Gradient of the mean loss (1/B) sum_s (log D(f_idx[s]) - t[idx[s]])^2 over a
 * batch of B = batch samples (idx_dev: B int32 row indices into feat_dev and
 * target_dev).  grad_dev: PDST_MLP_NTRAIN + 1 FP32; the last entry receives
 * the mean loss.  Per-sample work in one kernel, then a fixed-order sum over
 * the batch per parameter (deterministic).  Synchronous.
 */
pdst_status pdst_mlp_grad(const float *params_dev, const float *feat_dev, const int32_t *idx_dev,
                          const float *target_dev, int32_t batch, float *grad_dev, void *stream);

/* One Adam step (bias-corrected, step >= 1) on the trained parameters;
 * m_dev, v_dev: PDST_MLP_NTRAIN FP32 moment vectors.  Asynchronous. */
pdst_status pdst_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev,
                          int64_t step, double lr, double beta1, double beta2, double eps,
                          void *stream);

/* ---- outer nonlinear loop ------------------------------------------------
 * The paper's inversion (after Eq. 6) solves Eq. 6 for the model
 * perturbation, updates the model, rebuilds G from the updated model and
 * repeats until the RMS traveltime error falls below a threshold.  The rays
 * (the traveltime module) stay fixed here; what follows the model is the depth
 * kernel of each horizontal cell, by this synthetic kernel module: with
 * s_h = (1/nz) sum_k (1 + m[h*nz + k]) (the column's mean relative S-wave
 * velocity, summed in depth order) and a = kernel_power,
 *     z0(h, t) = z0_factor * T_t * s_h^a,
 *     K[h][t][k] = (z_k / z0) * exp(1 - z_k / z0) * dz,  z_k = (k + 1/2) dz,
 * a faster column being sampled deeper (the 1-D table of Eq. 5's synthetic
 * form at m = 0). */

/* K (device, nx*ny x n_periods x nz FP64, cell slowest, depth fastest) from
 * the model m_dev (n FP64, device); periods_host: n_periods values T (host).
 * The grid's dz_km is the layer thickness.  Asynchronous on `stream`.
 * Errors: PDST_ERR_ARG (NULL pointers, non-finite or non-positive factor or
 * period). */
pdst_status pdst_depth_kernels_from_model(pdst_handle_t h, const double *periods_host,
                                          double z0_factor, double kernel_power,
                                          const double *m_dev, double *kdz_cells_dev,
                                          void *stream);

/* Replace the depth kernels of G: every kept value copy (all dtypes and
 * layouts) is expanded again as value(r, h, k) = l_h(r) * K[h][t(r)][k] from
 * the per-cell table kdz_cells_dev (device, as above), the ray lengths and the
 * sparsity pattern unchanged -- the same values pdst_build_G gives with that
 * table as kdz_cells.  A scaling set by pdst_set_col_scaling is not updated.
 * Needs keep_lengths at assembly (PDST_ERR_STATE otherwise).  Synchronous. */
pdst_status pdst_set_depth_kernels(pdst_handle_t h, const double *kdz_cells_dev, void *stream);

typedef struct {
    int32_t max_outer;     /* model updates at most (default 8) */
    int32_t reserved0;
    double rms_tol;        /* stop once RMS <= rms_tol (default 0) */
    double min_decrease;   /* stop once the RMS fell by less than this fraction since the
                              previous model (default 0.01); if it rose, the previous model
                              is returned */
    double z0_factor;      /* kernel depth per period (default 1.2 km/s) */
    double kernel_power;   /* a above (default 1; 0: the kernels do not follow the model) */
    pdst_lsqr_opts inner;  /* options of each update's solve (pdst_lsqr); with precond = 1
                              the column-norm scaling of the current G, with precond = 2 its
                              depth-block preconditioner, is set before each solve */
} pdst_outer_opts;

/* Fill *o with the defaults listed above (inner: pdst_lsqr_opts_default). */
void pdst_outer_opts_default(pdst_outer_opts *o);

typedef struct {
    int32_t updates;       /* model updates made */
    int32_t reason;        /* 1 RMS <= rms_tol; 2 the RMS stopped decreasing; 3 max_outer */
    int32_t inner_iters;   /* LSQR iterations over all updates */
    int32_t reserved;
    double rms_first;      /* RMS of d_obs - G(0) 0 = d_obs */
    double rms_final;      /* RMS of the returned model */
} pdst_outer_info;

/*
 * The outer loop from m = 0: for the current model m, K = kernels(m)
 * (pdst_depth_kernels_from_model), G(m) (pdst_set_depth_kernels), the data
 * residual r = d_obs - G(m) m and RMS = sqrt(mean(r^2)) (FP64 values); stop as
 * opts says (checked before each solve); else solve Eq. 6 for the update
 *     dm = argmin ||G(m) dm - r||^2 + w^2 ||L dm||^2 + lambda^2 ||dm||^2
 * by pdst_lsqr (itmax, tol, opts->inner) and set m <- m + dm.
 *   d_obs_dev     m_rows FP64 observed traveltime perturbations (device)
 *   periods_host  n_periods values T of the handle's periods (host)
 *   m_out_dev     n FP64 (device): the final model
 *   rms_hist_host NULL or max_outer + 1 doubles: the RMS before each solve and of
 *                 the final model (updates + 1 entries written)
 * The handle needs FP64 values and keep_lengths; its values end as G of the
 * last model checked.  Synchronous.  Errors: as pdst_lsqr and
 * pdst_set_depth_kernels.
 */
pdst_status pdst_outer_loop(pdst_handle_t h, const double *d_obs_dev, const double *periods_host,
                            double w, double lambda, int32_t itmax, double tol,
                            const pdst_outer_opts *opts, double *m_out_dev,
                            double *rms_hist_host, pdst_outer_info *info, void *stream);

/*
 * Measurement aid (no counterpart in the paper): one sequential read of
 * `bytes` bytes at buf_dev (device, caller-owned, 16-byte aligned, bytes a
 * multiple of 16) with 16-byte streaming loads by a grid of 8 blocks per SM,
 * no gathers and no dependent loads; the data are summed so the loads are
 * kept, and nothing is written.  Timed by the caller on `stream`, it gives the
 * rate at which this GPU streams a sweep's value bytes, the ceiling against
 * which the sweeps' gathers are read.  Asynchronous.  Errors: PDST_ERR_ARG.
 */
pdst_status pdst_stream_read(const void *buf_dev, int64_t bytes, void *stream);

/* Message for the last error on the calling thread ("" if none). */
const char *pdst_last_error_string(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t pdst_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PDST_H */
