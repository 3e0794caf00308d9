/*
 * oracle.c -- plain FP64 CPU oracle for the regularised traveltime
 * least-squares solve.  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * product path.  It shares no code with the CUDA library.
 *
 * What it computes (pDSurfTomo, arXiv 2604.11920, and Paige & Saunders 1982):
 *
 *   1. The sensitivity matrix G of Eq. 5-6 in its synthetic form
 *      G[r, h*nz + k] = l_h(r) * Kdz[t(r)][k]: every horizontal cell h that the
 *      ray of row r crosses contributes all nz depth columns (Eq. 5), columns
 *      are ordered depth-fastest (Eq. 7).  l_h(r) is the length of the ray
 *      inside cell h, obtained by cutting the quadratic Bezier ray into
 *      N = max(1, ceil(4 * polygon_length / dx)) chords of equal parameter
 *      step (a quarter cell or less each), giving each chord to the cell that
 *      holds its midpoint (clamped to the grid) and summing chord lengths per
 *      cell in chord order.
 *   2. Its transpose (rows ascending inside each column).
 *   3. The 3-D 7-point graph Laplacian (L x)_j = sum over existing neighbours
 *      i of (x_j - x_i).
 *   4. LSQR (Paige & Saunders 1982, the solver the paper names beside LSMR in
 *      "Solver for the Large-scale Linear System") on
 *          min ||G m - d||^2 + w^2 ||L m||^2 + damp^2 ||m||^2,
 *      with the operator A = [G; w L] and the damping handled by LSQR's own
 *      damped recurrence, or, with a right diagonal scaling m = D y, on
 *      A_D = [G D; w L D; lam D] with no recurrence damping, or, with a
 *      right block-diagonal matrix P (one nz x nz block per horizontal
 *      cell), on A_P = [G P; w L P; lam P] in the same way.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so the G arithmetic rounds once per written operation).
 * Loops over independent rows or columns may run in OpenMP threads; each
 * output element is still computed by one thread in a fixed order, so
 * results do not depend on the thread count.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ G ---- */

/* Bezier point B(tau) = (1-tau)^2 P0 + 2 tau (1-tau) P1 + tau^2 P2, evaluated
 * as ((b0*p0 + b1*p1) + b2*p2) with b0 = a*a, b1 = (2*tau)*a, b2 = tau*tau,
 * a = 1 - tau. */
static void bezier(const double *c, double tau, double *x, double *y)
{
    double a = 1.0 - tau;
    double b0 = a * a;
    double b1 = (2.0 * tau) * a;
    double b2 = tau * tau;
    double tx0 = b0 * c[0], tx1 = b1 * c[2], tx2 = b2 * c[4];
    double ty0 = b0 * c[1], ty1 = b1 * c[3], ty2 = b2 * c[5];
    *x = (tx0 + tx1) + tx2;
    *y = (ty0 + ty1) + ty2;
}

/* Number of chords of one ray; 0 for a ray of zero (or non-finite) length. */
static int64_t chord_count(const double *c, double dx)
{
    double ax = c[2] - c[0], ay = c[3] - c[1];
    double bx = c[4] - c[2], by = c[5] - c[3];
    double la = sqrt(ax * ax + ay * ay);
    double lb = sqrt(bx * bx + by * by);
    double lp = la + lb;
    if (!(lp > 0.0))
        return 0;
    double q = (4.0 * lp) / dx;
    double nf = ceil(q);
    if (nf < 1.0)
        nf = 1.0;
    return (int64_t)nf;
}

static int clamp_cell(double coord, double dx, int ncell)
{
    double f = floor(coord / dx);
    if (f < 0.0)
        f = 0.0;
    if (f > (double)(ncell - 1))
        f = (double)(ncell - 1);
    return (int)f;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Walk one ray: acc[h] += chord length for every chord, in chord order.
 * touched[] receives each newly hit cell once; returns how many. */
/* Lower node of the bilinear interpolation along one axis and the fraction
 * towards the next node: nodes at (i + 1/2) dx, i = 0..n-1 (cell centres);
 * i0 = floor(coord/dx - 1/2) clamped to [0, n-2], t = coord/dx - 1/2 - i0
 * clamped to [0, 1]. */
static int bilin_axis(double coord, double dx, int n, double *t)
{
    double f = coord / dx - 0.5;
    double i0 = floor(f);
    if (i0 < 0.0)
        i0 = 0.0;
    if (i0 > (double)(n - 2))
        i0 = (double)(n - 2);
    double tt = f - i0;
    if (tt < 0.0)
        tt = 0.0;
    if (tt > 1.0)
        tt = 1.0;
    *t = tt;
    return (int)i0;
}

static void add_to(int h, double v, double *acc, unsigned char *seen, int *touched, int *nt)
{
    if (!seen[h]) {
        seen[h] = 1;
        acc[h] = 0.0;
        touched[(*nt)++] = h;
    }
    acc[h] = acc[h] + v;
}

/* Walk one ray: interp 0 gives each chord's length to the cell holding its
 * midpoint; interp 1 (Eq. 1's bilinear coefficients v_ik) splits it over the
 * four grid nodes around the midpoint with bilinear weights, in the order
 * (i0, j0), (i0+1, j0), (i0, j0+1), (i0+1, j0+1). */
static int walk_ray(const double *c, int nx, int ny, double dx, int interp, double *acc,
                    unsigned char *seen, int *touched)
{
    int64_t N = chord_count(c, dx);
    int nt = 0;
    if (N == 0)
        return 0;
    double px, py;
    bezier(c, 0.0, &px, &py);
    for (int64_t s = 1; s <= N; ++s) {
        double tau = (double)s / (double)N;
        double qx, qy;
        bezier(c, tau, &qx, &qy);
        double ex = qx - px, ey = qy - py;
        double len = sqrt(ex * ex + ey * ey);
        double mx = 0.5 * (px + qx), my = 0.5 * (py + qy);
        if (interp == 0) {
            int ix = clamp_cell(mx, dx, nx);
            int iy = clamp_cell(my, dx, ny);
            add_to(iy * nx + ix, len, acc, seen, touched, &nt);
        } else {
            double tx, ty;
            int ix = bilin_axis(mx, dx, nx, &tx);
            int iy = bilin_axis(my, dx, ny, &ty);
            double a = 1.0 - tx, b = 1.0 - ty;
            add_to(iy * nx + ix, len * (a * b), acc, seen, touched, &nt);
            add_to(iy * nx + ix + 1, len * (tx * b), acc, seen, touched, &nt);
            add_to((iy + 1) * nx + ix, len * (a * ty), acc, seen, touched, &nt);
            add_to((iy + 1) * nx + ix + 1, len * (tx * ty), acc, seen, touched, &nt);
        }
        px = qx;
        py = qy;
    }
    return nt;
}

/* Per-row number of distinct cells hit (row r has cells[r] * nz entries). */
int oracle_G_count(int nx, int ny, double dx, int interp, int64_t n_rows, const double *ctrl,
                   int32_t *cells_out)
{
    int H = nx * ny;
    int rc = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)H);
        unsigned char *seen = (unsigned char *)calloc((size_t)H, 1);
        int *touched = (int *)malloc(sizeof(int) * (size_t)H);
        if (!acc || !seen || !touched) {
#pragma omp atomic write
            rc = -1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t r = 0; r < n_rows; ++r) {
                int nt = walk_ray(ctrl + 6 * r, nx, ny, dx, interp, acc, seen, touched);
                cells_out[r] = nt;
                for (int i = 0; i < nt; ++i)
                    seen[touched[i]] = 0;
            }
        }
        free(acc);
        free(seen);
        free(touched);
    }
    return rc;
}

/* Fill CSR columns/values given row_ptr (= nz * prefix sum of the counts).
 * Value of (row r, cell h, depth k): l_h(r) * K, one rounding, with
 * K = kdz[t][k] (the same depth kernel under every cell), or, when kdz_cells
 * is given, K = kdz_cells[h][t][k] (a depth kernel per horizontal cell: the
 * laterally varying case, where G is no longer l (x) Kdz). */
int oracle_G_fill(int nx, int ny, int nz, double dx, int interp, int64_t n_rows,
                  const double *ctrl, const int32_t *row_period, const double *kdz,
                  const double *kdz_cells, int n_periods,
                  const int64_t *row_ptr, int32_t *col, double *val)
{
    int H = nx * ny;
    int rc = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)H);
        unsigned char *seen = (unsigned char *)calloc((size_t)H, 1);
        int *touched = (int *)malloc(sizeof(int) * (size_t)H);
        if (!acc || !seen || !touched) {
#pragma omp atomic write
            rc = -1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t r = 0; r < n_rows; ++r) {
                int nt = walk_ray(ctrl + 6 * r, nx, ny, dx, interp, acc, seen, touched);
                qsort(touched, (size_t)nt, sizeof(int), cmp_int);
                const double *kt = kdz + (int64_t)row_period[r] * nz;
                int64_t p = row_ptr[r];
                for (int i = 0; i < nt; ++i) {
                    int h = touched[i];
                    if (kdz_cells)
                        kt = kdz_cells + ((int64_t)h * n_periods + row_period[r]) * nz;
                    for (int k = 0; k < nz; ++k) {
                        col[p] = h * nz + k;
                        val[p] = acc[h] * kt[k];
                        ++p;
                    }
                    seen[h] = 0;
                }
            }
        }
        free(acc);
        free(seen);
        free(touched);
    }
    return rc;
}

/* Transpose a CSR matrix (m x n) by counting sort; row indices come out
 * ascending inside every column because rows are visited in order. */
void oracle_transpose(int64_t m, int32_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val, int64_t *col_ptr, int32_t *row_idx, double *val_t)
{
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t j = 0; j <= n; ++j)
        col_ptr[j] = 0;
    for (int64_t p = 0; p < row_ptr[m]; ++p)
        col_ptr[col[p] + 1] += 1;
    for (int32_t j = 0; j < n; ++j)
        col_ptr[j + 1] += col_ptr[j];
    for (int32_t j = 0; j < n; ++j)
        next[j] = col_ptr[j];
    for (int64_t r = 0; r < m; ++r)
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
            int64_t q = next[col[p]]++;
            row_idx[q] = (int32_t)r;
            val_t[q] = val[p];
        }
    free(next);
}

/* y = S x for a CSR matrix S with m rows. */
void oracle_spmv(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                 const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        double s = 0.0;
        for (int64_t p = ptr[r]; p < ptr[r + 1]; ++p)
            s += val[p] * x[idx[p]];
        y[r] = s;
    }
}

/* ------------------------------------------------------------ Laplacian -- */

/* (L x)_j = sum over the existing 7-point neighbours i of j of (x_j - x_i).
 * Neighbours are visited as k-1, k+1, ix-1, ix+1, iy-1, iy+1. */
void oracle_laplacian(int nx, int ny, int nz, const double *x, double *y)
{
    int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        int k = (int)(j % nz);
        int64_t hh = j / nz;
        int ix = (int)(hh % nx), iy = (int)(hh / nx);
        double s = 0.0;
        if (k > 0) s += x[j] - x[j - 1];
        if (k < nz - 1) s += x[j] - x[j + 1];
        if (ix > 0) s += x[j] - x[j - nz];
        if (ix < nx - 1) s += x[j] - x[j + nz];
        if (iy > 0) s += x[j] - x[j - (int64_t)nx * nz];
        if (iy < ny - 1) s += x[j] - x[j + (int64_t)nx * nz];
        y[j] = s;
    }
}

/* Squared 2-norm of every column of the augmented operator [G; w L; lam I]:
 * ||G_:j||^2 + w^2 (deg_j^2 + deg_j) + lam^2, the Laplacian column holding
 * deg_j on the diagonal and -1 at each neighbour. */
void oracle_aug_colnorm2(int32_t n, const int64_t *col_ptr, const double *val_t, int nx,
                         int ny, int nz, double w, double lam, double *out)
{
    for (int32_t j = 0; j < n; ++j) {
        double g = 0.0;
        for (int64_t q = col_ptr[j]; q < col_ptr[j + 1]; ++q)
            g += val_t[q] * val_t[q];
        int k = j % nz, hh = j / nz, ix = hh % nx, iy = hh / nx;
        int deg = (k > 0) + (k < nz - 1) + (ix > 0) + (ix < nx - 1) + (iy > 0) + (iy < ny - 1);
        out[j] = g + w * w * ((double)deg * deg + deg) + lam * lam;
    }
}

/* ----------------------------------------------------------------- LSQR -- */

typedef struct {
    int64_t m;                  /* rows of G */
    int32_t n;                  /* columns */
    const int64_t *rp;          /* G, CSR */
    const int32_t *ci;
    const double *va;
    const int64_t *cp;          /* G^T, CSR of the transpose */
    const int32_t *ri;
    const double *vt;
    int nx, ny, nz;
    double w;                   /* smoothing weight */
    const double *D;            /* NULL or column scaling */
    double lam_rows;            /* > 0: append lam*D rows (scaled problem) */
    double *tmp_n, *tmp_n2;     /* work vectors of length n */
    const double *P;            /* NULL or per-cell depth blocks: (nx*ny) x nz x nz, row-major */
} op_t;

/* out_h = P_h in_h for every cell h (depth-fastest column order), or with
 * transpose != 0 out_h = P_h^T in_h.  out and in must not overlap. */
static void blocks_apply(const double *P, int32_t n, int nz, int transpose, const double *in,
                         double *out)
{
    const int32_t H = n / nz;
    for (int32_t h = 0; h < H; ++h) {
        const double *Ph = P + (size_t)h * nz * nz;
        const double *x = in + (size_t)h * nz;
        double *y = out + (size_t)h * nz;
        for (int i = 0; i < nz; ++i) {
            double s = 0.0;
            for (int k = 0; k < nz; ++k)
                s += (transpose ? Ph[k * nz + i] : Ph[i * nz + k]) * x[k];
            y[i] = s;
        }
    }
}

static int64_t op_rows(const op_t *A)
{
    return A->m + A->n + (A->lam_rows > 0.0 ? A->n : 0);
}

/* y = A v, A = [G; w L] (times D or the block matrix P on the right, plus
 * lam D or lam P rows). */
static void op_apply(const op_t *A, const double *v, double *y)
{
    const double *vs = v;
    if (A->D) {
        for (int32_t j = 0; j < A->n; ++j)
            A->tmp_n[j] = A->D[j] * v[j];
        vs = A->tmp_n;
    } else if (A->P) {
        blocks_apply(A->P, A->n, A->nz, 0, v, A->tmp_n);
        vs = A->tmp_n;
    }
    oracle_spmv(A->m, A->rp, A->ci, A->va, vs, y);
    oracle_laplacian(A->nx, A->ny, A->nz, vs, y + A->m);
    for (int32_t j = 0; j < A->n; ++j)
        y[A->m + j] *= A->w;
    if (A->lam_rows > 0.0)
        for (int32_t j = 0; j < A->n; ++j)
            y[A->m + A->n + j] = A->lam_rows * vs[j];
}

/* z = A^T u.  L is symmetric, so L^T = L. */
static void op_apply_t(const op_t *A, const double *u, double *z)
{
    oracle_spmv(A->n, A->cp, A->ri, A->vt, u, z);
    oracle_laplacian(A->nx, A->ny, A->nz, u + A->m, A->tmp_n2);
    for (int32_t j = 0; j < A->n; ++j)
        z[j] += A->w * A->tmp_n2[j];
    if (A->lam_rows > 0.0)
        for (int32_t j = 0; j < A->n; ++j)
            z[j] += A->lam_rows * u[A->m + A->n + j];
    if (A->D)
        for (int32_t j = 0; j < A->n; ++j)
            z[j] *= A->D[j];
    else if (A->P) {
        memcpy(A->tmp_n2, z, sizeof(double) * (size_t)A->n);
        blocks_apply(A->P, A->n, A->nz, 1, A->tmp_n2, z);
    }
}

static double norm2(int64_t len, const double *x)
{
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i)
        s += x[i] * x[i];
    return sqrt(s);
}

static void scale(int64_t len, double a, double *x)
{
    for (int64_t i = 0; i < len; ++i)
        x[i] *= a;
}

/* Public operator products (used by tests for residual checks). */
void oracle_apply_A(int64_t m, int32_t n, const int64_t *rp, const int32_t *ci,
                    const double *va, int nx, int ny, int nz, double w, const double *D,
                    double lam_rows, const double *v, double *y, const double *P)
{
    op_t A = {m, n, rp, ci, va, NULL, NULL, NULL, nx, ny, nz, w, D, lam_rows, NULL, NULL, P};
    A.tmp_n = (double *)malloc(sizeof(double) * (size_t)n);
    op_apply(&A, v, y);
    free(A.tmp_n);
}

void oracle_apply_At(int64_t m, int32_t n, const int64_t *cp, const int32_t *ri,
                     const double *vt, int nx, int ny, int nz, double w, const double *D,
                     double lam_rows, const double *u, double *z, const double *P)
{
    op_t A = {m, n, NULL, NULL, NULL, cp, ri, vt, nx, ny, nz, w, D, lam_rows, NULL, NULL, P};
    A.tmp_n2 = (double *)malloc(sizeof(double) * (size_t)n);
    op_apply_t(&A, u, z);
    free(A.tmp_n2);
}

/*
 * LSQR, Paige & Saunders (1982): Golub-Kahan bidiagonalisation of A started
 * from b, with the lower bidiagonal system reduced by plane rotations, the
 * damping folded in by one extra rotation per step, the norm estimates of the
 * paper (||A||_F, cond(A), ||r||, ||A^T r||, ||x||) and its stopping rules:
 *   istop 1: ||r|| <= btol ||b|| + atol ||A|| ||x||      (rule S1)
 *   istop 2: ||A^T r|| / (||A|| ||r||) <= atol            (rule S2)
 *   istop 3: cond(A) >= conlim                            (rule S3)
 *   istop 4-6: the same three with the tolerances at machine precision
 *   istop 7: the iteration limit.
 * Here A is the operator of op_t and "||r||" includes the damping term.
 *
 * est[0..7] = itn, istop, rnorm, arnorm, anorm, acond, xnorm, bnorm.
 * If rec_k > 0, U (rec_k x op_rows) and V (rec_k x n) receive the first rec_k
 * normalised bidiagonalisation vectors u_2.. and v_2.. (u_1, v_1 first).
 * rhist (itmax) receives ||r|| after every iteration, if not NULL.
 */
int oracle_lsqr(int64_t m, int32_t n, const int64_t *rp, const int32_t *ci,
                const double *va, const int64_t *cp, const int32_t *ri, const double *vt,
                int nx, int ny, int nz, double w, const double *D, double lam_rows,
                double damp, const double *b, double atol, double btol, double conlim,
                int itmax, double *x, double *est, int rec_k, double *U, double *V,
                double *rhist, int n_ck, const double *ck_tol, double *ck_x,
                int32_t *ck_itn, const double *P)
{
    op_t A = {m, n, rp, ci, va, cp, ri, vt, nx, ny, nz, w, D, lam_rows, NULL, NULL, P};
    int64_t M = op_rows(&A);
    double *u = (double *)malloc(sizeof(double) * (size_t)M);
    double *Av = (double *)malloc(sizeof(double) * (size_t)M);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *Atu = (double *)malloc(sizeof(double) * (size_t)n);
    double *wv = (double *)malloc(sizeof(double) * (size_t)n);
    A.tmp_n = (double *)malloc(sizeof(double) * (size_t)n);
    A.tmp_n2 = (double *)malloc(sizeof(double) * (size_t)n);
    if (!u || !Av || !v || !Atu || !wv || !A.tmp_n || !A.tmp_n2)
        return -1;

    const double eps = DBL_EPSILON;
    double ctol = conlim > 0.0 ? 1.0 / conlim : 0.0;
    int itn = 0, istop = 0, nrec = 0;
    double anorm = 0.0, acond = 0.0, ddnorm = 0.0, res2 = 0.0;
    double xnorm = 0.0, xxnorm = 0.0, z = 0.0, cs2 = -1.0, sn2 = 0.0;
    double dampsq = damp * damp;

    for (int32_t j = 0; j < n; ++j)
        x[j] = 0.0;
    /* beta_1 u_1 = b (the augmented right-hand side [d; 0]) */
    for (int64_t i = 0; i < M; ++i)
        u[i] = i < m ? b[i] : 0.0;
    double beta = norm2(M, u), alpha = 0.0;
    double bnorm = beta;
    if (beta > 0.0) {
        scale(M, 1.0 / beta, u);
        op_apply_t(&A, u, v);
        alpha = norm2(n, v);
    } else {
        for (int32_t j = 0; j < n; ++j)
            v[j] = 0.0;
    }
    if (alpha > 0.0)
        scale(n, 1.0 / alpha, v);
    if (rec_k > 0) {
        memcpy(U, u, sizeof(double) * (size_t)M);
        memcpy(V, v, sizeof(double) * (size_t)n);
        nrec = 1;
    }
    memcpy(wv, v, sizeof(double) * (size_t)n);
    double rhobar = alpha, phibar = beta, rnorm = beta, arnorm = alpha * beta;

    if (arnorm > 0.0) {
        while (itn < itmax) {
            ++itn;
            /* beta u = A v - alpha u ; alpha v = A^T u - beta v */
            op_apply(&A, v, Av);
            for (int64_t i = 0; i < M; ++i)
                u[i] = Av[i] - alpha * u[i];
            beta = norm2(M, u);
            if (beta > 0.0) {
                scale(M, 1.0 / beta, u);
                anorm = sqrt(anorm * anorm + alpha * alpha + beta * beta + dampsq);
                op_apply_t(&A, u, Atu);
                for (int32_t j = 0; j < n; ++j)
                    v[j] = Atu[j] - beta * v[j];
                alpha = norm2(n, v);
                if (alpha > 0.0)
                    scale(n, 1.0 / alpha, v);
            }
            if (rec_k > nrec) {
                memcpy(U + (size_t)nrec * M, u, sizeof(double) * (size_t)M);
                memcpy(V + (size_t)nrec * n, v, sizeof(double) * (size_t)n);
                ++nrec;
            }
            /* rotation that eliminates the damping row */
            double rhobar1 = rhobar, psi = 0.0;
            if (damp > 0.0) {
                rhobar1 = sqrt(rhobar * rhobar + dampsq);
                double cs1 = rhobar / rhobar1, sn1 = damp / rhobar1;
                psi = sn1 * phibar;
                phibar = cs1 * phibar;
            }
            /* rotation that eliminates beta from the lower bidiagonal */
            double rho = sqrt(rhobar1 * rhobar1 + beta * beta);
            double cs = rhobar1 / rho, sn = beta / rho;
            double theta = sn * alpha;
            rhobar = -cs * alpha;
            double phi = cs * phibar;
            phibar = sn * phibar;
            double tau = sn * phi;

            /* x and w updates; ||w_k||^2 / rho_k^2 feeds the cond(A) estimate */
            double t1 = phi / rho, t2 = -theta / rho;
            double wn2 = 0.0;
            for (int32_t j = 0; j < n; ++j)
                wn2 += wv[j] * wv[j];
            ddnorm += wn2 / (rho * rho);
            for (int32_t j = 0; j < n; ++j) {
                x[j] = x[j] + t1 * wv[j];
                wv[j] = v[j] + t2 * wv[j];
            }

            /* ||x|| estimate from the LQ factors of the upper bidiagonal R_k */
            double delta = sn2 * rho;
            double gambar = -cs2 * rho;
            double rhs = phi - delta * z;
            double zbar = rhs / gambar;
            xnorm = sqrt(xxnorm + zbar * zbar);
            double gamma = sqrt(gambar * gambar + theta * theta);
            cs2 = gambar / gamma;
            sn2 = theta / gamma;
            z = rhs / gamma;
            xxnorm = xxnorm + z * z;

            acond = anorm * sqrt(ddnorm);
            res2 = res2 + psi * psi;
            rnorm = sqrt(phibar * phibar + res2);
            arnorm = alpha * fabs(tau);
            if (rhist)
                rhist[itn - 1] = rnorm;

            double test1 = rnorm / bnorm;
            double test2 = arnorm / (anorm * rnorm + eps);
            double test3 = 1.0 / (acond + eps);
            double t1s = test1 / (1.0 + anorm * xnorm / bnorm);
            double rtol = btol + atol * anorm * xnorm / bnorm;
            /* checkpoints (output only): the iterate at which a solve with
             * atol = btol = ck_tol[c] would stop on S1 or S2 -- the iteration
             * does not depend on the tolerances, so that solve's answer */
            for (int c = 0; c < n_ck; ++c) {
                if (ck_itn[c] > 0)
                    continue;
                double tc = ck_tol[c];
                if (test1 <= tc + tc * anorm * xnorm / bnorm || test2 <= tc) {
                    ck_itn[c] = itn;
                    memcpy(ck_x + (size_t)c * n, x, sizeof(double) * (size_t)n);
                }
            }
            if (test1 <= rtol) istop = 1;
            else if (test2 <= atol) istop = 2;
            else if (test3 <= ctol) istop = 3;
            else if (1.0 + t1s <= 1.0) istop = 4;
            else if (1.0 + test2 <= 1.0) istop = 5;
            else if (1.0 + test3 <= 1.0) istop = 6;
            else if (itn >= itmax) istop = 7;
            if (istop != 0)
                break;
        }
    }
    est[0] = itn;
    est[1] = istop;
    est[2] = rnorm;
    est[3] = arnorm;
    est[4] = anorm;
    est[5] = acond;
    est[6] = xnorm;
    est[7] = bnorm;
    free(u);
    free(Av);
    free(v);
    free(Atu);
    free(wv);
    free(A.tmp_n);
    free(A.tmp_n2);
    return 0;
}

int oracle_num_threads(void)
{
    int t = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
#endif
    return t;
}
