// lsqr_dev.cuh -- device helpers shared by the single-system and batched
// LSQR kernels: vector loads, the 7-point Laplacian and the FP64 scalar
// recurrence of LSQR (Paige & Saunders 1982).
#pragma once

#include <cfloat>

#include "common.cuh"
#include "dfloat.cuh"

namespace pdst {

constexpr unsigned FULL = 0xffffffffu;

// Unroll depth of the streaming loops: enough independent 16-byte loads per
// lane to cover HBM latency at 32 resident warps per SM.
template <class AT> struct Unroll { static constexpr int U = 4; };
template <> struct Unroll<double> { static constexpr int U = 2; };
template <> struct Unroll<dfl> { static constexpr int U = 2; };


// ------------------------------------------------------------ load helpers

template <class VT> struct Pack4;
template <> struct Pack4<float> {
    static __device__ __forceinline__ void ld(const float *p, float v[4]) {
        float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct Pack4<double> {
    static __device__ __forceinline__ void ld(const double *p, double v[4]) {
        double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
        double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct Pack4<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float v[4]) {
        uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xffff0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
};
template <> struct Pack4<dfl> {
    static __device__ __forceinline__ void ld(const dfl *p, dfl v[4]) {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = dfl(a.x, a.y); v[1] = dfl(a.z, a.w); v[2] = dfl(b.x, b.y); v[3] = dfl(b.z, b.w);
    }
};

// Two consecutive values (any even nz): 8-byte loads for FP32, 16 for FP64 and
// double-float, 4 for BF16; streamed (evict-first) like the quads.
template <class VT> struct Pack2;
template <> struct Pack2<float> {
    static __device__ __forceinline__ void ld(const float *p, float v[2]) {
        const float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct Pack2<double> {
    static __device__ __forceinline__ void ld(const double *p, double v[2]) {
        const double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct Pack2<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float v[2]) {
        const unsigned t = __ldcs(reinterpret_cast<const unsigned *>(p));
        v[0] = __uint_as_float(t << 16);
        v[1] = __uint_as_float(t & 0xffff0000u);
    }
};
template <> struct Pack2<dfl> {
    static __device__ __forceinline__ void ld(const dfl *p, dfl v[2]) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = dfl(t.x, t.y); v[1] = dfl(t.z, t.w);
    }
};

template <class VT> struct Wide { using T = VT; };
template <> struct Wide<__nv_bfloat16> { using T = float; };

template <class ST> __device__ __forceinline__ void ldx4(const ST *p, ST v[4]);
template <> __device__ __forceinline__ void ldx4<float>(const float *p, float v[4]) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <> __device__ __forceinline__ void ldx4<double>(const double *p, double v[4]) {
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <> __device__ __forceinline__ void ldx4<dfl>(const dfl *p, dfl v[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = dfl(a.x, a.y); v[1] = dfl(a.z, a.w); v[2] = dfl(b.x, b.y); v[3] = dfl(b.z, b.w);
}

template <class ST> __device__ __forceinline__ void ldx2(const ST *p, ST v[2]);
template <> __device__ __forceinline__ void ldx2<float>(const float *p, float v[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = t.x; v[1] = t.y;
}
template <> __device__ __forceinline__ void ldx2<double>(const double *p, double v[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = t.x; v[1] = t.y;
}
template <> __device__ __forceinline__ void ldx2<dfl>(const dfl *p, dfl v[2]) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = dfl(t.x, t.y); v[1] = dfl(t.z, t.w);
}

__device__ __forceinline__ float ldval(const float *p) { return __ldcs(p); }
__device__ __forceinline__ dfl ldval(const dfl *p) { return __ldcs(p); }
__device__ __forceinline__ double ldval(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ldval(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}

// (L x)_j = sum over existing 7-point neighbours i of (x_j - x_i).
template <class AT, class XT>
__device__ __forceinline__ AT laplace(const XT *__restrict__ x, int64_t j, int nx, int ny, int nz) {
    const int k = (int)(j % nz);
    const int64_t hh = j / nz;
    const int ix = (int)(hh % nx), iy = (int)(hh / nx);
    const int64_t sy = (int64_t)nx * nz;
    const AT c = (AT)x[j];
    AT s = 0;
    if (k > 0) s += c - (AT)x[j - 1];
    if (k < nz - 1) s += c - (AT)x[j + 1];
    if (ix > 0) s += c - (AT)x[j - nz];
    if (ix < nx - 1) s += c - (AT)x[j + nz];
    if (iy > 0) s += c - (AT)x[j - sy];
    if (iy < ny - 1) s += c - (AT)x[j + sy];
    return s;
}


__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Bulk prefetch of the bytes [p, p + bytes) into L2 by the copy engine
// (cp.async.bulk.prefetch.L2: a hint, nothing to wait for).  The range is
// shrunk to 16-byte boundaries, so it never leaves [p, p + bytes).  One
// thread issues it; the warp's later loads of the range then hit L2.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint64_t bytes) {
    const uint64_t a = (uint64_t)__cvta_generic_to_global(p);
    const uint64_t s = (a + 15u) & ~(uint64_t)15u, e = (a + bytes) & ~(uint64_t)15u;
    if (e > s) {
        const uint64_t n = e - s < ((uint64_t)1 << 30) ? e - s : ((uint64_t)1 << 30);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)n)
                     : "memory");
    }
}

// Paige & Saunders' stopping tests S1-S3 and their machine-precision forms
// on the current estimates (istop 1-6), itmax (7); SciPy's numbering.
static __device__ void stop_tests(LsqrScalars *sc) {
    const double eps = DBL_EPSILON;
    const double bnorm = sc->bnorm, anorm = sc->anorm, xnorm = sc->xnorm, rnorm = sc->rnorm;
    const double test1 = rnorm / bnorm;
    const double test2 = sc->arnorm / (anorm * rnorm + eps);
    const double test3 = 1.0 / (sc->acond + eps);
    const double t1s = test1 / (1.0 + anorm * xnorm / bnorm);
    const double rtol = sc->btol + sc->atol * anorm * xnorm / bnorm;
    int istop = 0;
    if (test1 <= rtol) istop = 1;
    else if (test2 <= sc->atol) istop = 2;
    else if (test3 <= sc->ctol) istop = 3;
    else if (1.0 + t1s <= 1.0) istop = 4;
    else if (1.0 + test2 <= 1.0) istop = 5;
    else if (1.0 + test3 <= 1.0) istop = 6;
    else if (sc->itn >= sc->itmax) istop = 7;
    sc->istop = istop;
    if (!isfinite(rnorm) || !isfinite(sc->arnorm)) {
        sc->err = 1;
        sc->done = 1;
    }
}

// One LSQR step of the scalar recurrence (Paige & Saunders 1982): damping
// rotation, plane rotation, x/w update coefficients, norm estimates and
// stopping rules.  alpha_new = ||v-bar_{i+1}||, sc->beta = beta_{i+1},
// sc->alpha = alpha_i, sc->wnorm2 = ||w_i||^2.
static __device__ void lsqr_step(LsqrScalars *sc, double alpha_new) {
    const double alpha = sc->alpha, beta = sc->beta, damp = sc->damp;
    const double dampsq = damp * damp;
    if (beta > 0.0)
        sc->anorm = sqrt(sc->anorm * sc->anorm + alpha * alpha + beta * beta + dampsq);
    else
        alpha_new = alpha;
    double rhobar = sc->rhobar, phibar = sc->phibar, rhobar1 = rhobar, psi = 0.0;
    if (damp > 0.0) {
        rhobar1 = sqrt(rhobar * rhobar + dampsq);
        const double cs1 = rhobar / rhobar1, sn1 = damp / rhobar1;
        psi = sn1 * phibar;
        phibar = cs1 * phibar;
    }
    const double rho = sqrt(rhobar1 * rhobar1 + beta * beta);
    if (!(rho > 0.0) || !isfinite(rho)) {
        sc->err = 1;
        sc->done = 1;
        return;
    }
    const double cs = rhobar1 / rho, sn = beta / rho;
    const double theta = sn * alpha_new;
    sc->rhobar = -cs * alpha_new;
    const double phi = cs * phibar;
    phibar = sn * phibar;
    sc->phibar = phibar;
    const double tau = sn * phi;
    sc->t1 = phi / rho;
    sc->t2 = -theta / rho;
    sc->ddnorm += sc->wnorm2 / (rho * rho);
    // ||x|| estimate from the LQ factors of the upper bidiagonal R_k
    const double delta = sc->sn2 * rho, gambar = -sc->cs2 * rho;
    const double rhs = phi - delta * sc->z;
    const double zbar = rhs / gambar;
    sc->xnorm = sqrt(sc->xxnorm + zbar * zbar);
    const double gamma = sqrt(gambar * gambar + theta * theta);
    sc->cs2 = gambar / gamma;
    sc->sn2 = theta / gamma;
    sc->z = rhs / gamma;
    sc->xxnorm += sc->z * sc->z;
    sc->acond = sc->anorm * sqrt(sc->ddnorm);
    sc->res2 += psi * psi;
    sc->rnorm = sqrt(phibar * phibar + sc->res2);
    sc->arnorm = alpha_new * fabs(tau);
    sc->alpha = alpha_new;
    sc->itn += 1;
    sc->pending = 1;
    if (sc->hist) sc->hist[sc->itn - 1] = sc->rnorm;
    stop_tests(sc);
    if (!isfinite(sc->t1) || !isfinite(sc->t2)) {
        sc->err = 1;
        sc->done = 1;
    }
}

// Givens rotation (c, s, r) of (a, b): r = sqrt(a^2 + b^2) >= 0.
static __device__ __forceinline__ void givens(double a, double b, double &c, double &s,
                                              double &r) {
    r = hypot(a, b);
    if (r == 0.0) {
        c = 1.0;
        s = 0.0;
    } else {
        c = a / r;
        s = b / r;
    }
}

// LSMR state after the start step (beta_1 u_1 = b, alpha_1 v_1 = A^T u_1).
static __device__ void lsmr_init(LsqrScalars *sc, double alpha1) {
    const double beta1 = sc->beta;
    sc->alphabar = alpha1;
    sc->zetabar = alpha1 * beta1;
    sc->cbar = 1.0;
    sc->sbar = 0.0;
    sc->rho_prev = 1.0;
    sc->rhobar_prev = 1.0;
    sc->betadd = beta1;
    sc->betad = 0.0;
    sc->rhod_prev = 1.0;
    sc->tautilde_prev = 0.0;
    sc->thetatilde = 0.0;
    sc->zeta_prev = 0.0;
    sc->dsum = 0.0;
    sc->anorm2 = alpha1 * alpha1;
    sc->rbar_max = 0.0;
    sc->rbar_min = DBL_MAX;
}

// One LSMR step (Fong & Saunders 2011) after the bidiagonalisation produced
// beta_{k+1} (sc->beta) and alpha_{k+1} (alpha_new): the damping rotation,
// the rotations P_k and Pbar_k, the coefficients of the vector update
//   hbar = h - t1 hbar,  x += t2 hbar,  h = v - t3 h,
// and the estimates: ||A^T r|| = |zetabar_{k+1}|; ||r|| through the rotation
// Qtilde_{k-1} of (rhodot_{k-1}, thetabar_k) applied to betahat and to R_k y_k
// (||r||^2 = d + (betadot - taudot)^2 + betadotdot^2, d summing what the
// damping rotations split off); ||A|| ~ ||B_k||_F; cond(A) ~ max/min rhobar_j.
// The stopping tests need ||x_k||, so they run after the update (k_upd).
static __device__ void lsmr_step(LsqrScalars *sc, double alpha_new) {
    const double beta = sc->beta, lam = sc->damp;
    if (!(beta > 0.0)) alpha_new = sc->alpha;
    double chat, shat, alphahat;
    givens(sc->alphabar, lam, chat, shat, alphahat);
    double c, s, rho;
    givens(alphahat, beta, c, s, rho);
    if (!(rho > 0.0) || !isfinite(rho)) {
        sc->err = 1;
        sc->done = 1;
        return;
    }
    const double theta_next = s * alpha_new;
    sc->alphabar = c * alpha_new;
    const double thetabar = sc->sbar * rho;
    double cbar, sbar, rhobar;
    givens(sc->cbar * rho, theta_next, cbar, sbar, rhobar);
    const double zeta = cbar * sc->zetabar;
    sc->zetabar = -sbar * sc->zetabar;
    sc->cbar = cbar;
    sc->sbar = sbar;
    sc->t1 = thetabar * rho / (sc->rho_prev * sc->rhobar_prev);
    sc->t2 = zeta / (rho * rhobar);
    sc->t3 = theta_next / rho;
    // ||r_k||
    const double betaacute = chat * sc->betadd, betacheck = -shat * sc->betadd;
    const double betahat = c * betaacute;
    sc->betadd = -s * betaacute;
    const double thetatilde_prev = sc->thetatilde;
    double ctilde, stilde, rhotilde_prev;
    givens(sc->rhod_prev, thetabar, ctilde, stilde, rhotilde_prev);
    sc->thetatilde = stilde * rhobar;
    sc->rhod_prev = ctilde * rhobar;
    sc->betad = -stilde * sc->betad + ctilde * betahat;
    sc->tautilde_prev = (sc->zeta_prev - thetatilde_prev * sc->tautilde_prev) / rhotilde_prev;
    const double taud = (zeta - sc->thetatilde * sc->tautilde_prev) / sc->rhod_prev;
    sc->dsum += betacheck * betacheck;
    const double dr = sc->betad - taud;
    sc->rnorm = sqrt(sc->dsum + dr * dr + sc->betadd * sc->betadd);
    // ||A||, cond(A), ||A^T r||
    sc->anorm2 += beta * beta;
    sc->anorm = sqrt(sc->anorm2);
    sc->anorm2 += alpha_new * alpha_new;
    sc->rbar_max = fmax(sc->rbar_max, rhobar);
    sc->rbar_min = fmin(sc->rbar_min, rhobar);
    sc->acond = sc->rbar_max / sc->rbar_min;
    sc->arnorm = fabs(sc->zetabar);
    sc->rho_prev = rho;
    sc->rhobar_prev = rhobar;
    sc->zeta_prev = zeta;
    sc->alpha = alpha_new;
    sc->itn += 1;
    sc->pending = 1;
    if (sc->hist) sc->hist[sc->itn - 1] = sc->rnorm;
    if (!isfinite(sc->rnorm) || !isfinite(sc->arnorm) || !isfinite(sc->t1) ||
        !isfinite(sc->t2) || !isfinite(sc->t3)) {
        sc->err = 1;
        sc->done = 1;
    }
}

}  // namespace pdst
