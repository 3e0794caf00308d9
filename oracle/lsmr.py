"""LSMR oracle (Fong & Saunders 2011) -- TEST INFRASTRUCTURE ONLY.

Called by the tests and the smoke check, never by the product path; it shares
no code with the CUDA library.  LSMR is the solver pDSurfTomo actually uses
for the linearised traveltime system (its least-squares module names LSMR and
LSQR as the two mainstream Krylov solvers; DSurfTomo, SciPy and CuPy all run
LSMR).  Like LSQR it is built on the Golub-Kahan bidiagonalisation of
A = [G; w L] (or [G D; w L D; lam D] with a right scaling), but it minimises
||A^T r_k|| over the Krylov space instead of ||r_k||.

The iteration follows the algorithm of Fong & Saunders (SIAM J. Sci. Comput.
33, 2011), in its order and notation, FP64, one iteration per loop pass:

  init   beta_1 u_1 = b, alpha_1 v_1 = A^T u_1, alphabar_1 = alpha_1,
         zetabar_1 = alpha_1 beta_1, rho_0 = rhobar_0 = cbar_0 = 1, sbar_0 = 0,
         h_1 = v_1, hbar_0 = 0, x_0 = 0
  step k bidiagonalisation: beta_{k+1} u_{k+1} = A v_k - alpha_k u_k,
                            alpha_{k+1} v_{k+1} = A^T u_{k+1} - beta_{k+1} v_k
         damping rotation:  alphahat_k = |(alphabar_k, lam)|,
                            chat = alphabar_k / alphahat_k, shat = lam / alphahat_k
         rotation P_k:      rho_k = |(alphahat_k, beta_{k+1})|, c_k = alphahat_k / rho_k,
                            s_k = beta_{k+1} / rho_k, theta_{k+1} = s_k alpha_{k+1},
                            alphabar_{k+1} = c_k alpha_{k+1}
         rotation Pbar_k:   thetabar_k = sbar_{k-1} rho_k,
                            rhobar_k = |(cbar_{k-1} rho_k, theta_{k+1})|,
                            cbar_k = cbar_{k-1} rho_k / rhobar_k,
                            sbar_k = theta_{k+1} / rhobar_k,
                            zeta_k = cbar_k zetabar_k, zetabar_{k+1} = -sbar_k zetabar_k
         updates:           hbar_k = h_k - (thetabar_k rho_k / (rho_{k-1} rhobar_{k-1})) hbar_{k-1}
                            x_k = x_{k-1} + (zeta_k / (rho_k rhobar_k)) hbar_k
                            h_{k+1} = v_{k+1} - (theta_{k+1} / rho_k) h_k

Estimates (section 3 of the paper):
  ||A^T r_k|| = |zetabar_{k+1}|;
  ||r_k||: the rotations P_k (and the damping rotation) applied to beta_1 e_1
  give betahat_k and betadotdot_{k+1}; a third rotation Qtilde_{k-1} built
  from (rhodot_{k-1}, thetabar_k) carries betahat into betadot_k and
  R_k y_k into taudot_k, so that
      ||r_k||^2 = d_k + (betadot_k - taudot_k)^2 + betadotdot_{k+1}^2,
  d_k summing the squares the damping rotations split off;
  ||A|| ~ ||B_k||_F (alpha_1^2 + sum of beta_{j+1}^2 + alpha_{j+1}^2);
  cond(A) ~ max / min of rhobar_j over the steps;
  ||x_k|| from x_k itself.
Stopping tests as in LSQR (S1, S2, S3 and their machine-precision forms,
istop numbering 1-7 as in SciPy).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import CSR, apply_A, apply_At


@dataclass
class LSMRResult:
    x: np.ndarray
    itn: int
    istop: int
    rnorm: float
    arnorm: float
    anorm: float
    acond: float
    xnorm: float
    bnorm: float
    arhist: Optional[np.ndarray] = None


def _rot(a: float, b: float):
    """Givens rotation (c, s, r) with r = sqrt(a^2 + b^2) >= 0."""
    r = float(np.hypot(a, b))
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def lsmr(G: CSR, GT: CSR, grid, w: float, damp: float, b: np.ndarray,
         atol: float = 1e-8, btol: float = 1e-8, conlim: float = 1e8, itmax: int = 300,
         D: Optional[np.ndarray] = None, lam_rows: float = 0.0,
         history: bool = False) -> LSMRResult:
    """LSMR on [G; w L] with damping `damp` (or on [G D; w L D; lam_rows D])."""
    m, n = G.n_rows, G.n_cols
    M = m + n + (n if lam_rows > 0 else 0)
    b = np.asarray(b, dtype=np.float64)
    bfull = np.zeros(M)
    bfull[: b.shape[0]] = b

    def A(v):
        return apply_A(G, grid, w, v, D=D, lam_rows=lam_rows)

    def At(u):
        return apply_At(GT, grid, w, u, D=D, lam_rows=lam_rows)

    lam = float(damp)
    x = np.zeros(n)
    beta = float(np.linalg.norm(bfull))
    bnorm = beta
    hist = [] if history else None
    if beta == 0.0:
        return LSMRResult(x, 0, 0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, np.array([]) if history else None)
    u = bfull / beta
    v = At(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LSMRResult(x, 0, 0, beta, 0.0, 0.0, 0.0, 0.0, bnorm,
                          np.array([]) if history else None)
    v = v / alpha

    # rotations and recurrences
    alphabar, zetabar = alpha, alpha * beta
    rho_prev, rhobar_prev, cbar, sbar = 1.0, 1.0, 1.0, 0.0
    h, hbar = v.copy(), np.zeros(n)
    # ||r|| estimate state
    betadd, betad, rhod_prev = beta, 0.0, 1.0
    tautilde_prev, thetatilde, zeta_prev, dsum = 0.0, 0.0, 0.0, 0.0
    # ||A||, cond(A)
    anorm2 = alpha * alpha
    rbar_max, rbar_min = 0.0, np.inf
    ctol = 1.0 / conlim if conlim > 0 else 0.0
    eps = np.finfo(np.float64).eps
    itn, istop = 0, 0
    rnorm, arnorm, anorm, acond, xnorm = beta, alpha * beta, alpha, 0.0, 0.0

    while itn < itmax:
        itn += 1
        # bidiagonalisation
        u = A(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
            v = At(u) - beta * v
            alpha = float(np.linalg.norm(v))
            if alpha > 0.0:
                v = v / alpha
        # damping rotation
        chat, shat, alphahat = _rot(alphabar, lam)
        # rotation P_k
        c, s, rho = _rot(alphahat, beta)
        theta_next = s * alpha
        alphabar = c * alpha
        # rotation Pbar_k
        thetabar = sbar * rho
        cbar, sbar, rhobar = _rot(cbar * rho, theta_next)
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar
        # h-bar, x, h
        hbar = h - (thetabar * rho / (rho_prev * rhobar_prev)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta_next / rho) * h
        # ||r||: damping rotation and P_k on beta_1 e_1, then Qtilde_{k-1}
        betaacute = chat * betadd
        betacheck = -shat * betadd
        betahat = c * betaacute
        betadd = -s * betaacute
        thetatilde_prev = thetatilde
        ctilde, stilde, rhotilde_prev = _rot(rhod_prev, thetabar)
        thetatilde = stilde * rhobar
        rhod_prev = ctilde * rhobar
        betad = -stilde * betad + ctilde * betahat
        tautilde_prev = (zeta_prev - thetatilde_prev * tautilde_prev) / rhotilde_prev
        taud = (zeta - thetatilde * tautilde_prev) / rhod_prev
        dsum += betacheck * betacheck
        rnorm = float(np.sqrt(dsum + (betad - taud) ** 2 + betadd * betadd))
        # ||A||, cond(A), ||A^T r||, ||x||
        anorm2 += beta * beta
        anorm = float(np.sqrt(anorm2))
        anorm2 += alpha * alpha
        rbar_max = max(rbar_max, rhobar)
        rbar_min = min(rbar_min, rhobar)
        acond = rbar_max / rbar_min
        arnorm = abs(zetabar)
        xnorm = float(np.linalg.norm(x))
        rho_prev, rhobar_prev, zeta_prev = rho, rhobar, zeta
        if history:
            hist.append(arnorm)
        # stopping tests (LSQR's, on these estimates)
        test1 = rnorm / bnorm
        test2 = arnorm / (anorm * rnorm + eps)
        test3 = 1.0 / (acond + eps)
        t1 = test1 / (1.0 + anorm * xnorm / bnorm)
        rtol = btol + atol * anorm * xnorm / bnorm
        if test1 <= rtol:
            istop = 1
        elif test2 <= atol:
            istop = 2
        elif test3 <= ctol:
            istop = 3
        elif 1.0 + t1 <= 1.0:
            istop = 4
        elif 1.0 + test2 <= 1.0:
            istop = 5
        elif 1.0 + test3 <= 1.0:
            istop = 6
        elif itn >= itmax:
            istop = 7
        if istop:
            break
    return LSMRResult(x=x, itn=itn, istop=istop, rnorm=rnorm, arnorm=arnorm, anorm=anorm,
                      acond=acond, xnorm=xnorm, bnorm=bnorm,
                      arhist=np.array(hist) if history else None)
