"""FP64 oracle of the outer nonlinear loop of the inversion.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): called by the tests and
never by the product.

What it computes (the paragraph after Eq. 6 of the paper: solve Eq. 6 for the
model perturbation, update the model, rebuild the sensitivity matrix from the
updated model, repeat until the RMS traveltime error is below a threshold),
with the synthetic stand-in of this build for the sensitivity-kernel module:

* the depth kernel under horizontal cell h at period T follows that cell's
  1-D model: with s_h = (1/nz) sum_k (1 + m[h*nz + k]) (the mean relative
  S-wave velocity of the column, summed in depth order),
      z0(h, T) = z0_factor * T * s_h^a      (a = kernel_power: 1 the kernel
                                             follows the model, 0 it does not),
      K[h][t][k] = (z_k / z0) * exp(1 - z_k / z0) * dz,   z_k = (k + 1/2) dz,
  so a faster column is sampled deeper (the kernel scales with wavelength);
  at m = 0 this is the 1-D table of Eq. 5's synthetic form;
* the predicted traveltime perturbation is F(m) = G(m) m and the data
  residual of Eq. 6 is r = d_obs - F(m); RMS = sqrt(mean(r^2));
* each outer iteration solves Eq. 6 for the update,
      dm = argmin ||G(m) dm - r||^2 + w^2 ||L dm||^2 + lambda^2 ||dm||^2
  (LSQR, Paige & Saunders 1982, oracle.lsqr), and sets m <- m + dm.

Stopping (checked before each solve, on the residual of the current model):
reason 1 RMS <= rms_tol; reason 2 the RMS fell by less than the fraction
min_decrease since the previous model (the loop keeps the model with the
smaller RMS); reason 3 max_outer updates made.

Parity status: pinned in tests/test_oracle_outer.py (the kernel table's depth
integral against its closed form z0 e, its m = 0 case against the 1-D table,
the loop on a model-independent kernel against iterated Tikhonov in closed
form on a dense system, and recovery of a planted model).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import build_G, lsqr, spmv, transpose


def kernel_table(periods_s, nx: int, ny: int, nz: int, dz: float, m: np.ndarray,
                 z0_factor: float = 1.2, kernel_power: float = 1.0) -> np.ndarray:
    """K[h][t][k] (nx*ny, T, nz) from the model m (column order h*nz + k)."""
    H = nx * ny
    M = np.asarray(m, dtype=np.float64).reshape(H, nz)
    s = np.zeros(H)
    for k in range(nz):
        s = s + (1.0 + M[:, k])
    s = s / nz
    if kernel_power != 1.0:
        s = s ** kernel_power
    T = np.asarray(periods_s, dtype=np.float64)
    z0 = (z0_factor * T)[None, :] * s[:, None]                 # (H, T)
    z = (np.arange(nz, dtype=np.float64) + 0.5) * dz           # (nz,)
    q = z[None, None, :] / z0[:, :, None]
    return q * np.exp(1.0 - q) * dz


def G_of_model(p, m, z0_factor: float = 1.2, kernel_power: float = 1.0):
    kc = kernel_table(p.periods_s, p.nx, p.ny, p.nz, p.dz_km, m, z0_factor, kernel_power)
    return build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period, p.kdz, kdz_cells=kc,
                   interp=getattr(p, "interp", 0))


def forward(p, m, z0_factor: float = 1.2, kernel_power: float = 1.0) -> np.ndarray:
    """F(m) = G(m) m."""
    return spmv(G_of_model(p, m, z0_factor, kernel_power), m)


@dataclass
class OuterResult:
    m: np.ndarray
    rms: List[float] = field(default_factory=list)   # RMS before each solve, and at the end
    reason: int = 0
    updates: int = 0                                  # models updated (solves applied)
    inner_iters: List[int] = field(default_factory=list)


def outer_loop(p, d_obs, w: float, lam: float, itmax: int, tol: float, max_outer: int,
               rms_tol: float, min_decrease: float, z0_factor: float = 1.2,
               kernel_power: float = 1.0) -> OuterResult:
    n = p.n
    grid = (p.nx, p.ny, p.nz)
    m = np.zeros(n)
    res = OuterResult(m=m)
    prev_m = None
    while True:
        G = G_of_model(p, m, z0_factor, kernel_power)
        r = np.asarray(d_obs, dtype=np.float64) - spmv(G, m)
        rms = float(np.sqrt(np.mean(r * r)))
        res.rms.append(rms)
        if rms <= rms_tol:
            res.reason = 1
            break
        if len(res.rms) > 1 and rms > (1.0 - min_decrease) * res.rms[-2]:
            res.reason = 2
            if rms > res.rms[-2]:
                m = prev_m          # keep the model with the smaller misfit
            break
        if res.updates == max_outer:
            res.reason = 3
            break
        sol = lsqr(G, transpose(G), grid, w, lam, r, atol=tol, btol=tol, itmax=itmax)
        res.inner_iters.append(sol.itn)
        prev_m = m
        m = m + sol.x
        res.updates += 1
    res.m = m
    return res
