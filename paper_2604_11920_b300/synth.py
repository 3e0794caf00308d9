"""Seeded synthetic inputs for the regularised traveltime least-squares solve.

This module produces the *inputs* of the solve and nothing else: station
positions, the (station pair, period) ray geometry, the period depth-kernel
table, planted velocity models and unit Gaussian noise.  It holds none of the
method's arithmetic (no path sampling, no sensitivity matrix, no LSQR); both
the CUDA library and the FP64 oracle consume what it returns.

Conventions (the paper's Eq. 5-7 ordering, with the readings listed below):

* grid nx x ny x nz, horizontal cell size dx_km, layer thickness dz_km;
* model column index j = (iy*nx + ix)*nz + k (depth fastest, Eq. 7);
* data row index r = p*T + t (pair major, period minor); pairs are all
  i < j station pairs in lexicographic order;
* a ray is a quadratic Bezier curve with control points P0 (station i),
  P1 and P2 (station j).  A straight ray has P1 at the midpoint; a bent ray
  (rays are traced per period, Sec. "Parallelization in TravelTime
  Computation") moves P1 perpendicular to the chord by U(-b, b) x length;
* depth kernel K_T(z) = (z/z0) exp(1 - z/z0), z0 = 1.2 T km, evaluated at
  layer centres z_k = (k + 1/2) dz and multiplied by dz.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One synthetic tomography system (inputs only)."""

    name: str
    nx: int
    ny: int
    nz: int
    dx_km: float
    dz_km: float
    stations: np.ndarray        # (S, 2) float64, km
    pairs: np.ndarray           # (P, 2) int32, station indices i < j
    periods_s: np.ndarray       # (T,) float64
    ctrl: np.ndarray            # (mG, 6) float64: P0x P0y P1x P1y P2x P2y per row
    row_period: np.ndarray      # (mG,) int32 period index of each row
    kdz: np.ndarray             # (T, nz) float64, K_T(z_k) * dz
    w: float                    # smoothing weight
    lam: float                  # damping
    tol: float                  # atol = btol
    itmax: int
    model_kind: str
    noise_frac: float
    seed: int
    m_true: Optional[np.ndarray] = None   # (n,) planted model
    noise: Optional[np.ndarray] = None    # (mG,) unit normal draws
    kdz_cells: Optional[np.ndarray] = None  # (nx*ny, T, nz): per-cell kernels (lateral case)
    interp: int = 0                       # 0: cell lengths; 1: bilinear node coefficients (Eq. 1)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def m_rows(self) -> int:
        return int(self.ctrl.shape[0])

    @property
    def n_periods(self) -> int:
        return int(self.periods_s.shape[0])


# ---------------------------------------------------------------- geometry

def station_positions(rng: np.random.Generator, n_st: int, nx: int, ny: int,
                      dx: float) -> np.ndarray:
    """Stations uniform in the model square [0, nx*dx) x [0, ny*dx)."""
    st = np.empty((n_st, 2), dtype=np.float64)
    st[:, 0] = rng.uniform(0.0, nx * dx, n_st)
    st[:, 1] = rng.uniform(0.0, ny * dx, n_st)
    return st


def station_pairs(n_st: int) -> np.ndarray:
    """All i < j pairs in lexicographic order."""
    ii, jj = np.triu_indices(n_st, k=1)
    return np.stack([ii, jj], axis=1).astype(np.int32)


def ray_controls(rng: np.random.Generator, stations: np.ndarray,
                 pairs: np.ndarray, n_periods: int,
                 bend: float) -> np.ndarray:
    """Quadratic-Bezier control points per (pair, period) row.

    bend = 0 gives straight rays (P1 at the chord midpoint).  Otherwise the
    control point is displaced perpendicular to the chord by
    U(-bend, bend) x chord length, drawn independently per row.
    """
    P = pairs.shape[0]
    p0 = stations[pairs[:, 0]]
    p2 = stations[pairs[:, 1]]
    mid = 0.5 * (p0 + p2)
    d = p2 - p0
    length = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    perp = np.zeros_like(d)
    ok = length > 0
    perp[ok, 0] = -d[ok, 1] / length[ok]
    perp[ok, 1] = d[ok, 0] / length[ok]
    ctrl = np.empty((P, n_periods, 6), dtype=np.float64)
    ctrl[:, :, 0:2] = p0[:, None, :]
    ctrl[:, :, 4:6] = p2[:, None, :]
    if bend > 0.0:
        off = rng.uniform(-bend, bend, size=(P, n_periods))
        ctrl[:, :, 2:4] = (mid[:, None, :]
                           + (off * length[:, None])[:, :, None] * perp[:, None, :])
    else:
        ctrl[:, :, 2:4] = mid[:, None, :]
    return ctrl.reshape(P * n_periods, 6)


def depth_kernel_table(periods_s: np.ndarray, nz: int, dz: float) -> np.ndarray:
    """Kdz[t, k] = K_T(z_k) * dz with K_T(z) = (z/z0) exp(1 - z/z0), z0 = 1.2 T."""
    z = (np.arange(nz, dtype=np.float64) + 0.5) * dz
    z0 = 1.2 * np.asarray(periods_s, dtype=np.float64)[:, None]
    return (z[None, :] / z0) * np.exp(1.0 - z[None, :] / z0) * dz


def depth_kernel_cells(periods_s: np.ndarray, nx: int, ny: int, nz: int, dz: float,
                       amp: float = 0.3) -> np.ndarray:
    """Laterally varying depth kernels, (nx*ny, T, nz): under cell (ix, iy) the
    kernel depth is z0 = 1.2 T (1 + amp sin(2 pi (ix+0.5)/nx) cos(2 pi (iy+0.5)/ny)),
    the stand-in for a 1-D velocity model that changes across the grid; cells
    ordered h = iy*nx + ix as the columns."""
    z = (np.arange(nz, dtype=np.float64) + 0.5) * dz
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = (np.sin(2.0 * np.pi * (ix + 0.5) / nx) * np.cos(2.0 * np.pi * (iy + 0.5) / ny)).reshape(-1)
    z0 = 1.2 * np.asarray(periods_s, dtype=np.float64)[None, :, None] * (1.0 + amp * f)[:, None, None]
    return (z[None, None, :] / z0) * np.exp(1.0 - z[None, None, :] / z0) * dz


# ---------------------------------------------------------------- models

def checkerboard(nx: int, ny: int, nz: int, block: int, amp: float) -> np.ndarray:
    """amp * (-1)^(floor(ix/b) + floor(iy/b) + floor(k/b)), column order (iy, ix, k)."""
    iy, ix, k = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    sign = (ix // block + iy // block + k // block) % 2
    return (amp * (1.0 - 2.0 * sign)).reshape(-1).astype(np.float64)


def gaussian_blobs(rng: np.random.Generator, nx: int, ny: int, nz: int,
                   n_blobs: int = 12, amp: float = 0.08) -> np.ndarray:
    """Sum of signed 3-D Gaussian blobs rescaled to max |m| = amp."""
    iy, ix, k = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                            np.arange(nz) + 0.5, indexing="ij")
    m = np.zeros((ny, nx, nz), dtype=np.float64)
    for _ in range(n_blobs):
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        sh, sz = rng.uniform(4.0, 12.0), rng.uniform(2.0, 5.0)
        sgn = 1.0 if rng.uniform() < 0.5 else -1.0
        m += sgn * np.exp(-((ix - cx) ** 2 + (iy - cy) ** 2) / (2 * sh * sh)
                          - (k - cz) ** 2 / (2 * sz * sz))
    peak = np.max(np.abs(m))
    if peak > 0:
        m *= amp / peak
    return m.reshape(-1)


def noisy_rhs(g_m: np.ndarray, noise: np.ndarray, frac: float) -> np.ndarray:
    """d = G m_true + frac * RMS(G m_true) * z  (z unit normal, seeded)."""
    g_m = np.asarray(g_m, dtype=np.float64)
    rms = float(np.sqrt(np.mean(g_m * g_m))) if g_m.size else 0.0
    return g_m + frac * rms * np.asarray(noise, dtype=np.float64)


# ---------------------------------------------------------------- configs

def make_problem(name: str, nx: int, ny: int, nz: int, n_stations: int,
                 periods_s, bend: float, model: str, noise_frac: float,
                 w: float, lam: float, tol: float, itmax: int, seed: int,
                 dx_km: float = 1.0, dz_km: float = 2.0,
                 checker_block: int = 4, checker_amp: float = 0.05,
                 blob_amp: float = 0.08, lateral: bool = False, interp: int = 0) -> Problem:
    ss = np.random.SeedSequence(seed)
    r_st, r_ray, r_mod, r_noise = [np.random.default_rng(s) for s in ss.spawn(4)]
    periods = np.asarray(periods_s, dtype=np.float64)
    T = periods.shape[0]
    st = station_positions(r_st, n_stations, nx, ny, dx_km)
    pairs = station_pairs(n_stations)
    ctrl = ray_controls(r_ray, st, pairs, T, bend)
    row_period = np.tile(np.arange(T, dtype=np.int32), pairs.shape[0])
    kdz = depth_kernel_table(periods, nz, dz_km)
    if model == "checkerboard":
        m_true = checkerboard(nx, ny, nz, checker_block, checker_amp)
    elif model == "blobs":
        m_true = gaussian_blobs(r_mod, nx, ny, nz, amp=blob_amp)
    else:
        raise ValueError(f"unknown model kind {model!r}")
    noise = r_noise.standard_normal(ctrl.shape[0])
    kdz_cells = depth_kernel_cells(periods, nx, ny, nz, dz_km) if lateral else None
    return Problem(name=name, nx=nx, ny=ny, nz=nz, dx_km=dx_km, dz_km=dz_km,
                   stations=st, pairs=pairs, periods_s=periods, ctrl=ctrl,
                   row_period=row_period, kdz=kdz, w=w, lam=lam, tol=tol,
                   itmax=itmax, model_kind=model, noise_frac=noise_frac,
                   seed=seed, m_true=m_true, noise=noise, kdz_cells=kdz_cells, interp=interp)


def tiny(seed: int = 0) -> Problem:
    """16x16x8 grid, 20 stations (190 pairs) x 8 periods 2..16 s, straight rays,
    +-5 % checkerboard of 4-cell blocks, 1 % noise, w = 1, lambda = 0.1."""
    return make_problem("tiny_16x16x8", 16, 16, 8, 20, np.arange(2.0, 17.0, 2.0),
                        bend=0.0, model="checkerboard", noise_frac=0.01,
                        w=1.0, lam=0.1, tol=1e-8, itmax=300, seed=seed)


def tiny_lateral(seed: int = 0) -> Problem:
    """The 16x16x8 system with bent rays and depth kernels that vary across the
    grid (depth_kernel_cells): G is no longer separable into l (x) Kdz."""
    return make_problem("tiny_lateral_16x16x8", 16, 16, 8, 20, np.arange(2.0, 17.0, 2.0),
                        bend=0.15, model="checkerboard", noise_frac=0.01,
                        w=1.0, lam=0.1, tol=1e-8, itmax=300, seed=seed, lateral=True)


def tiny_bilinear(seed: int = 0) -> Problem:
    """The 16x16x8 system with bent rays, laterally varying kernels and Eq. 1's
    bilinear node coefficients (each chord split over the four nodes around it)."""
    return make_problem("tiny_bilinear_16x16x8", 16, 16, 8, 20, np.arange(2.0, 17.0, 2.0),
                        bend=0.15, model="checkerboard", noise_frac=0.01,
                        w=1.0, lam=0.1, tol=1e-8, itmax=300, seed=seed, lateral=True,
                        interp=1)


def mid(seed: int = 1) -> Problem:
    """64x64x16 grid, 120 stations (7,140 pairs) x 24 log-spaced periods 2..40 s,
    Bezier rays with +-0.15 bend, +-8 % Gaussian blobs, 2 % noise, w = 2,
    lambda = 0.05, tol 1e-6."""
    return make_problem("mid_64x64x16", 64, 64, 16, 120, np.geomspace(2.0, 40.0, 24),
                        bend=0.15, model="blobs", noise_frac=0.02,
                        w=2.0, lam=0.05, tol=1e-6, itmax=5000, seed=seed)


def large(seed: int = 2) -> Problem:
    """100x100x20 grid, 240 stations (28,680 pairs) x 30 periods 2..40 s."""
    return make_problem("large_100x100x20", 100, 100, 20, 240, np.geomspace(2.0, 40.0, 30),
                        bend=0.15, model="blobs", noise_frac=0.02,
                        w=2.0, lam=0.05, tol=1e-6, itmax=5000, seed=seed)


def paper_shaped(seed: int = 3) -> Problem:
    """Stand-in for the paper's field problem (the data are not available): the
    paper's 20 x 37 horizontal grid with 18 depth layers (13,320 unknowns), 229
    stations (26,106 pairs) x 14 periods 1..8 s = 365,484 rows; cells of 1.5 km,
    layers of 1 km, bent rays, Eq. 1's bilinear node coefficients, one depth
    kernel per period (a 1-D starting model, as in the paper's first
    iteration)."""
    return make_problem("paper_20x37x18", 20, 37, 18, 229, np.geomspace(1.0, 8.0, 14),
                        bend=0.15, model="blobs", noise_frac=0.02,
                        w=2.0, lam=0.05, tol=1e-6, itmax=5000, seed=seed,
                        dx_km=1.5, dz_km=1.0, interp=1)


BATCH_GRIDS = ((24, 24, 8), (32, 32, 12), (48, 48, 16), (64, 64, 16))


def batched_system(seed: int) -> Problem:
    """One uneven-size member of the batched workload: grid drawn from
    BATCH_GRIDS, 30-120 stations, 8-24 log-spaced periods in 2..40 s."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    nx, ny, nz = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
    n_st = int(rng.integers(30, 121))
    T = int(rng.integers(8, 25))
    return make_problem(f"batch_{seed}", nx, ny, nz, n_st, np.geomspace(2.0, 40.0, T),
                        bend=0.15, model="blobs", noise_frac=0.02,
                        w=2.0, lam=0.05, tol=1e-6, itmax=2000, seed=seed)


def batched_rhs_models(p: Problem):
    """The 16 right-hand-side recipes sharing one G: 8 checkerboards (block
    2..8, then block 8 with the opposite sign) at the system's lambda, and the
    blob model at 8 damping values logspace(-3, 0, 8).  Returns a list of
    (model vector, lambda)."""
    out = []
    for b in (2, 3, 4, 5, 6, 7, 8):
        out.append((checkerboard(p.nx, p.ny, p.nz, b, 0.05), p.lam))
    out.append((-checkerboard(p.nx, p.ny, p.nz, 8, 0.05), p.lam))
    for lam in np.logspace(-3.0, 0.0, 8):
        out.append((p.m_true, float(lam)))
    return out


def batched(n_systems: int = 64, first_seed: int = 1000):
    return [batched_system(first_seed + i) for i in range(n_systems)]


def rhs_noise(seed: int, m_rows: int, stream: int = 0) -> np.ndarray:
    """Extra seeded unit-normal noise vectors (one per right-hand side)."""
    return np.random.default_rng(np.random.SeedSequence([seed, 100 + stream])).standard_normal(m_rows)


def custom(nx: int, ny: int, nz: int, n_stations: int, n_periods: int, bend: float,
           seed: int, w: float = 1.0, lam: float = 0.1, model: str = "checkerboard",
           tol: float = 1e-8, itmax: int = 500, dx_km: float = 1.0,
           dz_km: float = 2.0) -> Problem:
    """Small ad-hoc systems for tests (ragged sizes, edge cases)."""
    return make_problem(f"custom_{nx}x{ny}x{nz}_{seed}", nx, ny, nz, n_stations,
                        np.geomspace(2.0, 40.0, n_periods) if n_periods > 1 else np.array([8.0]),
                        bend=bend, model=model, noise_frac=0.01, w=w, lam=lam,
                        tol=tol, itmax=itmax, seed=seed, dx_km=dx_km, dz_km=dz_km,
                        checker_block=2)
