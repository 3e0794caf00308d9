"""FP64 oracle of the per-column features of G used by the learned
preconditioner (test infrastructure).  Definitions, for column j = h*nz + k:

  f0 log(||G_:j|| + 1e-8)             f1 log(1 + rows in column j)
  f2 (k + 1/2) / nz                   f3 sum_r G_rj^2 log T(r) / sum_r G_rj^2 (0 if empty)
  f4, f5, f6 log of mean / min / max of (||G_:i|| + 1e-8) over existing 7-point neighbours
  f7 log(max_r |G_rj| + 1e-8)

Computed from the oracle's CSC (transpose) arrays with plain loops over
columns; pinned by hand-computed values on a one-ray system in
tests/test_oracle_precond.py.
"""
import numpy as np

EPS = 1e-8


def features(GT, nx, ny, nz, row_period, log_periods):
    n = GT.n_rows
    F = np.zeros((n, 8))
    norms = np.zeros(n)
    for j in range(n):
        lo, hi = GT.ptr[j], GT.ptr[j + 1]
        g = GT.val[lo:hi]
        rows = GT.idx[lo:hi]
        s2 = float(np.sum(g * g))
        norms[j] = np.sqrt(s2)
        F[j, 0] = np.log(norms[j] + EPS)
        F[j, 1] = np.log1p(hi - lo)
        F[j, 2] = ((j % nz) + 0.5) / nz
        F[j, 3] = float(np.sum(g * g * log_periods[row_period[rows]])) / s2 if s2 > 0 else 0.0
        F[j, 7] = np.log((np.max(np.abs(g)) if hi > lo else 0.0) + EPS)
    for j in range(n):
        k, hh = j % nz, j // nz
        ix, iy = hh % nx, hh // nx
        nb = []
        if k > 0: nb.append(j - 1)
        if k < nz - 1: nb.append(j + 1)
        if ix > 0: nb.append(j - nz)
        if ix < nx - 1: nb.append(j + nz)
        if iy > 0: nb.append(j - nx * nz)
        if iy < ny - 1: nb.append(j + nx * nz)
        t = norms[nb] + EPS if nb else np.array([EPS])
        F[j, 4], F[j, 5], F[j, 6] = np.log(t.mean()), np.log(t.min()), np.log(t.max())
    return F
