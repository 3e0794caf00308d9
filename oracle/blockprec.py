"""Per-cell depth-block right preconditioner for LSQR on [G; w L; lam I].

TEST INFRASTRUCTURE ONLY (see the package docstring): the product computes
its own blocks on the device and never calls this module.

The columns of the augmented operator A = [G; w L; lam I] come in groups of
nz, one group per horizontal cell h (Eq. 7's depth-fastest order).  Within a
group they are strongly coupled: a row of G touches all nz depths of a cell
with the depth kernel of its period (Eq. 5), and L couples neighbouring
depths.  The preconditioner takes the diagonal block of the normal matrix for
each cell,

    B_h = A_h^T A_h,   A_h = the nz columns of A of cell h,

factors it as B_h = R_h^T R_h (Cholesky, R_h upper triangular) and solves
LSQR on A P with P = blockdiag(P_h), P_h = R_h^{-1}; the model is m = P y.
Every column group of A P is then orthonormal (P_h^T B_h P_h = I), the block
generalisation of column-norm scaling.  As with a diagonal scaling, the
damping becomes explicit operator rows lam P (m = P y makes the damping of y
a different problem), so the minimiser is the same m*.

Parity status: pinned in tests/test_oracle_blockprec.py against the diagonal
blocks of a dense A^T A built from an independent loop-based Laplacian,
against Gram matrices of the oracle's own A P products, and through the
dense-QR solution of the augmented system.
"""
from __future__ import annotations

import numpy as np

from . import CSR, laplacian


def _cell_columns_G(GT: CSR, h: int, nz: int):
    """The nz columns of G for cell h as (row index, value) lists (rows of
    G^T h*nz .. h*nz + nz - 1)."""
    out = []
    for k in range(nz):
        j = h * nz + k
        a, b = int(GT.ptr[j]), int(GT.ptr[j + 1])
        out.append((GT.idx[a:b], GT.val[a:b]))
    return out


def depth_block(GT: CSR, grid, w: float, lam: float, h: int) -> np.ndarray:
    """B_h = A_h^T A_h for A = [G; w L; lam I] (nz x nz, FP64), from the
    definition: the dot products of the cell's columns of G, of w L (each
    column is L applied to a unit vector) and of lam I."""
    nx, ny, nz = grid
    n = nx * ny * nz
    cols = _cell_columns_G(GT, h, nz)
    B = np.zeros((nz, nz))
    for i in range(nz):
        ri, vi = cols[i]
        for k in range(i, nz):
            rk, vk = cols[k]
            common, ia, ik = np.intersect1d(ri, rk, assume_unique=True, return_indices=True)
            B[i, k] = float(np.dot(vi[ia], vk[ik])) if common.size else 0.0
            B[k, i] = B[i, k]
    Lc = np.zeros((nz, n))
    for k in range(nz):
        e = np.zeros(n)
        e[h * nz + k] = 1.0
        Lc[k] = laplacian(nx, ny, nz, e)
    B += (w * w) * (Lc @ Lc.T)
    B += (lam * lam) * np.eye(nz)
    return B


def depth_blocks(GT: CSR, grid, w: float, lam: float, cells=None) -> np.ndarray:
    """B_h for the given cells (all nx*ny cells by default): (len, nz, nz)."""
    nx, ny, nz = grid
    cells = range(nx * ny) if cells is None else cells
    return np.stack([depth_block(GT, grid, w, lam, int(h)) for h in cells])


def inverse_cholesky(B: np.ndarray) -> np.ndarray:
    """P_h = R_h^{-1} with B_h = R_h^T R_h, R_h upper triangular with a
    positive diagonal, for every block of B (..., nz, nz)."""
    B = np.asarray(B, dtype=np.float64)
    Lo = np.linalg.cholesky(B)                 # B = Lo Lo^T, Lo = R^T
    R = np.swapaxes(Lo, -1, -2)
    eye = np.broadcast_to(np.eye(B.shape[-1]), B.shape)
    return np.linalg.solve(R, eye)             # R P = I


def block_precond(GT: CSR, grid, w: float, lam: float) -> np.ndarray:
    """P (nx*ny, nz, nz) for the augmented operator of the given w, lam."""
    return inverse_cholesky(depth_blocks(GT, grid, w, lam))


def apply_blocks(P: np.ndarray, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    """m = P x (or P^T x), cell by cell."""
    H, nz, _ = P.shape
    xb = np.asarray(x, dtype=np.float64).reshape(H, nz)
    op = np.swapaxes(P, 1, 2) if transpose else P
    return np.einsum("hik,hk->hi", op, xb).reshape(-1)
