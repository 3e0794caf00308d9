"""Pins of the oracle's per-cell depth-block preconditioner (oracle/blockprec.py).

B_h is checked against the diagonal blocks of a dense A^T A whose Laplacian
is the Kronecker sum of 1-D path Laplacians (not the oracle's loop), P_h
against the Cholesky identities, the preconditioned operator of the C oracle
against the blocks it should orthonormalise, and the preconditioned LSQR
against the dense-QR minimiser of the augmented system.
"""
import numpy as np
import pytest

import oracle
from oracle import blockprec
from paper_2604_11920_b300 import synth
from test_oracle_lsqr import augmented_dense


def _dense_blocks(p, G, w, lam):
    A = augmented_dense(p, G, w, lam)
    N = A.T @ A
    H, nz = p.nx * p.ny, p.nz
    return np.stack([N[h * nz:(h + 1) * nz, h * nz:(h + 1) * nz] for h in range(H)])


@pytest.mark.parametrize("w,lam", [(1.0, 0.1), (0.0, 0.3), (2.5, 0.0)])
def test_blocks_equal_dense_normal_matrix(tiny_system, w, lam):
    p, G, GT, _ = tiny_system
    B = blockprec.depth_blocks(GT, (p.nx, p.ny, p.nz), w, lam)
    np.testing.assert_allclose(B, _dense_blocks(p, G, w, lam), rtol=1e-13, atol=1e-12)


def test_blocks_on_a_ragged_grid_with_one_depth_and_edges():
    """3 x 5 x 3 grid (corner, edge and interior cells, top and bottom depths)
    and a 4 x 2 x 1 grid (a single depth: 1 x 1 blocks = squared column norms)."""
    for nx, ny, nz, nst in ((3, 5, 3, 6), (4, 2, 1, 5)):
        p = synth.custom(nx, ny, nz, nst, 3, bend=0.1, seed=11)
        G = oracle.build_G_problem(p)
        GT = oracle.transpose(G)
        B = blockprec.depth_blocks(GT, (nx, ny, nz), 1.3, 0.2)
        np.testing.assert_allclose(B, _dense_blocks(p, G, 1.3, 0.2), rtol=1e-13, atol=1e-12)
        if nz == 1:
            np.testing.assert_allclose(B[:, 0, 0], oracle.aug_colnorm2(GT, nx, ny, nz, 1.3, 0.2),
                                       rtol=1e-13)


def test_inverse_cholesky_identities(tiny_system):
    p, G, GT, _ = tiny_system
    B = blockprec.depth_blocks(GT, (p.nx, p.ny, p.nz), p.w, p.lam)
    P = blockprec.inverse_cholesky(B)
    nz = p.nz
    assert np.all(np.tril(P, -1) == 0.0)                      # upper triangular
    assert np.all(np.diagonal(P, axis1=1, axis2=2) > 0.0)     # positive diagonal
    I = np.einsum("hki,hkl,hlj->hij", P, B, P)                # P^T B P
    np.testing.assert_allclose(I, np.broadcast_to(np.eye(nz), I.shape), atol=1e-9)
    R = np.linalg.inv(P)                                      # B = R^T R
    np.testing.assert_allclose(np.einsum("hki,hkj->hij", R, R), B, rtol=1e-10,
                               atol=1e-10 * np.abs(B).max())


def test_preconditioned_operator_has_orthonormal_cell_groups(tiny_system):
    """The columns of [G P; w L P; lam P] of one cell, produced by the C
    oracle's operator on unit vectors, are orthonormal; the adjoint product
    is the transpose of the forward one."""
    p, G, GT, _ = tiny_system
    grid = (p.nx, p.ny, p.nz)
    P = blockprec.block_precond(GT, grid, p.w, p.lam)
    nz = p.nz
    for h in (0, 17, p.nx * p.ny - 1):
        cols = []
        for k in range(nz):
            e = np.zeros(p.n)
            e[h * nz + k] = 1.0
            cols.append(oracle.apply_A(G, grid, p.w, e, lam_rows=p.lam, P=P))
        C = np.stack(cols)
        np.testing.assert_allclose(C @ C.T, np.eye(nz), atol=1e-9)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(p.n)
    u = rng.standard_normal(G.n_rows + 2 * p.n)
    lhs = np.dot(oracle.apply_A(G, grid, p.w, v, lam_rows=p.lam, P=P), u)
    rhs = np.dot(v, oracle.apply_At(GT, grid, p.w, u, lam_rows=p.lam, P=P))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_block_preconditioned_lsqr_reaches_the_qr_minimiser(tiny_system):
    """m = P y on [G P; w L P; lam P] (no recurrence damping) is the minimiser
    of ||G m - d||^2 + w^2 ||L m||^2 + lam^2 ||m||^2, and takes fewer
    iterations than column-norm scaling on this system."""
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    Q, R = np.linalg.qr(A)
    m_qr = np.linalg.solve(R, Q.T @ b)
    P = blockprec.block_precond(GT, grid, p.w, p.lam)
    res = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=1e-10, btol=1e-10, itmax=20000,
                      P=P, lam_rows=p.lam)
    assert res.istop in (1, 2)
    m = blockprec.apply_blocks(P, res.x)
    assert np.linalg.norm(m - m_qr) / np.linalg.norm(m_qr) < 1e-6
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    col = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=1e-10, btol=1e-10, itmax=20000,
                      D=D, lam_rows=p.lam)
    assert res.itn < col.itn


def test_single_depth_blocks_equal_column_norm_scaling():
    """With nz = 1 every block is 1 x 1 and P_h = 1/||A_:h||: the block form is
    column-norm scaling, iterate for iterate."""
    p = synth.custom(8, 6, 1, 10, 4, bend=0.1, seed=3)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    grid = (p.nx, p.ny, p.nz)
    P = blockprec.block_precond(GT, grid, p.w, p.lam)
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    np.testing.assert_allclose(P[:, 0, 0], D, rtol=1e-14)
    a = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=25, P=P,
                    lam_rows=p.lam)
    b = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=25, D=D,
                    lam_rows=p.lam)
    np.testing.assert_allclose(a.x, b.x, rtol=1e-10, atol=1e-14)


def test_blocks_definite_without_rays_or_damping():
    """Cells that no ray crosses, and lambda = 0: with w > 0 every block is still
    positive definite (a proper subset of the Laplacian's columns is linearly
    independent: its only null vector is the constant one), and the
    preconditioned LSQR still reaches the dense-QR minimiser."""
    p = synth.custom(12, 12, 4, 3, 2, bend=0.0, seed=5, w=1.0, lam=0.0)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    grid = (p.nx, p.ny, p.nz)
    cnt = np.diff(GT.ptr).reshape(p.nx * p.ny, p.nz).sum(axis=1)
    assert (cnt == 0).sum() > 50                               # most cells see no ray
    B = blockprec.depth_blocks(GT, grid, p.w, 0.0)
    assert np.all(np.linalg.eigvalsh(B) > 1e-3)
    P = blockprec.inverse_cholesky(B)
    A = augmented_dense(p, G, p.w, 0.0)[: G.n_rows + p.n]     # no damping rows
    b = np.concatenate([d, np.zeros(p.n)])
    m_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    res = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=1e-12, btol=1e-12, itmax=20000, P=P)
    m = blockprec.apply_blocks(P, res.x)
    assert np.linalg.norm(m - m_ls) / np.linalg.norm(m_ls) < 1e-6
