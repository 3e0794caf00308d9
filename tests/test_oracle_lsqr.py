"""Pins of the oracle's operators and of its LSQR (Paige & Saunders 1982).

The oracle's solution is compared with a dense Householder QR of the
augmented system, its iterates with SciPy's independent LSQR, and it must
recover planted models exactly on consistent data and satisfy the
Golub-Kahan relations.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
from paper_2604_11920_b300 import synth


def path_laplacian(n):
    """1-D graph Laplacian of a path with n nodes."""
    if n == 1:
        return sp.csr_matrix((1, 1))
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    return sp.diags([main, -np.ones(n - 1), -np.ones(n - 1)], [0, -1, 1]).tocsr()


def kron_laplacian(nx, ny, nz):
    """3-D 7-point graph Laplacian as the Kronecker sum of 1-D path Laplacians,
    in the column order (iy, ix, k) with k fastest."""
    Iz, Ix, Iy = sp.identity(nz), sp.identity(nx), sp.identity(ny)
    return (sp.kron(sp.kron(Iy, Ix), path_laplacian(nz))
            + sp.kron(sp.kron(Iy, path_laplacian(nx)), Iz)
            + sp.kron(sp.kron(path_laplacian(ny), Ix), Iz)).tocsr()


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (3, 1, 2), (4, 5, 3), (16, 16, 8)])
def test_laplacian_is_kronecker_sum(dims):
    nx, ny, nz = dims
    x = np.random.default_rng(1).standard_normal(nx * ny * nz)
    np.testing.assert_allclose(oracle.laplacian(nx, ny, nz, x), kron_laplacian(nx, ny, nz) @ x,
                               rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.laplacian(nx, ny, nz, np.ones_like(x)), 0.0)


def augmented_dense(p, G, w, lam):
    L = kron_laplacian(p.nx, p.ny, p.nz).toarray()
    return np.vstack([G.to_scipy().toarray(), w * L, lam * np.eye(p.n)])


def test_aug_colnorm2(tiny_system):
    p, G, GT, _ = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    np.testing.assert_allclose(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam),
                               np.sum(A * A, axis=0), rtol=1e-12)


def test_lsqr_matches_dense_householder_qr(tiny_system):
    """Converged LSQR = argmin ||G m - d||^2 + w^2||L m||^2 + lam^2||m||^2."""
    p, G, GT, d = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    Q, R = np.linalg.qr(A)
    m_qr = np.linalg.solve(R, Q.T @ b)
    res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-10, btol=1e-10,
                      itmax=20000)
    assert res.istop in (1, 2)
    assert np.linalg.norm(res.x - m_qr) / np.linalg.norm(m_qr) < 1e-6
    # the estimates at termination agree with the explicit residuals
    r = b - A @ res.x
    np.testing.assert_allclose(res.rnorm, np.linalg.norm(r), rtol=1e-8)
    np.testing.assert_allclose(res.arnorm, np.linalg.norm(A.T @ r), rtol=1e-3, atol=1e-9)
    np.testing.assert_allclose(res.xnorm, np.linalg.norm(res.x), rtol=1e-6)
    np.testing.assert_allclose(res.bnorm, np.linalg.norm(d), rtol=1e-14)
    # the ||B_k||_F estimate of ||A|| is at least the largest singular value
    assert res.anorm >= np.linalg.norm(A, 2) * (1 - 1e-9)


def scipy_operator(p, G):
    L = kron_laplacian(p.nx, p.ny, p.nz)
    return sp.vstack([G.to_scipy(), p.w * L]).tocsr()


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_lsqr_iterates_match_scipy(tiny_system, k):
    """Same algorithm, independent code: iterates agree at fixed k while the
    bidiagonalisation is still orthogonal (rounding grows ~10x per step on
    this system afterwards, see the orthogonality test)."""
    p, G, GT, d = tiny_system
    A = scipy_operator(p, G)
    b = np.concatenate([d, np.zeros(p.n)])
    ref = sla.lsqr(A, b, damp=p.lam, atol=0, btol=0, conlim=0, iter_lim=k)
    res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                      itmax=k)
    assert res.itn == ref[2] == k
    assert np.linalg.norm(res.x - ref[0]) / np.linalg.norm(ref[0]) < 1e-12
    # scipy returns (x, istop, itn, r1norm, r2norm, anorm, acond, arnorm, xnorm, var)
    np.testing.assert_allclose([res.rnorm, res.anorm, res.acond, res.arnorm, res.xnorm],
                               [ref[4], ref[5], ref[6], ref[7], ref[8]], rtol=1e-11)


def test_lsqr_stop_rule_matches_scipy(tiny_system):
    p, G, GT, d = tiny_system
    A = scipy_operator(p, G)
    b = np.concatenate([d, np.zeros(p.n)])
    for tol in (1e-4, 1e-6):
        ref = sla.lsqr(A, b, damp=p.lam, atol=tol, btol=tol, iter_lim=20000)
        res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=tol, btol=tol,
                          itmax=20000)
        assert res.istop == ref[1]
        assert abs(res.itn - ref[2]) <= max(3, 0.1 * ref[2])


def test_exact_recovery_min_norm(tiny_system):
    """w = lam = 0, consistent data d = G m_true with m_true = G^T z in the row
    space: LSQR from x0 = 0 converges to the minimum-norm solution m_true."""
    p, G, GT, _ = tiny_system
    z = np.random.default_rng(5).standard_normal(G.n_rows)
    m_true = oracle.spmv(GT, z)
    d = oracle.spmv(G, m_true)
    res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), 0.0, 0.0, d, atol=1e-14, btol=1e-14,
                      conlim=1e14, itmax=8000)
    # G alone is ill-conditioned on its row space; the planted model is still
    # recovered to the 1e-4 model-error bound used for all parity checks
    assert np.linalg.norm(res.x - m_true) / np.linalg.norm(m_true) < 1e-4
    # and nothing outside the row space is added: x stays in range(G^T)
    z_ls = np.linalg.lstsq(G.to_scipy().toarray().T, res.x, rcond=None)
    assert np.linalg.norm(oracle.spmv(GT, z_ls[0]) - res.x) < 1e-8 * np.linalg.norm(res.x)


def test_exact_recovery_overdetermined():
    """4x4x2 grid (32 unknowns), 20 stations x 8 periods = 1,520 rows, random
    planted model, noise-free data: the unique solution is recovered."""
    p = synth.custom(4, 4, 2, 20, 8, bend=0.15, seed=3)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    m_true = np.random.default_rng(9).standard_normal(p.n)
    d = oracle.spmv(G, m_true)
    res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), 0.0, 0.0, d, atol=1e-15, btol=1e-15,
                      conlim=1e15, itmax=5000)
    assert np.linalg.norm(res.x - m_true) / np.linalg.norm(m_true) < 1e-9


def test_golub_kahan_invariants(tiny_system):
    """Orthonormal U, V to 1e-10 while the process is still orthogonal (the
    first 9 steps on this system: its leading singular values are well
    separated, so finite-precision Golub-Kahan loses orthogonality about 10x
    per step once the top Ritz value converges), the two-term recurrences for
    20 steps, and non-increasing ||r||."""
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    K = 21
    res = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=K - 1,
                      record=K, history=True)
    U, V = res.U, res.V
    for k in range(2, 10):
        assert np.abs(U[:k] @ U[:k].T - np.eye(k)).max() < 1e-10
        assert np.abs(V[:k] @ V[:k].T - np.eye(k)).max() < 1e-10
    # A v_i = alpha_i u_i + beta_{i+1} u_{i+1};  A^T u_{i+1} = beta_{i+1} v_i + alpha_{i+1} v_{i+1}
    for i in range(K - 1):
        Av = oracle.apply_A(G, grid, p.w, V[i])
        alpha, beta = U[i] @ Av, U[i + 1] @ Av
        assert np.linalg.norm(Av - alpha * U[i] - beta * U[i + 1]) < 1e-11 * np.linalg.norm(Av)
        Atu = oracle.apply_At(GT, grid, p.w, U[i + 1])
        a2 = V[i + 1] @ Atu
        assert np.linalg.norm(Atu - beta * V[i] - a2 * V[i + 1]) < 1e-11 * np.linalg.norm(Atu)
    assert np.all(np.diff(res.rhist) <= 1e-12 * res.rhist[0])
    long = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=400,
                       history=True)
    assert np.all(np.diff(long.rhist) <= 1e-12 * long.rhist[0])


def test_damping_does_not_change_bidiagonalisation(tiny_system):
    """lam enters only the scalar recurrence: U, V are bit-identical."""
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    runs = [oracle.lsqr(G, GT, grid, p.w, lam, d, atol=0, btol=0, conlim=0, itmax=12, record=13)
            for lam in (0.0, 0.05, 1.0)]
    for r in runs[1:]:
        assert np.array_equal(r.U, runs[0].U) and np.array_equal(r.V, runs[0].V)
    assert not np.array_equal(runs[0].x, runs[1].x)


def test_column_scaled_form_has_same_minimiser(tiny_system):
    """m = D y on [G D; w L D; lam D] with no recurrence damping reaches the
    same minimiser as the damped unscaled problem."""
    p, G, GT, d = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    m_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    res = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, d, atol=1e-10, btol=1e-10,
                      itmax=20000, D=D, lam_rows=p.lam)
    m = D * res.x
    assert np.linalg.norm(m - m_ref) / np.linalg.norm(m_ref) < 1e-6
    plain = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-10, btol=1e-10,
                        itmax=20000)
    assert res.itn < plain.itn  # column scaling helps on this system


def test_zero_rhs_and_zero_iterations(tiny_system):
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    r0 = oracle.lsqr(G, GT, grid, p.w, p.lam, np.zeros_like(d))
    assert r0.itn == 0 and r0.istop == 0 and not r0.x.any()
    r1 = oracle.lsqr(G, GT, grid, p.w, p.lam, d, itmax=0)
    assert r1.itn == 0 and not r1.x.any()


def test_checkpoints_equal_separate_solves(tiny_system):
    """The checkpoint output of one run is, for each tolerance t, exactly what a
    separate solve with atol = btol = t returns (the iteration does not depend
    on the tolerances; only the stopping point does)."""
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    ladder = (1e-3, 1e-5, 1e-7, 1e-9)
    one = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=1e-12, btol=1e-12, itmax=20000,
                      checkpoints=ladder)
    assert np.all(np.diff(one.ck_itn) >= 0) and one.ck_itn[0] > 0
    for c, t in enumerate(ladder):
        sep = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=t, btol=t, itmax=20000)
        assert sep.istop in (1, 2)
        assert one.ck_itn[c] == sep.itn
        assert np.array_equal(one.ck_x[c], sep.x)
