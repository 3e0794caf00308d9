"""Pins of the LSMR oracle (Fong & Saunders 2011) against things other than
itself: SciPy's independent LSMR (iterates and estimates at fixed k, stopping
rule), the dense Householder-QR minimiser, the true residuals of its own
iterates (||r_k|| and ||A^T r_k|| estimates), the monotone decrease of
||A^T r_k|| that defines the method, and the equality of the damped and the
explicitly scaled forms."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import oracle
from oracle.lsmr import lsmr
from test_oracle_lsqr import augmented_dense, scipy_operator


def grid(p):
    return (p.nx, p.ny, p.nz)


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_lsmr_iterates_match_scipy(tiny_system, k):
    p, G, GT, d = tiny_system
    A = scipy_operator(p, G)
    b = np.concatenate([d, np.zeros(p.n)])
    # scipy returns (x, istop, itn, normr, normar, norma, conda, normx)
    ref = sla.lsmr(A, b, damp=p.lam, atol=0, btol=0, conlim=0, maxiter=k)
    res = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=k)
    assert res.itn == ref[2] == k
    assert np.linalg.norm(res.x - ref[0]) / np.linalg.norm(ref[0]) < 1e-12
    np.testing.assert_allclose([res.rnorm, res.arnorm, res.anorm, res.xnorm],
                               [ref[3], ref[4], ref[5], ref[7]], rtol=1e-11)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_lsmr_estimates_equal_true_norms(tiny_system, k):
    """||r_k|| (with the damping term) and ||A^T r_k|| from the recurrences
    equal the norms recomputed from x_k."""
    p, G, GT, d = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    res = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=k)
    r = b - A @ res.x
    np.testing.assert_allclose(res.rnorm, np.linalg.norm(r), rtol=1e-10)
    np.testing.assert_allclose(res.arnorm, np.linalg.norm(A.T @ r), rtol=1e-8)
    np.testing.assert_allclose(res.xnorm, np.linalg.norm(res.x), rtol=1e-14)


def test_lsmr_matches_dense_householder_qr(tiny_system):
    p, G, GT, d = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    Q, R = np.linalg.qr(A)
    m_qr = np.linalg.solve(R, Q.T @ b)
    res = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=1e-10, btol=1e-10, itmax=20000)
    assert res.istop in (1, 2)
    assert np.linalg.norm(res.x - m_qr) / np.linalg.norm(m_qr) < 1e-6
    # and LSQR reaches the same minimiser
    ref = oracle.lsqr(G, GT, grid(p), p.w, p.lam, d, atol=1e-10, btol=1e-10, itmax=20000)
    assert np.linalg.norm(res.x - ref.x) / np.linalg.norm(ref.x) < 1e-6


def test_lsmr_normal_residual_decreases(tiny_system):
    """LSMR minimises ||A^T r_k|| over the Krylov space, so the true value
    never increases from one step to the next."""
    p, G, GT, d = tiny_system
    A = augmented_dense(p, G, p.w, p.lam)
    b = np.concatenate([d, np.zeros(2 * p.n)])
    prev = np.inf
    for k in range(1, 13):
        res = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=k)
        cur = np.linalg.norm(A.T @ (b - A @ res.x))
        assert cur <= prev * (1 + 1e-9)
        prev = cur


def test_lsmr_stop_rule_matches_scipy(tiny_system):
    p, G, GT, d = tiny_system
    A = scipy_operator(p, G)
    b = np.concatenate([d, np.zeros(p.n)])
    for tol in (1e-4, 1e-6):
        ref = sla.lsmr(A, b, damp=p.lam, atol=tol, btol=tol, maxiter=20000)
        res = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=tol, btol=tol, itmax=20000)
        assert res.istop == ref[1]
        assert abs(res.itn - ref[2]) <= max(3, 0.02 * ref[2])


def test_lsmr_scaled_form_has_same_minimiser(tiny_system):
    """Right scaling m = D y with explicit lambda D rows (no recurrence damping)."""
    p, G, GT, d = tiny_system
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    a = lsmr(G, GT, grid(p), p.w, p.lam, d, atol=1e-10, btol=1e-10, itmax=20000)
    s = lsmr(G, GT, grid(p), p.w, 0.0, d, atol=1e-10, btol=1e-10, itmax=20000, D=D,
             lam_rows=p.lam)
    assert np.linalg.norm(D * s.x - a.x) / np.linalg.norm(a.x) < 1e-6
    assert s.itn < a.itn


def test_lsmr_zero_rhs(tiny_system):
    p, G, GT, d = tiny_system
    res = lsmr(G, GT, grid(p), p.w, p.lam, np.zeros_like(d))
    assert res.itn == 0 and not res.x.any()
