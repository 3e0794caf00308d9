"""Pins of the oracle's outer nonlinear loop (oracle/outer.py), independent of
its own code:

* the depth-kernel table follows its definition: the depth integral of
  K_T(z) = (z/z0) exp(1 - z/z0) over [0, Z] is e z0 (1 - (1 + Z/z0) e^(-Z/z0))
  in closed form, so the midpoint sums of a finely layered table give z0 per
  (cell, period), z0 = 1.2 T mean_k(1 + m) -- a wrong mean, scale, sign or
  layer thickness fails;
* with a kernel that does not follow the model (kernel_power = 0) G is fixed
  and the loop is iterated Tikhonov regularisation, whose iterates have the
  closed form m_{k+1} = m_k + R^-1 G^T (d - G m_k), R = G^T G + w^2 L^T L +
  lambda^2 I: checked on a dense system with numpy's solver;
* the stopping rules fire as stated, and on noise-free data from a planted
  model the RMS misfit falls below a tenth of its start.
"""
import numpy as np

import oracle
from oracle import outer
from paper_2604_11920_b300 import synth


def test_kernel_table_depth_integral_closed_form():
    rng = np.random.default_rng(5)
    nx, ny, nz, dz = 3, 2, 4000, 0.025
    m = rng.uniform(-0.1, 0.1, nx * ny * nz)
    periods = np.array([2.0, 3.5, 5.0])
    K = outer.kernel_table(periods, nx, ny, nz, dz, m)
    assert K.shape == (nx * ny, 3, nz)
    s = 1.0 + m.reshape(nx * ny, nz).mean(axis=1)
    Z = nz * dz
    for h in range(nx * ny):
        for t, T in enumerate(periods):
            z0 = 1.2 * T * s[h]
            exact = np.e * z0 * (1.0 - (1.0 + Z / z0) * np.exp(-Z / z0))
            assert abs(K[h, t].sum() - exact) <= 1e-4 * exact
    # kernel_power = 0: every column keeps the 1-D kernel of its period
    K0 = outer.kernel_table(periods, nx, ny, nz, dz, m, kernel_power=0.0)
    for t, T in enumerate(periods):
        exact = np.e * 1.2 * T * (1.0 - (1.0 + Z / (1.2 * T)) * np.exp(-Z / (1.2 * T)))
        assert np.allclose(K0[:, t].sum(axis=1), exact, rtol=1e-4)


def test_kernel_table_at_zero_model_is_the_1d_table():
    p = synth.tiny()
    K = outer.kernel_table(p.periods_s, p.nx, p.ny, p.nz, p.dz_km, np.zeros(p.n))
    for h in (0, 17, p.nx * p.ny - 1):
        assert np.allclose(K[h], p.kdz, rtol=1e-15, atol=0)
    G0 = outer.G_of_model(p, np.zeros(p.n))
    G = oracle.build_G_problem(p)
    assert np.array_equal(G0.idx, G.idx) and np.allclose(G0.val, G.val, rtol=1e-15, atol=0)


def _dense(p):
    G = oracle.build_G_problem(p).to_scipy().toarray()
    L = np.stack([oracle.laplacian(p.nx, p.ny, p.nz, e) for e in np.eye(p.n)], axis=1)
    return G, L


def test_fixed_kernel_loop_is_iterated_tikhonov():
    p = synth.custom(4, 4, 2, 10, 4, bend=0.1, seed=61, w=0.7, lam=0.3)
    G, L = _dense(p)
    rng = np.random.default_rng(3)
    d = G @ rng.uniform(-0.05, 0.05, p.n) + 0.01 * rng.standard_normal(G.shape[0])
    R = G.T @ G + p.w ** 2 * (L.T @ L) + p.lam ** 2 * np.eye(p.n)
    res = outer.outer_loop(p, d, p.w, p.lam, itmax=5000, tol=1e-14, max_outer=4, rms_tol=0.0,
                           min_decrease=0.0, kernel_power=0.0)
    assert res.reason == 3 and res.updates == 4 and len(res.rms) == 5
    m = np.zeros(p.n)
    for k in range(5):
        r = d - G @ m
        assert abs(res.rms[k] - np.sqrt(np.mean(r * r))) <= 1e-9 * res.rms[k]
        if k < 4:
            m = m + np.linalg.solve(R, G.T @ r)
    assert np.linalg.norm(res.m - m) <= 1e-9 * np.linalg.norm(m)
    # iterated Tikhonov lowers the data misfit at every step
    assert np.all(np.diff(res.rms) < 0)


def test_stopping_rules():
    p = synth.custom(4, 4, 2, 10, 4, bend=0.1, seed=62, w=0.7, lam=0.3)
    d = outer.forward(p, synth.checkerboard(p.nx, p.ny, p.nz, 2, 0.05))
    big = outer.outer_loop(p, d, p.w, p.lam, 500, 1e-10, max_outer=5, rms_tol=1e9,
                           min_decrease=0.0)
    assert big.reason == 1 and big.updates == 0 and not big.m.any()
    two = outer.outer_loop(p, d, p.w, p.lam, 500, 1e-10, max_outer=2, rms_tol=0.0,
                           min_decrease=0.0)
    assert two.reason == 3 and two.updates == 2
    slow = outer.outer_loop(p, d, p.w, p.lam, 500, 1e-10, max_outer=20, rms_tol=0.0,
                            min_decrease=0.99)
    assert slow.reason == 2 and 1 <= slow.updates < 20
    assert slow.rms[-1] > 0.01 * slow.rms[-2]


def test_planted_model_misfit_falls():
    p = synth.custom(10, 9, 4, 18, 5, bend=0.15, seed=63, w=0.3, lam=0.02, dz_km=1.0)
    m_true = synth.checkerboard(p.nx, p.ny, p.nz, 2, 0.08)
    d = outer.forward(p, m_true)
    res = outer.outer_loop(p, d, p.w, p.lam, 3000, 1e-10, max_outer=6, rms_tol=0.0,
                           min_decrease=0.0)
    assert res.updates == 6
    assert res.rms[-1] < 0.1 * res.rms[0]
    assert res.rms[1] < res.rms[0] and res.rms[2] < res.rms[1]
    # the kernel follows the model: G(m) differs from G(0) at the result
    G0 = outer.G_of_model(p, np.zeros(p.n))
    Gm = outer.G_of_model(p, res.m)
    assert np.max(np.abs(Gm.val - G0.val)) > 1e-3 * np.max(np.abs(G0.val))
