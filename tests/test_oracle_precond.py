"""Pins of the preconditioner oracles: the MLP's gradient against central
finite differences, closed-form special cases, and the column features on a
system whose G is known in closed form."""
import json
import math
import os

import numpy as np

import oracle
from oracle import features as ofeat
from oracle import mlp


def random_setup(seed=0, n=37):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, 8)) * 2 + 1
    theta = mlp.init_params(rng, F.mean(axis=0), F.std(axis=0) + 0.1)
    theta[2 * 8:] += 0.05 * rng.standard_normal(mlp.NTRAIN)    # non-zero biases too
    t = rng.standard_normal(n)
    return theta, F, t


def test_mlp_gradient_matches_central_differences():
    theta, F, t = random_setup()
    loss, grad = mlp.loss_and_grad(theta, F, t)
    assert grad.shape == (mlp.NTRAIN,)
    rng = np.random.default_rng(1)
    idx = np.concatenate([np.arange(0, 512, 37), [512 + 64 + 5, 512 + 64 + 4096 + 3,
                                                   mlp.NTRAIN - 1, mlp.NTRAIN - 10]])
    idx = np.unique(np.concatenate([idx, rng.choice(mlp.NTRAIN, 40, replace=False)]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[16 + i] += h
        tm[16 + i] -= h
        fd = (mlp.loss_and_grad(tp, F, t)[0] - mlp.loss_and_grad(tm, F, t)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_mlp_zero_weights_gives_softplus_of_bias():
    theta, F, _ = random_setup()
    theta[16:] = 0.0
    theta[-1] = 0.7
    logD, _ = mlp.forward(theta, F)
    np.testing.assert_allclose(logD, math.log(math.log1p(math.exp(0.7))), rtol=1e-14)


def test_mlp_large_negative_output_is_linear_in_log():
    theta, F, _ = random_setup()
    theta[16:] = 0.0
    theta[-1] = -30.0
    logD, _ = mlp.forward(theta, F)
    np.testing.assert_allclose(logD, -30.0, rtol=1e-12)


def test_adam_first_step_moves_by_lr_times_sign():
    theta, F, t = random_setup()
    _, g = mlp.loss_and_grad(theta, F, t)
    th2, m, v = mlp.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    step = (th2 - theta)[16:]
    nz = np.abs(g) > 1e-4
    np.testing.assert_allclose(step[nz], -1e-3 * np.sign(g[nz]), rtol=1e-3)


def test_features_on_a_single_straight_ray():
    """One straight ray along cell row iy = 2 of a 12 x 4 x 3 grid (the golden
    'row_of_cells' case): columns of the 11 hit cells hold l_h * Kdz[k] for one
    row, all others are empty; every feature follows in closed form."""
    case = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "closed_form_rays.json")))["cases"][0]
    nx, ny, nz = case["nx"], case["ny"], 3
    p0, p2 = case["p0"], case["p2"]
    ctrl = np.array([[p0[0], p0[1], (p0[0] + p2[0]) / 2, (p0[1] + p2[1]) / 2, p2[0], p2[1]]])
    kdz = np.array([[0.9, 0.5, 0.2]])
    G = oracle.build_G(nx, ny, nz, 1.0, ctrl, np.zeros(1, np.int32), kdz)
    GT = oracle.transpose(G)
    logT = np.array([math.log(6.0)])
    F = ofeat.features(GT, nx, ny, nz, np.zeros(1, np.int32), logT)
    lengths = dict(zip(case["cells"], case["lengths"]))
    norm = np.zeros(nx * ny * nz)
    for h, l in lengths.items():
        for k in range(nz):
            norm[h * nz + k] = l * kdz[0, k]
    for j in range(nx * ny * nz):
        h, k = j // nz, j % nz
        hit = h in lengths
        assert math.isclose(F[j, 0], math.log(norm[j] + 1e-8), rel_tol=1e-12, abs_tol=1e-12)
        assert F[j, 1] == (math.log(2.0) if hit else 0.0)
        assert F[j, 2] == (k + 0.5) / nz
        assert math.isclose(F[j, 3], math.log(6.0) if hit else 0.0, rel_tol=1e-12)
        assert math.isclose(F[j, 7], math.log(norm[j] + 1e-8), rel_tol=1e-12, abs_tol=1e-12)
    # a corner column (ix = 0, iy = 0, k = 0) has neighbours k+1, ix+1, iy+1, all empty
    assert math.isclose(F[0, 4], math.log(1e-8), rel_tol=1e-12)
    # column of cell (ix=5, iy=2), k=1: neighbours k-1, k+1 (same cell, hit), ix-1, ix+1
    # (hit), iy-1, iy+1 (empty)
    h = 2 * nx + 5
    j = h * nz + 1
    nb = [norm[j - 1], norm[j + 1], norm[j - nz], norm[j + nz], 0.0, 0.0]
    t = np.array(nb) + 1e-8
    assert math.isclose(F[j, 4], math.log(t.mean()), rel_tol=1e-12)
    assert math.isclose(F[j, 5], math.log(t.min()), rel_tol=1e-12)
    assert math.isclose(F[j, 6], math.log(t.max()), rel_tol=1e-12)
