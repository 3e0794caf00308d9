"""Pins of the oracle's sensitivity-matrix assembly (Eq. 5-7, synthetic form).

The oracle is checked against values fixed by hand (tests/golden), against an
independent closed-form midpoint rule for straight rays, against a power-basis
re-evaluation of curved rays and against the arc length of the curve.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_rays.json")


def _one_ray_G(nx, ny, nz, dx, p0, p1, p2, kdz=None):
    ctrl = np.array([[p0[0], p0[1], p1[0], p1[1], p2[0], p2[1]]], dtype=np.float64)
    if kdz is None:
        kdz = np.arange(1, nz + 1, dtype=np.float64)[None, :] * 0.5
    return oracle.build_G(nx, ny, nz, dx, ctrl, np.zeros(1, np.int32), kdz), kdz


def _cell_lengths(G, kdz, nz, row=0, t=0):
    lo, hi = G.ptr[row], G.ptr[row + 1]
    cols, vals = G.idx[lo:hi], G.val[lo:hi]
    cells = cols[::nz] // nz
    lengths = vals[::nz] / kdz[t, 0]
    return cells, lengths, cols, vals


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_closed_form_rays(case):
    nz = 3
    p0, p2 = case["p0"], case["p2"]
    p1 = [(p0[0] + p2[0]) / 2, (p0[1] + p2[1]) / 2]
    G, kdz = _one_ray_G(case["nx"], case["ny"], nz, case["dx"], p0, p1, p2)
    cells, lengths, cols, vals = _cell_lengths(G, kdz, nz)
    assert list(cells) == case["cells"]
    np.testing.assert_allclose(lengths, case["lengths"], rtol=1e-12, atol=1e-12)
    # every hit cell contributes all nz depth columns, depth fastest (Eq. 5, Eq. 7)
    assert G.nnz == nz * len(case["cells"])
    for i, h in enumerate(case["cells"]):
        assert list(cols[i * nz:(i + 1) * nz]) == [h * nz + k for k in range(nz)]
        np.testing.assert_allclose(vals[i * nz:(i + 1) * nz], case["lengths"][i] * kdz[0],
                                   rtol=1e-12, atol=1e-12)


def test_straight_rays_match_midpoint_rule():
    """Random straight rays: the Bezier walk must equal the closed-form
    midpoint rule P0 + (s - 1/2)/N (P2 - P0), each chord of length L/N."""
    rng = np.random.default_rng(11)
    nx, ny, nz, dx = 7, 5, 2, 1.5
    checked = 0
    for _ in range(200):
        p0 = rng.uniform([0, 0], [nx * dx, ny * dx])
        p2 = rng.uniform([0, 0], [nx * dx, ny * dx])
        L = math.hypot(*(p2 - p0))
        N = max(1, math.ceil(4 * L / dx))
        s = (np.arange(1, N + 1) - 0.5) / N
        mids = p0[None, :] + s[:, None] * (p2 - p0)[None, :]
        frac = mids / dx - np.floor(mids / dx)
        if np.min(np.minimum(frac, 1 - frac)) < 1e-7 or abs(4 * L / dx - round(4 * L / dx)) < 1e-9:
            continue  # a midpoint or N on a rounding boundary: not a clean closed form
        ix = np.clip(np.floor(mids[:, 0] / dx), 0, nx - 1).astype(int)
        iy = np.clip(np.floor(mids[:, 1] / dx), 0, ny - 1).astype(int)
        h = iy * nx + ix
        exp_cells, counts = np.unique(h, return_counts=True)
        G, kdz = _one_ray_G(nx, ny, nz, dx, p0, (p0 + p2) / 2, p2)
        cells, lengths, _, _ = _cell_lengths(G, kdz, nz)
        assert np.array_equal(cells, exp_cells)
        np.testing.assert_allclose(lengths, counts * L / N, rtol=1e-11)
        np.testing.assert_allclose(lengths.sum(), L, rtol=1e-12)
        checked += 1
    assert checked > 150


def test_curved_rays_total_length():
    """Bent rays: the per-cell lengths sum to the chord polygon length computed
    from the power-basis form B = P0 + 2 tau (P1 - P0) + tau^2 (P0 - 2 P1 + P2),
    which is within the chord-approximation error of the arc length."""
    rng = np.random.default_rng(12)
    nx, ny, nz, dx = 9, 8, 2, 1.0
    for _ in range(50):
        p0 = rng.uniform([0, 0], [nx, ny])
        p2 = rng.uniform([0, 0], [nx, ny])
        chord = p2 - p0
        L = math.hypot(*chord)
        perp = np.array([-chord[1], chord[0]]) / L
        p1 = (p0 + p2) / 2 + rng.uniform(-0.15, 0.15) * L * perp
        G, kdz = _one_ray_G(nx, ny, nz, dx, p0, p1, p2)
        cells, lengths, _, _ = _cell_lengths(G, kdz, nz)
        lp = math.hypot(*(p1 - p0)) + math.hypot(*(p2 - p1))
        N = max(1, math.ceil(4 * lp / dx))
        tau = np.arange(N + 1) / N
        a1, a2 = 2 * (p1 - p0), p0 - 2 * p1 + p2
        pts = p0[None, :] + tau[:, None] * a1[None, :] + (tau ** 2)[:, None] * a2[None, :]
        poly = np.sum(np.hypot(*np.diff(pts, axis=0).T))
        np.testing.assert_allclose(lengths.sum(), poly, rtol=1e-12)
        arc = integrate.quad(lambda t: math.hypot(*(a1 + 2 * t * a2)), 0, 1, epsabs=1e-13)[0]
        assert poly <= arc * (1 + 1e-12)
        assert arc - poly <= 0.02 * arc
        # every hit cell holds at least one sampled chord midpoint of the curve
        mids = 0.5 * (pts[1:] + pts[:-1])
        hh = (np.clip(np.floor(mids[:, 1]), 0, ny - 1) * nx + np.clip(np.floor(mids[:, 0]), 0, nx - 1))
        assert set(cells.tolist()) == set(hh.astype(int).tolist())


def test_depth_expansion_is_rank_one_per_row(tiny_system):
    """G[r, (h,k)] / Kdz[t(r), k] depends on h only (synthetic Eq. 5 form)."""
    p, G, _, _ = tiny_system
    for r in range(0, G.n_rows, 37):
        lo, hi = G.ptr[r], G.ptr[r + 1]
        k = G.idx[lo:hi] % p.nz
        ratio = (G.val[lo:hi] / p.kdz[p.row_period[r], k]).reshape(-1, p.nz)
        np.testing.assert_allclose(ratio, ratio[:, :1] * np.ones((1, p.nz)), rtol=1e-15)


def test_tiny_system_shape(tiny_system):
    p, G, GT, _ = tiny_system
    assert G.n_rows == 1520 and G.n_cols == 2048
    assert np.all(np.diff(G.ptr) % p.nz == 0)
    # straight rays: every period of a pair crosses the same cells
    cells = [tuple(G.idx[G.ptr[r]:G.ptr[r + 1]:p.nz]) for r in range(16)]
    assert cells[0] == cells[7] and cells[8] == cells[15]
    # straight-ray row sums of l equal the station distance
    for r in range(0, G.n_rows, 101):
        t = p.row_period[r]
        l = G.val[G.ptr[r]:G.ptr[r + 1]:p.nz] / p.kdz[t, 0]
        c = p.ctrl[r]
        np.testing.assert_allclose(l.sum(), math.hypot(c[4] - c[0], c[5] - c[1]), rtol=1e-12)


def test_transpose_matches_scipy(tiny_system):
    _, G, GT, _ = tiny_system
    ref = G.to_scipy().T.tocsr()
    ref.sort_indices()
    assert np.array_equal(GT.ptr, ref.indptr)
    assert np.array_equal(GT.idx, ref.indices)
    assert np.array_equal(GT.val, ref.data)


def test_spmv_matches_scipy(tiny_system):
    _, G, _, _ = tiny_system
    x = np.random.default_rng(3).standard_normal(G.n_cols)
    np.testing.assert_allclose(oracle.spmv(G, x), G.to_scipy() @ x, rtol=1e-13, atol=1e-12)


# ------------------------------------------------ laterally varying kernels

def test_lateral_values_are_length_times_cell_kernel():
    """With a depth kernel per horizontal cell, every value is the ray length
    in the cell times that cell's kernel: l_h comes from the same rays built
    with an all-ones kernel table (value = l_h * 1 exactly), then one
    multiplication by kdz_cells[h][t][k]."""
    from paper_2604_11920_b300 import synth
    p = synth.tiny_lateral()
    G = oracle.build_G_problem(p)
    ones = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period,
                          np.ones_like(p.kdz))
    assert np.array_equal(G.ptr, ones.ptr) and np.array_equal(G.idx, ones.idx)
    rows = np.repeat(np.arange(G.n_rows), np.diff(G.ptr))
    h, k = G.idx // p.nz, G.idx % p.nz
    want = ones.val * p.kdz_cells[h, p.row_period[rows], k]
    assert np.array_equal(G.val, want)
    # the separable table under the same rays gives other values
    sep = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period, p.kdz)
    assert not np.allclose(G.val, sep.val)


def test_lateral_kernels_break_separability():
    """Two cells of one row: the ratio of their depth profiles varies with
    depth when their kernels differ (it is constant in the separable case)."""
    from paper_2604_11920_b300 import synth
    p = synth.tiny_lateral()
    G = oracle.build_G_problem(p)
    nz = p.nz
    found = False
    for r in range(G.n_rows):
        a, b = G.ptr[r], G.ptr[r + 1]
        if b - a < 2 * nz:
            continue
        c0 = G.val[a:a + nz]
        c1 = G.val[a + nz:a + 2 * nz]
        ratio = c0 / c1
        if np.ptp(ratio) > 1e-3 * np.abs(ratio).max():
            found = True
            break
    assert found


# ------------------------------------------------ bilinear node coefficients

def test_bilinear_straight_ray_along_a_node_row():
    """Ray along the node row y = 1.5 of an 8 x 4 grid (dx = 1), x from 0 to 8:
    32 chords of 0.25 whose boundaries fall on the nodes, so the midpoint rule
    integrates each node's hat function exactly: every node of the row gets
    length 1 (the edge nodes take the clamped ends), the next row's nodes are
    touched with weight 0."""
    ctrl = np.array([[0.0, 1.5, 4.0, 1.5, 8.0, 1.5]])
    G = oracle.build_G(8, 4, 1, 1.0, ctrl, np.zeros(1, np.int32), np.ones((1, 1)), interp=1)
    vals = dict(zip(G.idx.tolist(), G.val.tolist()))
    for ix in range(8):
        assert abs(vals[1 * 8 + ix] - 1.0) <= 1e-14
        assert vals[2 * 8 + ix] == 0.0
    assert set(vals) == {1 * 8 + ix for ix in range(8)} | {2 * 8 + ix for ix in range(8)}


def test_bilinear_coefficients_partition_the_path():
    """The four weights of a chord sum to one, so each row's coefficients sum
    to the same total length as the cell form."""
    from paper_2604_11920_b300 import synth
    p = synth.tiny_bilinear()
    ones = np.ones_like(p.kdz)
    Gb = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period, ones, interp=1)
    Gc = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl, p.row_period, ones, interp=0)
    rb = np.add.reduceat(Gb.val, Gb.ptr[:-1]) / p.nz
    rc = np.add.reduceat(Gc.val, Gc.ptr[:-1]) / p.nz
    np.testing.assert_allclose(rb, rc, rtol=1e-12)
    # a band of nodes: more columns per row than the cell form
    assert Gb.nnz > 1.5 * Gc.nnz
    with pytest.raises(ValueError):
        oracle.build_G(1, 4, 1, 1.0, p.ctrl[:1], p.row_period[:1], ones, interp=1)
