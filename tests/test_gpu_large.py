"""Full-size checks on the 100 x 100 x 20 system (200,000 unknowns, 240 stations,
28,680 pairs x 30 periods = 860,400 rows, about 1.1e9 stored entries).

The oracle cannot hold this G and its transpose in a test's time, so it is
used where it computes outputs one by one, and the rest is checked through
properties that hold at any size:

* assembly: sampled rows (rows are independent: the oracle builds just those
  paths) have the same cell runs, and (G x)_r on the device equals the
  oracle row times x to FP64 rounding, for FP64 and FP32 values;
* adjoint: <G v, u> = <v, G^T u> for non-negative u, v (G >= 0, no
  cancellation) to 1e-12;
* LSQR: after k steps the reported ||r|| and ||A^T r|| equal the true ones
  recomputed from the iterate with the (checked) FP64 products and the
  oracle's Laplacian; the FP32 sweeps track the FP64 ones; a full FP32
  column-scaled solve to tol 1e-6 stops on S1/S2, reports its true residual
  norm, and ends below the residual of an early iterate.
"""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    require_cuda()
    import torch
    p = synth.large()
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
    mt = to_dev(p.m_true)
    gm = torch.empty(h.m, dtype=torch.float64, device="cuda")
    h.apply_G(mt, gm, dtype="f64")
    rms = torch.sqrt(torch.mean(gm * gm))
    d = gm + p.noise_frac * rms * to_dev(p.noise)
    yield p, h, d
    h.close()


def test_large_sizes(large):
    p, h, _ = large
    assert (p.nx, p.ny, p.nz) == (100, 100, 20)
    assert h.m == 28680 * 30 == p.m_rows and h.n == 200000
    assert h.nnz > 5e8          # about 1.1e9 with this seed


def test_large_sampled_rows_match_oracle(large):
    import torch
    p, h, _ = large
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.choice(h.m, 3000, replace=False), [0, h.m - 1]]))
    Gs = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl[rows], p.row_period[rows], p.kdz)
    ptr, _, _ = h.export_csr(ptr_only=True)
    assert ptr[-1] == h.nnz
    assert np.array_equal(np.diff(ptr)[rows], np.diff(Gs.ptr))
    x = rng.standard_normal(h.n)
    absx = np.abs(x)
    scale = oracle.spmv(oracle.CSR(Gs.ptr, Gs.idx, np.abs(Gs.val), Gs.n_cols), absx)
    for dt, vals in (("f64", Gs.val), ("f32", Gs.val.astype(np.float32).astype(np.float64))):
        y = torch.empty(h.m, dtype=torch.float64, device="cuda")
        h.apply_G(to_dev(x), y, dtype=dt)
        want = oracle.spmv(oracle.CSR(Gs.ptr, Gs.idx, vals, Gs.n_cols), x)
        got = y.cpu().numpy()[rows]
        assert np.all(np.abs(got - want) <= 1e-13 * scale), dt


def test_large_adjoint_identity(large):
    import torch
    p, h, _ = large
    rng = np.random.default_rng(8)
    v = to_dev(rng.uniform(0.0, 1.0, h.n))
    u = to_dev(rng.uniform(0.0, 1.0, h.m))
    gv = torch.empty(h.m, dtype=torch.float64, device="cuda")
    gtu = torch.empty(h.n, dtype=torch.float64, device="cuda")
    for dt in ("f64", "f32"):
        h.apply_G(v, gv, dtype=dt)
        h.apply_G(u, gtu, trans=True, dtype=dt)
        a = float(torch.dot(gv, u))
        b = float(torch.dot(v, gtu))
        assert a > 0 and abs(a - b) <= 1e-12 * a, dt


def true_norms(p, h, d, m, lam):
    """||r|| and ||A^T r|| of the damped augmented problem at m, from the
    FP64 device products and the oracle Laplacian."""
    import torch
    grid = (p.nx, p.ny, p.nz)
    gm = torch.empty(h.m, dtype=torch.float64, device="cuda")
    h.apply_G(m, gm, dtype="f64")
    r1 = d - gm
    mh = m.cpu().numpy()
    lm = oracle.laplacian(*grid, mh)
    r2 = -p.w * lm
    rn = np.sqrt(float(torch.dot(r1, r1)) + r2 @ r2 + lam * lam * (mh @ mh))
    gtr = torch.empty(h.n, dtype=torch.float64, device="cuda")
    h.apply_G(r1, gtr, trans=True, dtype="f64")
    atr = gtr.cpu().numpy() + p.w * oracle.laplacian(*grid, r2) - lam * lam * mh
    return rn, float(np.linalg.norm(atr))


@pytest.mark.parametrize("k", [3, 6])
def test_large_lsqr_estimates_match_true_norms(large, k):
    p, h, d = large
    r64 = h.lsqr(d, p.w, p.lam, k, 0.0, dtype="f64", fmt="blocked", conlim=1e300)
    assert r64.info["iters"] == k
    rn, arn = true_norms(p, h, d, r64.m, p.lam)
    assert abs(r64.info["rnorm"] - rn) <= 1e-10 * rn
    assert abs(r64.info["arnorm"] - arn) <= 1e-6 * arn
    r32 = h.lsqr(d, p.w, p.lam, k, 0.0, dtype="f32", fmt="blocked", conlim=1e300)
    assert rel(r32.m.cpu().numpy(), r64.m.cpu().numpy()) <= 1e-4


def test_large_fp32_solve_to_tol(large):
    p, h, d = large
    h.set_col_scaling(None, p.w, p.lam)
    r = h.lsqr(d, p.w, p.lam, 20000, p.tol, dtype="f32", fmt="blocked", precond=1)
    assert r.info["istop"] in (1, 2) and r.info["iters"] < 20000
    rn, arn = true_norms(p, h, d, r.m, p.lam)
    assert abs(r.info["rnorm"] - rn) <= 1e-3 * rn
    # the stopping tests ran on the scaled operator A D; the unscaled ratio
    # ||A^T r|| / (||A_D||_F ||r||) is only bounded loosely here
    bn = r.info["bnorm"]
    assert rn <= bn
    s2 = arn / (r.info["anorm"] * rn)
    print(f"large FP32 solve: {r.info['iters']} it, istop {r.info['istop']}, "
          f"true ||A^T r|| / (||A|| ||r||) = {s2:.2e}")
    assert s2 <= 1e-2
    # LSQR's residual norm decreases monotonically: below the 6-step iterate's
    k6 = h.lsqr(d, p.w, p.lam, 6, 0.0, dtype="f64", fmt="blocked", conlim=1e300)
    assert rn < true_norms(p, h, d, k6.m, p.lam)[0]
