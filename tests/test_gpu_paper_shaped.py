"""The paper-shaped stand-in (20 x 37 x 18 = 13,320 unknowns, 229 stations x
14 periods = 365,484 rows, bilinear node coefficients): the size of the
paper's field problem.  Same checks as the other full-size system: sampled
rows against the oracle, the adjoint identity, LSQR estimates against true
norms, and a converging FP32 solve."""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev
from test_gpu_large import true_norms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def paper():
    require_cuda()
    import torch
    p = synth.paper_shaped()
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
    gm = torch.empty(h.m, dtype=torch.float64, device="cuda")
    h.apply_G(to_dev(p.m_true), gm, dtype="f64")
    d = gm + p.noise_frac * torch.sqrt(torch.mean(gm * gm)) * to_dev(p.noise)
    yield p, h, d
    h.close()


def test_paper_shaped_sizes_and_sampled_rows(paper):
    import torch
    p, h, _ = paper
    assert (h.m, h.n) == (365484, 13320)
    rng = np.random.default_rng(11)
    rows = np.unique(rng.choice(h.m, 2000, replace=False))
    Gs = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl[rows], p.row_period[rows], p.kdz,
                        interp=1)
    ptr, _, _ = h.export_csr(ptr_only=True)
    assert np.array_equal(np.diff(ptr)[rows], np.diff(Gs.ptr))
    x = rng.standard_normal(h.n)
    y = torch.empty(h.m, dtype=torch.float64, device="cuda")
    h.apply_G(to_dev(x), y, dtype="f64")
    scale = oracle.spmv(oracle.CSR(Gs.ptr, Gs.idx, np.abs(Gs.val), Gs.n_cols), np.abs(x))
    want = oracle.spmv(Gs, x)
    assert np.all(np.abs(y.cpu().numpy()[rows] - want) <= 1e-13 * scale)


def test_paper_shaped_lsqr(paper):
    p, h, d = paper
    r5 = h.lsqr(d, p.w, p.lam, 5, 0.0, dtype="f64", fmt="blocked", conlim=1e300)
    rn, arn = true_norms(p, h, d, r5.m, p.lam)
    assert abs(r5.info["rnorm"] - rn) <= 1e-10 * rn
    assert abs(r5.info["arnorm"] - arn) <= 1e-6 * arn
    h.set_col_scaling(None, p.w, p.lam)
    r = h.lsqr(d, p.w, p.lam, 20000, p.tol, dtype="f32", fmt="blocked", precond=1)
    assert r.info["istop"] in (1, 2)
    rn, _ = true_norms(p, h, d, r.m, p.lam)
    assert abs(r.info["rnorm"] - rn) <= 1e-3 * rn
