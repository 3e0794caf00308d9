"""Oracle parity on the 64 x 64 x 16 workload itself (171,360 rows, 65,536
unknowns, 113,560,864 stored entries): the system the benchmark times.

These tests run the kernel paths the benchmark runs -- the compile-time
4-entry-quad forward for 16 depth nodes (quads of 4), the blocked adjoint with
cells split over several work items, the column-scaled operator with lambda
rows -- against the FP64 CPU oracle built from the same seeded inputs:

* LSQR iterates at a fixed iteration count k (Paige & Saunders 1982), element
  by element, with the oracle's G, G^T and d (bars: 1e-10 for FP64 values,
  1e-9 double-float, 1e-4 FP32, 3e-2 BF16, unscaled and column-scaled);
* the converged solutions against the oracle's own tol-1e-12 solution stored
  in tests/golden/mid_mref.npy (written by tests/golden/make_mref.py,
  which calls only the oracle): the plain FP64 form and the two-phase FP32
  form, the benchmark's accuracy-matched path, within 1e-4 relative model
  error, and the relative residual difference within 1e-6.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MODEL_TOL = 1e-4
RESID_TOL = 1e-6
BARS = (("f64", "element", 1e-10), ("f64", "blocked", 1e-10), ("df64", "blocked", 1e-9),
        ("f32", "blocked", 1e-4), ("bf16", "blocked", 3e-2))


@pytest.fixture(scope="module")
def mid():
    require_cuda()
    p = synth.mid()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16", "df64"))
    assert h.nnz == G.nnz == 113560864
    yield p, G, GT, d, h
    h.close()


def aug_residual(p, G, m, d):
    """||[d; 0; 0] - [G; w L; lambda I] m|| evaluated by the oracle."""
    Am = oracle.apply_A(G, (p.nx, p.ny, p.nz), p.w, m)
    r = np.concatenate([d, np.zeros(p.n)]) - Am
    return float(np.sqrt(r @ r + p.lam * p.lam * (m @ m)))


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fixed_k_iterates_mid(mid, k):
    p, G, GT, d, h = mid
    grid = (p.nx, p.ny, p.nz)
    ref = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0, btol=0, conlim=0, itmax=k)
    dd = to_dev(d)
    for dt, fm, bar in BARS:
        r = h.lsqr(dd, p.w, p.lam, k, 0.0, dtype=dt, fmt=fm, conlim=1e300)
        assert r.info["iters"] == k and r.info["istop"] == 7
        e = rel(r.m.cpu().numpy(), ref.x)
        print(f"k={k} {dt}/{fm}: {e:.2e}")
        assert e < bar, (k, dt, fm, e)
        if dt == "f64":
            for key in ("rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm"):
                assert abs(r.info[key] - getattr(ref, key)) <= bar * abs(getattr(ref, key)), key


@pytest.mark.parametrize("k", [1, 3, 8])
def test_fixed_k_iterates_mid_column_scaled(mid, k):
    """The scaled operator [G D; w L D; lambda D] with the oracle's column norms
    as D (so both sides apply the same operator) and with the device's own
    column norms, which must equal the oracle's to rounding."""
    p, G, GT, d, h = mid
    grid = (p.nx, p.ny, p.nz)
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    c = h.col_norms(p.w, p.lam).cpu().numpy()
    assert np.max(np.abs(c * D - 1.0)) < 1e-13
    ref = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=k, D=D,
                      lam_rows=p.lam)
    dd = to_dev(d)
    h.set_col_scaling(to_dev(D))
    for dt, fm, bar in BARS:
        r = h.lsqr(dd, p.w, p.lam, k, 0.0, dtype=dt, fmt=fm, precond=1, conlim=1e300)
        e = rel(r.m.cpu().numpy(), D * ref.x)
        print(f"k={k} scaled {dt}/{fm}: {e:.2e}")
        assert e < bar, (k, dt, fm, e)
    h.set_col_scaling(None, p.w, p.lam)
    r = h.lsqr(dd, p.w, p.lam, k, 0.0, dtype="f64", fmt="blocked", precond=1, conlim=1e300)
    assert rel(r.m.cpu().numpy(), D * ref.x) < 1e-10


def test_converged_mid_matches_oracle_mref(mid):
    """Plain FP64 GPU LSQR at tol 1e-12 and the two-phase FP32 form (the
    benchmark's accuracy-matched path: FP32 solve to 1e-6, then FP32
    refinement sweeps on the FP64 residual) against the oracle's solution."""
    p, G, GT, d, h = mid
    m_ref = np.load(os.path.join(GOLDEN, "mid_mref.npy"))
    r_ref = aug_residual(p, G, m_ref, d)
    dd = to_dev(d)
    f64 = h.lsqr(dd, p.w, p.lam, 100000, 1e-12, dtype="f64", fmt="blocked")
    assert f64.info["istop"] in (1, 2)
    e64 = rel(f64.m.cpu().numpy(), m_ref)
    h.set_col_scaling(None, p.w, p.lam)
    two = h.lsqr(dd, p.w, p.lam, 100000, p.tol, dtype="f32", fmt="blocked", precond=1,
                 refine=3, refine_dtype="f32", refine_tol=3e-9)
    e2 = rel(two.m.cpu().numpy(), m_ref)
    one = h.lsqr(dd, p.w, p.lam, 100000, p.tol, dtype="f32", fmt="blocked", precond=1)
    e1 = rel(one.m.cpu().numpy(), m_ref)
    print(f"FP64 tol 1e-12: {e64:.2e} ({f64.info['iters']} it); FP32 one solve {e1:.2e}; "
          f"two-phase {e2:.2e} ({two.info['sweeps']} sweeps, {two.info['iters']} it)")
    assert e64 <= 1e-6
    assert e2 <= MODEL_TOL and e1 > 1e-3
    for m in (f64.m, two.m):
        assert abs(aug_residual(p, G, m.cpu().numpy(), d) - r_ref) / r_ref <= RESID_TOL
