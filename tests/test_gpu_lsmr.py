"""GPU parity of LSMR (Fong & Saunders 2011) against the FP64 LSMR oracle.

LSMR shares the Golub-Kahan sweeps with LSQR; only the scalar recurrence and
the x update differ.  Same bars as the LSQR tests: fixed-k FP64 iterates and
estimates to 1e-10 while the bidiagonalisation is orthogonal (k <= 8),
converged solutions to the parity bar, reduced-precision forms against the
tight-tolerance reference.
"""
import numpy as np
import pytest

import oracle
from oracle.lsmr import lsmr as oracle_lsmr
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

MODEL_TOL = 1e-4
RESID_TOL = 1e-6


@pytest.fixture(scope="module")
def tiny():
    require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "df64"))
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-12, btol=1e-12,
                      itmax=50000)
    return p, G, GT, d, h, ref


def residual_norm(p, G, m, d, lam):
    Am = oracle.apply_A(G, (p.nx, p.ny, p.nz), p.w, m)
    r = np.concatenate([d, np.zeros(p.n)]) - Am
    return np.sqrt(r @ r + lam * lam * (m @ m))


@pytest.mark.parametrize("fmt", ["element", "blocked"])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fixed_k_lsmr_fp64(tiny, fmt, k):
    p, G, GT, d, h, _ = tiny
    ref = oracle_lsmr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                      itmax=k)
    res = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, fmt=fmt, conlim=1e300, method="lsmr")
    assert res.info["iters"] == k and res.info["istop"] == 7
    assert rel(res.m.cpu().numpy(), ref.x) < 1e-10
    for key in ("rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm"):
        assert abs(res.info[key] - getattr(ref, key)) <= 1e-10 * abs(getattr(ref, key)), key


@pytest.mark.parametrize("k", [2, 8])
def test_fixed_k_lsmr_scaled(tiny, k):
    """Right scaling D = 1/||augmented column|| with explicit lambda rows."""
    p, G, GT, d, h, _ = tiny
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    ref = oracle_lsmr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, d, atol=0, btol=0, conlim=0,
                      itmax=k, D=D, lam_rows=p.lam)
    h.set_col_scaling(None, p.w, p.lam)
    res = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, fmt="blocked", precond=1, conlim=1e300,
                 method="lsmr")
    assert rel(res.m.cpu().numpy(), D * ref.x) < 1e-9
    assert abs(res.info["arnorm"] - ref.arnorm) <= 1e-9 * ref.arnorm


@pytest.mark.parametrize("fmt", ["element", "blocked"])
def test_converged_lsmr_fp64(tiny, fmt):
    p, G, GT, d, h, ref = tiny
    res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-10, fmt=fmt, method="lsmr")
    assert res.info["istop"] in (1, 2)
    assert rel(res.m.cpu().numpy(), ref.x) <= MODEL_TOL
    r_gpu = residual_norm(p, G, res.m.cpu().numpy(), d, p.lam)
    r_ref = residual_norm(p, G, ref.x, d, p.lam)
    assert abs(r_gpu - r_ref) / r_ref <= RESID_TOL
    # same iteration count as the oracle's LSMR at the same tolerance
    o = oracle_lsmr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-10, btol=1e-10,
                    itmax=50000)
    assert abs(res.info["iters"] - o.itn) <= max(3, 0.02 * o.itn)


@pytest.mark.parametrize("dtype", ["f32", "df64"])
def test_reduced_and_double_float_lsmr(tiny, dtype):
    p, G, GT, d, h, ref = tiny
    res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-6, dtype=dtype, fmt="blocked",
                 method="lsmr")
    assert res.info["istop"] in (1, 2)
    e = rel(res.m.cpu().numpy(), ref.x)
    f64 = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-6, fmt="blocked", method="lsmr")
    e64 = rel(f64.m.cpu().numpy(), ref.x)
    print(f"LSMR {dtype}: {res.info['iters']} it, error {e:.2e} (FP64 at the same tol {e64:.2e})")
    assert e <= 2 * e64 + 5e-3


def test_lsmr_two_phase_refinement(tiny):
    p, G, GT, d, h, ref = tiny
    h.set_col_scaling(None, p.w, p.lam)
    res = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype="f32", fmt="blocked", precond=1,
                 refine=3, refine_dtype="df64", refine_tol=1e-10, method="lsmr")
    assert res.info["sweeps"] >= 2
    assert rel(res.m.cpu().numpy(), ref.x) <= 1e-6


def test_lsmr_graph_and_plain_identical(tiny):
    p, G, GT, d, h, _ = tiny
    a = h.lsqr(to_dev(d), p.w, p.lam, 300, 1e-8, fmt="blocked", method="lsmr")
    b = h.lsqr(to_dev(d), p.w, p.lam, 300, 1e-8, fmt="blocked", method="lsmr", use_graph=False)
    assert a.info["iters"] == b.info["iters"]
    assert np.array_equal(a.m.cpu().numpy(), b.m.cpu().numpy())


def test_lsmr_errors(tiny):
    p, G, GT, d, h, _ = tiny
    with pytest.raises(pdst.PdstError):
        h.lsqr(to_dev(d), p.w, p.lam, 10, 1e-6, method=5)
    import torch
    m = torch.empty(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(pdst.PdstError):
        h.lsqr_noalloc(to_dev(d), p.w, p.lam, 10, 1e-6, m, method="lsmr")
