"""Depth-block right preconditioner (precond = 2) on the GPU against the oracle.

* B_h = A_h^T A_h from pdst_depth_blocks against oracle/blockprec.py (FP64,
  summation order only), on grids with edge and corner cells, odd depth
  counts, laterally varying kernels and bilinear node coefficients, and on
  sampled cells of the 64 x 64 x 16 workload;
* P_h = R_h^{-1} from pdst_set_block_precond against the oracle's inverse
  Cholesky factors of its own blocks;
* LSQR on [G P; w L P; lam P] at a fixed iteration count, with the oracle's
  P given to the device, against the oracle's block-preconditioned LSQR,
  element by element (FP64 1e-10, FP32 1e-4);
* converged solves against the oracle's minimiser, including the two-phase
  FP32 form on the 64 x 64 x 16 workload against its stored tol-1e-12
  solution (1e-4 relative model error, 1e-6 relative residual difference);
* the host-side errors of the new calls.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import blockprec
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _system(p, dtypes=("f64", "f32")):
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=dtypes)
    return G, GT, d, h


SMALL = [("tiny", lambda: synth.tiny()),
         ("lateral", lambda: synth.tiny_lateral()),
         ("bilinear", lambda: synth.tiny_bilinear()),
         ("ragged_5x7x5", lambda: synth.custom(5, 7, 5, 9, 3, bend=0.12, seed=21)),
         ("one_depth", lambda: synth.custom(9, 4, 1, 8, 4, bend=0.1, seed=22))]


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_depth_blocks_and_factors_match_oracle(name, make):
    require_cuda()
    p = make()
    G, GT, d, h = _system(p)
    grid = (p.nx, p.ny, p.nz)
    B_ref = blockprec.depth_blocks(GT, grid, p.w, p.lam)
    B = h.depth_blocks(p.w, p.lam).cpu().numpy()
    scale = np.abs(B_ref).reshape(len(B_ref), -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(B - B_ref) / scale) < 1e-13
    P_ref = blockprec.inverse_cholesky(B_ref)
    h.set_block_precond(None, p.w, p.lam)
    P = h.get_block_precond().cpu().numpy()
    assert np.all(np.tril(P, -1) == 0.0)
    pscale = np.abs(P_ref).reshape(len(P_ref), -1).max(axis=1)[:, None, None]
    err = np.max(np.abs(P - P_ref) / pscale)
    print(f"{name}: B ok, P max rel {err:.1e}")
    assert err < 1e-9
    h.close()


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_fixed_k_iterates_with_oracle_blocks(tiny_system, k):
    """The oracle's P given to the device: both sides apply the same operator."""
    require_cuda()
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    P = blockprec.block_precond(GT, grid, p.w, p.lam)
    ref = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=k, P=P,
                      lam_rows=p.lam)
    m_ref = blockprec.apply_blocks(P, ref.x)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16"))
    h.set_block_precond(to_dev(P), p.w, p.lam)
    dd = to_dev(d)
    for dt, bar in (("f64", 1e-10), ("f32", 1e-4), ("bf16", 3e-2)):
        r = h.lsqr(dd, p.w, p.lam, k, 0.0, dtype=dt, fmt="blocked", precond=2, conlim=1e300)
        assert r.info["iters"] == k and r.info["istop"] == 7
        e = rel(r.m.cpu().numpy(), m_ref)
        print(f"k={k} {dt}: {e:.2e}")
        assert e < bar, (dt, e)
        if dt == "f64":
            for key in ("rnorm", "arnorm", "anorm", "xnorm", "bnorm"):
                assert abs(r.info[key] - getattr(ref, key)) <= 1e-10 * abs(getattr(ref, key)), key
    h.close()


def test_converged_block_solve_reaches_the_minimiser(tiny_system):
    """FP64 at tol 1e-10 and the two-phase FP32 form with the device's own
    blocks reach the oracle's unpreconditioned tol-1e-12 minimiser, the FP64
    form in fewer iterations than column-norm scaling; LSMR runs on the same
    preconditioned operator."""
    require_cuda()
    p, G, GT, d = tiny_system
    grid = (p.nx, p.ny, p.nz)
    m_ref = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=1e-12, btol=1e-12, itmax=50000).x
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"))
    dd = to_dev(d)
    h.set_block_precond(None, p.w, p.lam)
    blk = h.lsqr(dd, p.w, p.lam, 20000, 1e-10, dtype="f64", fmt="blocked", precond=2)
    assert blk.info["istop"] in (1, 2)
    assert rel(blk.m.cpu().numpy(), m_ref) < 1e-7
    two = h.lsqr(dd, p.w, p.lam, 20000, 1e-6, dtype="f32", fmt="blocked", precond=2, refine=3,
                 refine_dtype="f32", refine_tol=1e-9)
    assert rel(two.m.cpu().numpy(), m_ref) < 1e-6
    lsmr = h.lsqr(dd, p.w, p.lam, 20000, 1e-10, dtype="f64", fmt="blocked", precond=2,
                  method="lsmr")
    assert rel(lsmr.m.cpu().numpy(), m_ref) < 1e-6
    h.set_col_scaling(None, p.w, p.lam)
    col = h.lsqr(dd, p.w, p.lam, 20000, 1e-10, dtype="f64", fmt="blocked", precond=1)
    print(f"iterations to 1e-10: blocks {blk.info['iters']}, column norms {col.info['iters']}")
    assert blk.info["iters"] < col.info["iters"]
    h.close()


def test_block_precond_errors(tiny_system):
    require_cuda()
    import torch
    p, G, GT, d = tiny_system
    h = pdst.build_G_problem(p, dtypes=("f64", "df64"))
    dd = to_dev(d)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        h.lsqr(dd, p.w, p.lam, 10, 1e-6, fmt="blocked", precond=2)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        h.get_block_precond()
    h.set_block_precond(None, p.w, p.lam)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr(dd, p.w, p.lam, 10, 1e-6, fmt="element", precond=2)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr(dd, p.w, p.lam, 10, 1e-6, dtype="df64", fmt="blocked", precond=2)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.set_block_precond(None, -1.0, p.lam)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr_noalloc(dd, p.w, p.lam, 10, 1e-6, torch.zeros(h.n, dtype=torch.float64,
                                                             device="cuda"), precond=2)
    h.close()
    # a cell that no ray crosses, with w = lambda = 0: B_h = 0 is not positive definite
    q = synth.custom(12, 12, 4, 3, 2, bend=0.0, seed=5)
    hq = pdst.build_G_problem(q, dtypes=("f64",))
    with pytest.raises(pdst.PdstError, match="PDST_ERR_BREAKDOWN"):
        hq.set_block_precond(None, 0.0, 0.0)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        hq.lsqr(to_dev(np.zeros(hq.m)), 0.0, 0.0, 10, 1e-6, fmt="blocked", precond=2)
    hq.set_block_precond(None, 0.0, 0.1)    # lambda > 0 makes every block definite
    hq.close()
    # nz > 32
    r = synth.custom(3, 3, 34, 4, 2, bend=0.0, seed=6)
    hr = pdst.build_G_problem(r, dtypes=("f64",))
    with pytest.raises(pdst.PdstError, match="PDST_ERR_LIMIT"):
        hr.set_block_precond(None, 1.0, 0.1)
    hr.close()


@pytest.fixture(scope="module")
def mid():
    require_cuda()
    p = synth.mid()
    G, GT, d, h = _system(p, dtypes=("f64", "f32"))
    yield p, G, GT, d, h
    h.close()


def test_mid_sampled_blocks(mid):
    p, G, GT, d, h = mid
    cells = [0, 63, 1000, 2080, 4095]
    B_ref = blockprec.depth_blocks(GT, (p.nx, p.ny, p.nz), p.w, p.lam, cells=cells)
    B = h.depth_blocks(p.w, p.lam).cpu().numpy()[cells]
    scale = np.abs(B_ref).reshape(len(cells), -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(B - B_ref) / scale) < 1e-12


def test_mid_two_phase_block_form_matches_oracle_mref(mid):
    """The two-phase FP32 form with the device's blocks against the oracle's
    tol-1e-12 solution of the 64 x 64 x 16 system."""
    p, G, GT, d, h = mid
    m_ref = np.load(os.path.join(GOLDEN, "mid_mref.npy"))
    Am = oracle.apply_A(G, (p.nx, p.ny, p.nz), p.w, m_ref)
    r_ref = float(np.sqrt(np.sum((np.concatenate([d, np.zeros(p.n)]) - Am) ** 2)
                          + p.lam ** 2 * (m_ref @ m_ref)))
    h.set_block_precond(None, p.w, p.lam)
    two = h.lsqr(to_dev(d), p.w, p.lam, 100000, p.tol, dtype="f32", fmt="blocked", precond=2,
                 refine=3, refine_dtype="f32", refine_tol=3e-9)
    m = two.m.cpu().numpy()
    e = rel(m, m_ref)
    Am2 = oracle.apply_A(G, (p.nx, p.ny, p.nz), p.w, m)
    r2 = float(np.sqrt(np.sum((np.concatenate([d, np.zeros(p.n)]) - Am2) ** 2)
                       + p.lam ** 2 * (m @ m)))
    print(f"mid block two-phase: {e:.2e} ({two.info['sweeps']} sweeps, {two.info['iters']} it)")
    assert e <= 1e-4
    assert abs(r2 - r_ref) / r_ref <= 1e-6


def test_empty_cells_and_zero_damping():
    """Most cells crossed by no ray and lambda = 0 (no lambda rows): the
    device's blocks equal the oracle's and the FP64 and two-phase FP32 block
    solves reach the oracle's tol-1e-12 solution."""
    require_cuda()
    p = synth.custom(12, 12, 4, 3, 2, bend=0.0, seed=5, w=1.0, lam=0.0)
    G, GT, d, h = _system(p)
    grid = (p.nx, p.ny, p.nz)
    B_ref = blockprec.depth_blocks(GT, grid, p.w, 0.0)
    B = h.depth_blocks(p.w, 0.0).cpu().numpy()
    scale = np.abs(B_ref).reshape(len(B_ref), -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(B - B_ref) / scale) < 1e-13
    ref = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=1e-12, btol=1e-12, itmax=50000)
    h.set_block_precond(None, p.w, 0.0)
    dd = to_dev(d)
    r64 = h.lsqr(dd, p.w, 0.0, 20000, 1e-11, dtype="f64", fmt="blocked", precond=2)
    assert r64.info["istop"] in (1, 2)
    assert rel(r64.m.cpu().numpy(), ref.x) < 1e-7
    two = h.lsqr(dd, p.w, 0.0, 20000, 1e-6, dtype="f32", fmt="blocked", precond=2, refine=3,
                 refine_dtype="f32", refine_tol=1e-10)
    assert rel(two.m.cpu().numpy(), ref.x) < 1e-6
    h.close()


@pytest.mark.parametrize("nz", [17, 18, 20, 32])
def test_fixed_k_iterates_deep_columns(nz):
    """Depth counts above 16 (the finish without the half-warp split; 18 and 20
    are the paper-shaped and 100 x 100 x 20 systems' depth counts, 32 the
    largest the blocks support): the device's blocks and, with the oracle's
    blocks given to it, FP64 and FP32 iterates at a fixed k against the
    oracle's."""
    require_cuda()
    p = synth.custom(7, 6, nz, 9, 3, bend=0.15, seed=70 + nz, w=1.0, lam=0.1, dz_km=1.0)
    G, GT, d, h = _system(p)
    grid = (p.nx, p.ny, p.nz)
    B_ref = blockprec.depth_blocks(GT, grid, p.w, p.lam)
    B = h.depth_blocks(p.w, p.lam).cpu().numpy()
    scale = np.abs(B_ref).reshape(len(B_ref), -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(B - B_ref) / scale) < 1e-13
    P = blockprec.inverse_cholesky(B_ref)
    h.set_block_precond(to_dev(P), p.w, p.lam)
    dd = to_dev(d)
    for k in (1, 6):
        ref = oracle.lsqr(G, GT, grid, p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=k, P=P,
                          lam_rows=p.lam)
        m_ref = blockprec.apply_blocks(P, ref.x)
        for dt, bar in (("f64", 1e-10), ("f32", 1e-4)):
            r = h.lsqr(dd, p.w, p.lam, k, 0.0, dtype=dt, fmt="blocked", precond=2, conlim=1e300)
            assert r.info["iters"] == k
            assert rel(r.m.cpu().numpy(), m_ref) < bar, (nz, k, dt)
    h.close()
