"""The outer nonlinear loop on the GPU (pdst_depth_kernels_from_model,
pdst_set_depth_kernels, pdst_outer_loop) against the FP64 oracle of the loop
(oracle/outer.py): the paragraph after Eq. 6 -- solve Eq. 6 for the update,
rebuild G from the updated model, stop on the RMS traveltime misfit.

Bars: the kernel table and G's values within a few ulp (the device's exp and
the host's may differ in the last bit; everything else rounds the same);
index arrays bit-exact; the loop at a fixed inner iteration count within the
FP64 fixed-k bar (1e-10) on the model and 1e-12 on the RMS history; converged
loops within the parity bar.
"""
import numpy as np
import pytest

import oracle
from oracle import outer
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def problem():
    return synth.custom(14, 12, 8, 16, 5, bend=0.15, seed=71, w=0.5, lam=0.05, dz_km=2.0)


@pytest.fixture(scope="module")
def sysm():
    require_cuda()
    p = problem()
    m_true = synth.checkerboard(p.nx, p.ny, p.nz, 3, 0.08)
    f = outer.forward(p, m_true)
    d_obs = f + 0.01 * np.sqrt(np.mean(f * f)) * p.noise
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "df64"), keep_lengths=True)
    yield p, m_true, d_obs, h
    h.close()


def test_kernel_table_matches_oracle(sysm):
    p, m_true, d_obs, h = sysm
    rng = np.random.default_rng(8)
    m = rng.uniform(-0.1, 0.1, p.n)
    for kp in (1.0, 0.0, 0.5):
        got = h.depth_kernels_from_model(p.periods_s, to_dev(m), 1.2, kp).cpu().numpy()
        ref = outer.kernel_table(p.periods_s, p.nx, p.ny, p.nz, p.dz_km, m, 1.2, kp)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 4e-16 * 8, kp


def test_set_depth_kernels_rebuilds_every_copy(sysm):
    p, m_true, d_obs, h = sysm
    rng = np.random.default_rng(9)
    m = rng.uniform(-0.1, 0.1, p.n)
    K = h.depth_kernels_from_model(p.periods_s, to_dev(m))
    h.set_depth_kernels(K)
    Gm = outer.G_of_model(p, m)
    ptr, idx, v64 = h.export_csr("f64")
    assert np.array_equal(ptr, Gm.ptr) and np.array_equal(idx, Gm.idx)
    assert np.max(np.abs(v64 - Gm.val) / np.maximum(np.abs(Gm.val), 1e-300)) < 4e-15
    _, _, v32 = h.export_csr("f32")
    assert np.array_equal(v32, v64.astype(np.float32).astype(np.float64))
    GT = oracle.transpose(Gm)
    cptr, cidx, c64 = h.export_csc("f64")
    assert np.array_equal(cptr, GT.ptr) and np.array_equal(cidx, GT.idx)
    assert np.max(np.abs(c64 - GT.val) / np.maximum(np.abs(GT.val), 1e-300)) < 4e-15
    _, _, cdf = h.export_csc("df64")
    assert np.all(np.abs(cdf - c64) <= 2.0 ** -48 * np.abs(c64))
    # the host's 1-D table, one copy per cell, gives back the assembly's values bit for bit
    K1 = np.broadcast_to(p.kdz, (p.nx * p.ny,) + p.kdz.shape).copy()
    h.set_depth_kernels(to_dev(K1))
    _, _, back = h.export_csr("f64")
    assert np.array_equal(back, oracle.build_G_problem(p).val)


def test_outer_loop_fixed_inner_iterations_match_oracle(sysm):
    p, m_true, d_obs, h = sysm
    k = 6
    ref = outer.outer_loop(p, d_obs, p.w, p.lam, itmax=k, tol=0.0, max_outer=3, rms_tol=0.0,
                           min_decrease=0.0)
    for fmt in ("element", "blocked"):
        m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, k, 0.0,
                                     max_outer=3, rms_tol=0.0, min_decrease=0.0, fmt=fmt,
                                     conlim=1e300)
        assert info["updates"] == ref.updates == 3 and info["reason"] == ref.reason == 3
        assert info["inner_iters"] == 3 * k
        assert np.max(np.abs(hist - ref.rms) / np.array(ref.rms)) < 1e-12
        assert rel(m.cpu().numpy(), ref.m) < 1e-10, fmt


def test_outer_loop_converged_match_oracle(sysm):
    p, m_true, d_obs, h = sysm
    ref = outer.outer_loop(p, d_obs, p.w, p.lam, itmax=5000, tol=1e-10, max_outer=6,
                           rms_tol=0.0, min_decrease=0.02)
    m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 5000, 1e-10,
                                 max_outer=6, rms_tol=0.0, min_decrease=0.02, fmt="blocked")
    print(f"oracle: {ref.updates} updates, reason {ref.reason}, RMS {ref.rms}; "
          f"GPU: {info}, RMS {list(hist)}")
    assert info["updates"] == ref.updates and info["reason"] == ref.reason
    assert np.max(np.abs(hist - ref.rms) / np.array(ref.rms)) < 1e-8
    assert rel(m.cpu().numpy(), ref.m) < 1e-6
    assert hist[-1] < 0.5 * hist[0]
    # the loop recovers the planted model better than its first update does
    first = outer.outer_loop(p, d_obs, p.w, p.lam, 5000, 1e-10, max_outer=1, rms_tol=0.0,
                             min_decrease=0.0)
    assert rel(m.cpu().numpy(), m_true) < rel(first.m, m_true)


def test_outer_loop_fp32_scaled_inner_solves(sysm):
    """The chosen form inside the loop (FP32 values, column-norm scaling of each
    rebuilt G, two-phase refinement): the same model as the FP64 oracle loop
    within the parity bar."""
    p, m_true, d_obs, h = sysm
    ref = outer.outer_loop(p, d_obs, p.w, p.lam, itmax=5000, tol=1e-10, max_outer=4,
                           rms_tol=0.0, min_decrease=0.0)
    m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 5000, 1e-6,
                                 max_outer=4, rms_tol=0.0, min_decrease=0.0, dtype="f32",
                                 fmt="blocked", precond=1, refine=3, refine_dtype="f32",
                                 refine_tol=1e-10)
    assert info["updates"] == 4
    assert rel(m.cpu().numpy(), ref.m) < 1e-4
    assert np.max(np.abs(hist - ref.rms) / np.array(ref.rms)) < 1e-4


def test_outer_loop_fp32_block_preconditioned_inner_solves(sysm):
    """The benchmark's form inside the loop: the depth blocks of every rebuilt G
    (precond = 2), FP32 values, two-phase refinement; the same model as the
    FP64 oracle loop within the parity bar."""
    p, m_true, d_obs, h = sysm
    ref = outer.outer_loop(p, d_obs, p.w, p.lam, itmax=5000, tol=1e-10, max_outer=4,
                           rms_tol=0.0, min_decrease=0.0)
    m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 5000, 1e-6,
                                 max_outer=4, rms_tol=0.0, min_decrease=0.0, dtype="f32",
                                 fmt="blocked", precond=2, refine=3, refine_dtype="f32",
                                 refine_tol=1e-10)
    assert info["updates"] == 4
    assert rel(m.cpu().numpy(), ref.m) < 1e-4
    assert np.max(np.abs(hist - ref.rms) / np.array(ref.rms)) < 1e-4


def test_outer_loop_stopping_and_errors(sysm):
    p, m_true, d_obs, h = sysm
    m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 100, 1e-8,
                                 max_outer=5, rms_tol=1e9)
    assert info["reason"] == 1 and info["updates"] == 0 and not m.cpu().numpy().any()
    assert hist[0] == pytest.approx(np.sqrt(np.mean(d_obs * d_obs)), rel=1e-13)
    ref = outer.outer_loop(p, d_obs, p.w, p.lam, 3000, 1e-10, max_outer=20, rms_tol=0.0,
                           min_decrease=0.6)
    m, hist, info = h.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 3000, 1e-10,
                                 max_outer=20, rms_tol=0.0, min_decrease=0.6)
    assert info["reason"] == ref.reason == 2 and info["updates"] == ref.updates
    assert rel(m.cpu().numpy(), ref.m) < 1e-6
    plain = pdst.build_G_problem(p, dtypes=("f64",))
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        plain.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 10, 1e-6)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        plain.set_depth_kernels(to_dev(np.ones((p.nx * p.ny, p.n_periods, p.nz))))
    plain.close()
    no64 = pdst.build_G_problem(p, dtypes=("f32",), keep_lengths=True)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        no64.outer_loop(to_dev(d_obs), p.periods_s, p.w, p.lam, 10, 1e-6)
    no64.close()
