"""GPU parity of LSQR (Paige & Saunders 1982) against the FP64 oracle.

* FP64 iterates at a fixed iteration count agree with the oracle while the
  Golub-Kahan process is still orthogonal (k <= 8 on these systems; after
  that rounding differences grow about 10x per step on both sides, so fixed-k
  agreement is not a property of the method).
* Converged solutions agree within the parity bar: relative model error
  ||m - m_ref|| / ||m_ref|| <= 1e-4 and relative residual difference <= 1e-6,
  m_ref being the oracle solved to a tighter tolerance.
* FP32 / BF16 forms report their error against m_ref.
"""
import numpy as np
import pytest

import oracle
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
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16", "df64"))
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-12, btol=1e-12,
                      itmax=50000)
    return p, G, GT, d, h, ref


def residual_norm(p, G, m, d, lam):
    """||[d;0;0] - [G; w L; lam I] m|| evaluated by the oracle."""
    Am = oracle.apply_A(G, (p.nx, p.ny, p.nz), p.w, m)
    r = np.concatenate([d, np.zeros(p.n)]) - Am
    return np.sqrt(r @ r + lam * lam * (m @ m))


@pytest.mark.parametrize("fmt", ["element", "blocked"])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fixed_k_iterates_fp64(tiny, fmt, k):
    p, G, GT, d, h, _ = tiny
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                      itmax=k)
    res = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, fmt=fmt, conlim=1e300)
    assert res.info["iters"] == k and res.info["istop"] == 7
    assert rel(res.m.cpu().numpy(), ref.x) < 1e-10
    for key in ("rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm"):
        assert abs(res.info[key] - getattr(ref, key)) <= 1e-10 * abs(getattr(ref, key)), key


@pytest.mark.parametrize("fmt", ["element", "blocked"])
def test_converged_fp64_matches_oracle(tiny, fmt):
    p, G, GT, d, h, ref = tiny
    res = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-8, fmt=fmt)
    m = res.m.cpu().numpy()
    assert res.info["istop"] in (1, 2)
    assert rel(m, ref.x) <= MODEL_TOL
    r_gpu = residual_norm(p, G, m, d, p.lam)
    r_ref = residual_norm(p, G, ref.x, d, p.lam)
    assert abs(r_gpu - r_ref) / r_ref <= RESID_TOL
    same = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-8, btol=1e-8,
                       itmax=20000)
    assert same.istop == res.info["istop"]
    assert abs(same.itn - res.info["iters"]) <= 0.1 * same.itn
    # the ||r|| estimate agrees with the residual the oracle evaluates
    assert abs(res.info["rnorm"] - r_gpu) <= 1e-6 * r_gpu


@pytest.mark.parametrize("dtype,fmt", [("f32", "element"), ("f32", "blocked"),
                                       ("bf16", "blocked")])
def test_reduced_precision_forms(tiny, dtype, fmt):
    """FP32 values/vectors (FP64 scalars) reach the FP64 form's accuracy at the
    same stopping tolerance, and the model error of each form is reported;
    BF16 values carry a ~4e-3 relative value error, so only a looser bound."""
    p, G, GT, d, h, ref = tiny
    out = {}
    for tol in (1e-6, 1e-8):
        r64 = h.lsqr(to_dev(d), p.w, p.lam, 20000, tol, dtype="f64", fmt=fmt)
        res = h.lsqr(to_dev(d), p.w, p.lam, 20000, tol, dtype=dtype, fmt=fmt)
        e64 = rel(r64.m.cpu().numpy(), ref.x)
        err = rel(res.m.cpu().numpy(), ref.x)
        out[tol] = (err, e64)
        print(f"{dtype}/{fmt} tol={tol:g}: iters={res.info['iters']} istop={res.info['istop']} "
              f"model error vs FP64 oracle {err:.3e} (FP64 form: {e64:.3e}, "
              f"{r64.info['iters']} iters)")
        assert res.info["istop"] in (1, 2, 7)
    err6, e646 = out[1e-6]
    if dtype == "f32":
        assert err6 <= 1.5 * e646 + 1e-4
        assert out[1e-8][0] <= MODEL_TOL
    else:
        assert err6 <= 3.0 * e646 + 2e-2


def test_switching_forms_on_one_handle(tiny):
    """Solving in FP64, then FP32, then BF16, then FP64 again on one handle
    gives the same answers as fresh handles (workspace reuse across dtypes)."""
    p, G, GT, d, h, ref = tiny
    dd = to_dev(d)
    seq = [("f64", "element"), ("f32", "blocked"), ("bf16", "blocked"), ("f64", "blocked"),
           ("f64", "element")]
    outs = [h.lsqr(dd, p.w, p.lam, 3000, 1e-6, dtype=dt, fmt=fm).m.cpu().numpy()
            for dt, fm in seq]
    for (dt, fm), m in zip(seq, outs):
        fresh = pdst.build_G_problem(p, dtypes=(dt,))
        mf = fresh.lsqr(dd, p.w, p.lam, 3000, 1e-6, dtype=dt, fmt=fm).m.cpu().numpy()
        assert np.array_equal(m, mf), (dt, fm)
        fresh.close()


def test_graph_and_plain_launches_identical(tiny):
    p, G, GT, d, h, _ = tiny
    dd = to_dev(d)
    a = h.lsqr(dd, p.w, p.lam, 300, 1e-8, use_graph=True, kblock=16).m.cpu().numpy()
    b = h.lsqr(dd, p.w, p.lam, 300, 1e-8, use_graph=False).m.cpu().numpy()
    c = h.lsqr(dd, p.w, p.lam, 300, 1e-8, use_graph=True, kblock=7).m.cpu().numpy()
    e = h.lsqr(dd, p.w, p.lam, 300, 1e-8, use_graph=True, kblock=16).m.cpu().numpy()
    f = h.lsqr(dd, p.w, p.lam, 300, 1e-8, profile=True)
    g = h.lsqr(dd, p.w, p.lam, 300, 1e-8, profile=2, kblock=16)
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, e)
    assert np.array_equal(a, f.m.cpu().numpy()) and np.array_equal(a, g.m.cpu().numpy())
    assert f.info["profiled_iters"] == 300 and f.info["fwd_ms"] > 0 and f.info["adj_ms"] > 0
    # the profiled graph replay counts only the iterations that ran
    assert g.info["profiled_iters"] == g.info["iters"] == f.info["iters"]
    assert g.info["fwd_ms"] > 0 and g.info["adj_ms"] > 0 and g.info["upd_ms"] > 0


def test_residual_history_non_increasing(tiny):
    torch = require_cuda()
    p, G, GT, d, h, _ = tiny
    hist = torch.zeros(400, dtype=torch.float64, device="cuda")
    res = h.lsqr(to_dev(d), p.w, p.lam, 400, 0.0, hist=hist, conlim=1e300)
    rh = hist.cpu().numpy()[: res.info["iters"]]
    assert res.info["iters"] == 400
    assert np.all(np.diff(rh) <= 1e-12 * rh[0])


def test_column_scaled_form(tiny):
    p, G, GT, d, h, ref = tiny
    h.set_col_scaling(None, p.w, p.lam)
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    # fixed-k agreement with the oracle's scaled operator [G D; w L D; lam D]
    for k in (1, 3, 6):
        o = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, d, atol=0, btol=0, conlim=0,
                        itmax=k, D=D, lam_rows=p.lam)
        r = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, precond=1, conlim=1e300)
        assert rel(r.m.cpu().numpy(), D * o.x) < 1e-10
    res = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-8, precond=1)
    assert rel(res.m.cpu().numpy(), ref.x) <= MODEL_TOL
    plain = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-8)
    assert res.info["iters"] < plain.info["iters"]
    # a caller-supplied D (the oracle's column norms) reaches the same minimiser
    h.set_col_scaling(to_dev(D))
    res2 = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-8, precond=1)
    assert rel(res2.m.cpu().numpy(), ref.x) <= MODEL_TOL
    assert abs(res2.info["iters"] - res.info["iters"]) <= 0.05 * res.info["iters"]


def test_edge_cases(tiny):
    p, G, GT, d, h, _ = tiny
    z = h.lsqr(to_dev(np.zeros_like(d)), p.w, p.lam, 100, 1e-8)
    assert z.info["iters"] == 0 and z.info["istop"] == 0 and not z.m.cpu().numpy().any()
    z0 = h.lsqr(to_dev(d), p.w, p.lam, 0, 1e-8)
    assert z0.info["iters"] == 0 and not z0.m.cpu().numpy().any()
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr(to_dev(d), -1.0, p.lam, 10, 1e-8)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr(to_dev(d), p.w, float("nan"), 10, 1e-8)
    h2 = pdst.build_G_problem(p, dtypes=("f32",))
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        h2.lsqr(to_dev(d), p.w, p.lam, 10, 1e-8, dtype="f64")
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        h2.lsqr(to_dev(d), p.w, p.lam, 10, 1e-8, dtype="f32", precond=1)


def test_empty_rows_and_ragged_system():
    require_cuda()
    p = synth.custom(13, 7, 3, 17, 5, bend=0.15, seed=21, w=1.0, lam=0.2, dx_km=1.5)
    p.ctrl = np.vstack([p.ctrl, [[4.0, 4.0, 4.0, 4.0, 4.0, 4.0]]])
    p.row_period = np.concatenate([p.row_period, [1]]).astype(np.int32)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G, noise=np.concatenate([p.noise, [0.3]]))
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-12, btol=1e-12,
                      itmax=50000)
    h = pdst.build_G_problem(p)
    for fmt in ("element", "blocked"):
        res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-10, fmt=fmt)
        assert rel(res.m.cpu().numpy(), ref.x) <= 1e-6


def test_host_entry_point(tiny):
    p, G, GT, d, h, ref = tiny
    res = h.lsqr_host(d, p.w, p.lam, 20000, 1e-8)
    dev = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-8)
    assert np.array_equal(res.m, dev.m.cpu().numpy())


@pytest.mark.parametrize("dtype,precond", [("f32", 0), ("f32", 1), ("bf16", 1)])
def test_two_phase_solve_reaches_fp64_solution(tiny, dtype, precond):
    """Reduced-precision solve first, then FP64 refinement sweeps on the
    correction (FP64 residual of the augmented system): the result meets the
    FP64 minimiser to the parity bar, which one reduced-precision solve cannot
    reach on this large-residual problem."""
    p, G, GT, d, h, ref = tiny
    if precond:
        h.set_col_scaling(None, p.w, p.lam)
    one = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype=dtype, fmt="blocked", precond=precond)
    res = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype=dtype, fmt="blocked", precond=precond,
                 refine=3, refine_dtype="f64", refine_tol=1e-10)
    e1 = rel(one.m.cpu().numpy(), ref.x)
    e = rel(res.m.cpu().numpy(), ref.x)
    print(f"{dtype} precond={precond}: one solve {e1:.2e} ({one.info['iters']} it); two-phase "
          f"{e:.2e} in {res.info['sweeps']} sweeps, {res.info['iters']} it")
    assert res.info["sweeps"] >= 2
    assert e <= 1e-6 and e < e1
    r_gpu = residual_norm(p, G, res.m.cpu().numpy(), d, p.lam)
    r_ref = residual_norm(p, G, ref.x, d, p.lam)
    assert abs(r_gpu - r_ref) / r_ref <= RESID_TOL
    # a second call on the same handle (workspace switched between dtypes) agrees
    again = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype=dtype, fmt="blocked",
                   precond=precond, refine=3, refine_dtype="f64", refine_tol=1e-10)
    assert np.array_equal(again.m.cpu().numpy(), res.m.cpu().numpy())


# ------------------------------------------------------------ double-float form
# Each FP64 value is held as hi + lo (two floats) and the sweeps run in
# double-float arithmetic: relative rounding about 2^-47 per operation instead
# of FP64's 2^-53.  Bars: 1e-9 on fixed-k iterates (sums of ~10^3 products per
# row, k <= 8 steps of a well-conditioned bidiagonalisation), the parity bar on
# converged solutions.

DF_ITER_TOL = 1e-9


def test_df64_values_split_exactly(tiny):
    """hi = fl32(v), lo = fl32(v - hi): |v - (hi + lo)| <= 2^-48 |v| for every stored value."""
    p, G, GT, d, h, _ = tiny
    ptr, idx, v64 = h.export_csr("f64")
    _, _, vdf = h.export_csr("df64")
    assert np.array_equal(v64, G.val)
    err = np.abs(vdf - v64)
    assert np.all(err <= 2.0 ** -48 * np.abs(v64))
    assert np.any(err > 0)       # the pairs do carry the bits below float precision
    nzm = v64 != 0
    assert np.max(np.abs(vdf - v64.astype(np.float32))[nzm] / np.abs(v64[nzm])) > 1e-9
    _, _, cdf = h.export_csc("df64")
    _, _, c64 = h.export_csc("f64")
    assert np.all(np.abs(cdf - c64) <= 2.0 ** -48 * np.abs(c64))


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fixed_k_iterates_df64(tiny, k):
    p, G, GT, d, h, _ = tiny
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                      itmax=k)
    res = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, dtype="df64", fmt="blocked", conlim=1e300)
    assert res.info["iters"] == k and res.info["istop"] == 7
    assert rel(res.m.cpu().numpy(), ref.x) < DF_ITER_TOL
    for key in ("rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm"):
        assert abs(res.info[key] - getattr(ref, key)) <= DF_ITER_TOL * abs(getattr(ref, key)), key
    # FP32 values are far from this bar at the same k
    f32 = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, dtype="f32", fmt="blocked", conlim=1e300)
    if k >= 2:
        assert rel(f32.m.cpu().numpy(), ref.x) > 100 * rel(res.m.cpu().numpy(), ref.x)


def test_converged_df64_matches_oracle(tiny):
    p, G, GT, d, h, ref = tiny
    res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-12, dtype="df64", fmt="blocked")
    assert res.info["istop"] in (1, 2)
    e = rel(res.m.cpu().numpy(), ref.x)
    assert e <= MODEL_TOL
    r_gpu = residual_norm(p, G, res.m.cpu().numpy(), d, p.lam)
    r_ref = residual_norm(p, G, ref.x, d, p.lam)
    assert abs(r_gpu - r_ref) / r_ref <= RESID_TOL
    # same solve in FP64 on the GPU: the two agree far inside the parity bar
    f64 = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-12, dtype="f64", fmt="blocked")
    assert rel(res.m.cpu().numpy(), f64.m.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("precond", [0, 1])
def test_two_phase_with_fp32_refinement(tiny, precond):
    """FP32 solve, then refinement sweeps with FP32 values on the FP64 residual:
    each sweep starts from the exact residual, so the FP32 operator only slows
    the contraction and the result meets the FP64 minimiser to the parity bar."""
    p, G, GT, d, h, ref = tiny
    if precond:
        h.set_col_scaling(None, p.w, p.lam)
    one = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype="f32", fmt="blocked", precond=precond)
    res = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype="f32", fmt="blocked", precond=precond,
                 refine=6, refine_dtype="f32", refine_tol=1e-10)
    e1 = rel(one.m.cpu().numpy(), ref.x)
    e = rel(res.m.cpu().numpy(), ref.x)
    print(f"precond={precond}: one solve {e1:.2e}; FP32 sweeps {e:.2e} "
          f"({res.info['sweeps']} sweeps, {res.info['iters']} it)")
    assert res.info["sweeps"] >= 2
    assert e <= 1e-4 and e < e1
    r_gpu = residual_norm(p, G, res.m.cpu().numpy(), d, p.lam)
    r_ref = residual_norm(p, G, ref.x, d, p.lam)
    assert abs(r_gpu - r_ref) / r_ref <= RESID_TOL


@pytest.mark.parametrize("dtype,precond", [("f32", 0), ("f32", 1)])
def test_two_phase_with_df64_refinement(tiny, dtype, precond):
    """FP32 solve, then double-float refinement sweeps on the FP64 residual:
    the same accuracy as FP64 refinement sweeps."""
    p, G, GT, d, h, ref = tiny
    if precond:
        h.set_col_scaling(None, p.w, p.lam)
    r64 = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype=dtype, fmt="blocked", precond=precond,
                 refine=3, refine_dtype="f64", refine_tol=1e-10)
    rdf = h.lsqr(to_dev(d), p.w, p.lam, 20000, 1e-6, dtype=dtype, fmt="blocked", precond=precond,
                 refine=3, refine_dtype="df64", refine_tol=1e-10)
    e64 = rel(r64.m.cpu().numpy(), ref.x)
    edf = rel(rdf.m.cpu().numpy(), ref.x)
    print(f"{dtype} precond={precond}: FP64 sweeps {e64:.2e}, double-float sweeps {edf:.2e} "
          f"({rdf.info['sweeps']} sweeps, {rdf.info['iters']} it)")
    assert rdf.info["sweeps"] >= 2
    assert edf <= 1e-6
    assert edf <= 10 * e64 + 1e-9


def test_df64_form_errors(tiny):
    p, G, GT, d, h, _ = tiny
    with pytest.raises(pdst.PdstError):
        h.lsqr(to_dev(d), p.w, p.lam, 10, 1e-6, dtype="df64", fmt="element")
    with pytest.raises(pdst.PdstError):
        h.lsqr(to_dev(d), p.w, p.lam, 10, 1e-6, dtype="f32", fmt="element", refine=2,
               refine_dtype="df64")
    with pytest.raises(pdst.PdstError):
        h.apply_G(to_dev(np.zeros(p.n)), to_dev(np.zeros(h.m)), dtype="df64")
    h2 = pdst.build_G_problem(p, dtypes=("f32",))
    with pytest.raises(pdst.PdstError):
        h2.lsqr(to_dev(d), p.w, p.lam, 10, 1e-6, dtype="df64", fmt="blocked")
    h2.close()


# ------------------------------------------------ every depth-count path
# nz % 4 == 0 uses 4-entry vector loads (compile-time quads for 8, 16 and 20 --
# the paths of the 64 x 64 x 16 and 100 x 100 x 20 workloads -- run-time
# quads otherwise, e.g. 12); nz % 6 == 0 otherwise 6-entry groups in the
# forward and three pairs per lane in the adjoint (6, 18, 30: the paper's 18
# depth nodes); other even nz 2-entry pairs (10, 14); odd nz one entry per
# lane (5).

@pytest.mark.parametrize("nz", [5, 6, 8, 10, 12, 14, 16, 18, 20, 30])
def test_fixed_k_iterates_other_depth_counts(nz):
    require_cuda()
    p = synth.make_problem(f"nz{nz}", 12, 10, nz, 14, np.geomspace(2.0, 16.0, 5), bend=0.15,
                           model="blobs", noise_frac=0.01, w=1.0, lam=0.1, tol=1e-8,
                           itmax=300, seed=nz, dz_km=1.0)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16", "df64"))
    for k in (2, 6):
        ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                          itmax=k)
        for dt, bar in (("f64", 1e-10), ("df64", 1e-9), ("f32", 1e-4), ("bf16", 3e-2)):
            r = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, dtype=dt, fmt="blocked", conlim=1e300)
            assert rel(r.m.cpu().numpy(), ref.x) < bar, (nz, k, dt)
    h.close()
