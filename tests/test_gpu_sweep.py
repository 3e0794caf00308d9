"""Damping sweep: solutions for several damping values from one Golub-Kahan
bidiagonalisation (u, v, alpha, beta do not depend on the damping, which
enters only the scalar recurrence of LSQR).

* Each value's result is bit-identical to a separate pdst_lsqr call with the
  same options (same kernels, same reduction order, the recurrence frozen
  once that value stops).
* Fixed-k FP64 iterates agree with the oracle's damped LSQR (k <= 8).
"""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

LAMS = [0.0, 1e-3, 1e-2, 0.05, 0.1, 0.3, 1.0, 3.0]


@pytest.fixture(scope="module")
def tiny():
    require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "df64"))
    return p, G, GT, d, h


@pytest.mark.parametrize("dtype,fmt", [("f64", "element"), ("f32", "blocked"),
                                       ("df64", "blocked")])
def test_sweep_equals_separate_solves(tiny, dtype, fmt):
    p, G, GT, d, h = tiny
    sw = h.lsqr_damping_sweep(to_dev(d), p.w, LAMS, 3000, 1e-7, dtype=dtype, fmt=fmt)
    assert len(sw) == len(LAMS)
    for lam, r in zip(LAMS, sw):
        one = h.lsqr(to_dev(d), p.w, lam, 3000, 1e-7, dtype=dtype, fmt=fmt)
        assert r.info["iters"] == one.info["iters"] and r.info["istop"] == one.info["istop"]
        assert np.array_equal(r.m.cpu().numpy(), one.m.cpu().numpy()), lam
        for key in ("rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm"):
            assert r.info[key] == one.info[key], (lam, key)
    # different damping values really stop at different iterations
    assert len({r.info["iters"] for r in sw}) > 1


@pytest.mark.parametrize("k", [2, 8])
def test_sweep_fixed_k_matches_oracle(tiny, k):
    p, G, GT, d, h = tiny
    sw = h.lsqr_damping_sweep(to_dev(d), p.w, LAMS, k, 0.0, conlim=1e300)
    for lam, r in zip(LAMS, sw):
        ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, lam, d, atol=0, btol=0, conlim=0,
                          itmax=k)
        assert r.info["iters"] == k
        assert rel(r.m.cpu().numpy(), ref.x) < 1e-10, lam
        assert abs(r.info["rnorm"] - ref.rnorm) <= 1e-10 * ref.rnorm


def test_sweep_edges_and_errors(tiny):
    p, G, GT, d, h = tiny
    z = h.lsqr_damping_sweep(to_dev(d), p.w, [0.1, 1.0], 0, 1e-6)
    assert all(not r.m.cpu().numpy().any() and r.info["iters"] == 0 for r in z)
    one = h.lsqr_damping_sweep(to_dev(d), p.w, [p.lam], 500, 1e-6, fmt="blocked")[0]
    ref = h.lsqr(to_dev(d), p.w, p.lam, 500, 1e-6, fmt="blocked")
    assert np.array_equal(one.m.cpu().numpy(), ref.m.cpu().numpy())
    zero = h.lsqr_damping_sweep(to_dev(np.zeros_like(d)), p.w, [0.1, 1.0], 100, 1e-6)
    assert all(not r.m.cpu().numpy().any() for r in zero)
    with pytest.raises(pdst.PdstError):
        h.lsqr_damping_sweep(to_dev(d), p.w, [-1.0], 10, 1e-6)
    with pytest.raises(pdst.PdstError):
        h.lsqr_damping_sweep(to_dev(d), p.w, [0.1], 10, 1e-6, precond=1)
    with pytest.raises(pdst.PdstError):
        h.lsqr_damping_sweep(to_dev(d), p.w, [0.1] * 65, 10, 1e-6)
    with pytest.raises(pdst.PdstError):
        h.lsqr_damping_sweep(to_dev(d), p.w, [0.1], 10, 1e-6, method="lsmr")
    # an ordinary solve after a sweep on the same handle is unaffected
    again = h.lsqr(to_dev(d), p.w, p.lam, 500, 1e-6, fmt="blocked")
    assert np.array_equal(again.m.cpu().numpy(), ref.m.cpu().numpy())
