"""GPU parity of the learned-preconditioner kernels against the FP64 oracles:
column features, MLP forward, MLP gradient (the training kernel), Adam, and
the column-norm power scaling."""
import math

import numpy as np
import pytest

import oracle
from oracle import features as ofeat
from oracle import mlp
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def systems():
    return [synth.tiny(), synth.custom(13, 7, 3, 17, 5, bend=0.15, seed=21, dx_km=1.5),
            synth.custom(9, 11, 8, 12, 7, bend=0.15, seed=5)]


@pytest.mark.parametrize("i", range(3))
def test_features_match_oracle(i):
    torch = require_cuda()
    p = systems()[i]
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    logT = np.log(p.periods_s)
    ref = ofeat.features(GT, p.nx, p.ny, p.nz, p.row_period, logT)
    h = pdst.build_G_problem(p)
    f = h.features(logT).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(f, ref, rtol=2e-6, atol=2e-6)


def test_mlp_forward_and_gradient_match_oracle():
    torch = require_cuda()
    rng = np.random.default_rng(3)
    n = 5000
    F = (rng.standard_normal((n, 8)) * 2 + 1).astype(np.float32)
    theta = mlp.init_params(rng, F.mean(axis=0), F.std(axis=0) + 0.1)
    theta[16:] += 0.05 * rng.standard_normal(mlp.NTRAIN)
    theta = theta.astype(np.float32).astype(np.float64)
    t = rng.standard_normal(n).astype(np.float32)
    P = torch.from_numpy(theta.astype(np.float32)).cuda()
    Fd = torch.from_numpy(F).cuda()
    D, L = pdst.mlp_forward(P, Fd, want_D=True, want_logD=True)
    ref_logD, _ = mlp.forward(theta, F.astype(np.float64))
    np.testing.assert_allclose(L.cpu().numpy(), ref_logD, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(np.log(D.cpu().numpy()), ref_logD, rtol=1e-4, atol=1e-5)
    idx = rng.choice(n, 1024, replace=False).astype(np.int32)
    g = pdst.mlp_grad(P, Fd, torch.from_numpy(idx).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    loss_ref, grad_ref = mlp.loss_and_grad(theta, F[idx].astype(np.float64), t[idx])
    assert abs(g[-1] - loss_ref) <= 1e-4 * loss_ref
    assert rel(g[:-1], grad_ref) < 1e-4
    # deterministic: same batch, same bits
    g2 = pdst.mlp_grad(P, Fd, torch.from_numpy(idx).cuda(), torch.from_numpy(t).cuda())
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)
    # one Adam step against the oracle's update
    m = torch.zeros(mlp.NTRAIN, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    pdst.mlp_adam(P, gd, m, v, 1, lr=1e-3)
    th_ref, _, _ = mlp.adam_step(theta, g[:-1], np.zeros(mlp.NTRAIN), np.zeros(mlp.NTRAIN), 1)
    np.testing.assert_allclose(P.cpu().numpy(), th_ref, rtol=1e-5, atol=1e-6)


def test_column_norms_and_power_scaling():
    torch = require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p)
    c = h.col_norms(p.w, p.lam).cpu().numpy()
    cref = np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    assert rel(c, cref) < 1e-13
    D = cref ** -0.5
    h.set_col_scaling_power(p.w, p.lam, 0.5)
    for k in (1, 4):
        o = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, d, atol=0, btol=0, conlim=0,
                        itmax=k, D=D, lam_rows=p.lam)
        r = h.lsqr(to_dev(d), p.w, p.lam, k, 0.0, precond=1, conlim=1e300)
        assert rel(r.m.cpu().numpy(), D * o.x) < 1e-10


def test_trained_network_gain_on_held_out_system():
    """The trained network (precond_mlp.json, trained on seeds 10000-10199) on a
    held-out 64 x 64 x 16 system (seed 20000): against no scaling it cuts the
    FP32 iterations to tol 1e-6 by a third, and it is at least on par with
    plain column-norm scaling; the scaled solves also end closer to the FP64
    solution."""
    torch = require_cuda()
    import time
    from paper_2604_11920_b300.train_precond import DEFAULT_OUT, learned_scaling, load_params
    from paper_2604_11920_b300.train_precond import make_rhs
    p = synth.mid(20000)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
    d = make_rhs(h, p)
    ref = h.lsqr(d, p.w, p.lam, 100000, 1e-10, dtype="f64", fmt="blocked")

    def solve(precond):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.lsqr(d, p.w, p.lam, 20000, p.tol, dtype="f32", fmt="blocked", precond=precond)
        torch.cuda.synchronize()
        e = float(torch.linalg.norm(r.m - ref.m) / torch.linalg.norm(ref.m))
        return r.info["iters"], time.perf_counter() - t0, e

    it_none, t_none, e_none = solve(0)
    h.set_col_scaling_power(p.w, p.lam, 1.0)
    it_cn, t_cn, e_cn = solve(1)
    learned_scaling(h, p, load_params(DEFAULT_OUT))
    it_l, t_l, e_l = solve(1)
    print(f"held-out seed 20000: none {it_none} it {t_none:.3f} s err {e_none:.3f}; "
          f"column-norm {it_cn} it {t_cn:.3f} s err {e_cn:.3f}; "
          f"learned {it_l} it {t_l:.3f} s err {e_l:.3f}")
    assert it_l <= 0.8 * it_none and e_l < e_none
    assert it_l <= 1.05 * it_cn
    h.close()
