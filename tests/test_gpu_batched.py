"""Batched LSQR (one persistent launch per phase over all systems, the
right-hand sides of a system sharing its G) against single-system LSQR and
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def small_batch():
    """Three uneven systems (one with nz not a multiple of 4) and their
    right-hand sides: checkerboards of several block sizes and noisy data."""
    probs = [synth.custom(12, 10, 8, 14, 6, bend=0.15, seed=31, w=1.0, lam=0.1),
             synth.custom(9, 13, 4, 18, 9, bend=0.1, seed=32, w=2.0, lam=0.05),
             synth.custom(7, 6, 3, 10, 4, bend=0.15, seed=33, w=0.5, lam=0.2)]
    nrhs = [3, 16, 1]
    out = []
    for p, R in zip(probs, nrhs):
        G = oracle.build_G_problem(p)
        cols, lams = [], []
        for j in range(R):
            b = 2 + (j % 5)
            m = synth.checkerboard(p.nx, p.ny, p.nz, b, 0.05) * (1 if j % 2 == 0 else -1)
            cols.append(oracle.rhs_for(p, G, m_model=m, noise=synth.rhs_noise(p.seed, p.m_rows, j)))
            lams.append(float(np.logspace(-3, 0, R)[j]) if R > 1 else p.lam)
        out.append((p, G, np.stack(cols, axis=1), lams))
    return out


@pytest.fixture(scope="module")
def batch():
    require_cuda()
    b = small_batch()
    hs = [pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16")) for p, _, _, _ in b]
    return b, hs


@pytest.mark.parametrize("k", [1, 3, 6])
def test_fixed_k_matches_single_system_solves(batch, k):
    b, hs = batch
    ds = [to_dev(D) for _, _, D, _ in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, _, _, _ in b],
                                       [l for _, _, _, l in b], k, 0.0, dtype="f64", tile_rows=4)
    for (p, G, D, lams), h, mo, inf in zip(b, hs, outs, infos):
        for j in range(D.shape[1]):
            single = h.lsqr(to_dev(D[:, j]), p.w, lams[j], k, 0.0, fmt="blocked", conlim=1e8)
            assert inf[j]["iters"] == single.info["iters"] == k
            assert rel(mo[:, j].cpu().numpy(), single.m.cpu().numpy()) < 1e-10


def test_converged_columns_match_oracle(batch):
    b, hs = batch
    ds = [to_dev(D) for _, _, D, _ in b]
    outs, infos, opts = pdst.lsqr_batched(hs, ds, [p.w for p, _, _, _ in b],
                                          [l for _, _, _, l in b], 20000, 1e-9, dtype="f64")
    assert opts["chosen_tile_rows"] in (2, 8, 32)
    assert sum(t > 0 for t in opts["tune_ms"]) == 3
    for (p, G, D, lams), mo, inf in zip(b, outs, infos):
        GT = oracle.transpose(G)
        for j in sorted({0, D.shape[1] - 1, D.shape[1] // 2}):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, lams[j], D[:, j], atol=1e-12,
                              btol=1e-12, itmax=50000)
            assert inf[j]["istop"] in (1, 2)
            assert rel(mo[:, j].cpu().numpy(), ref.x) <= 1e-4


def test_fp32_batched_close_to_fp32_single(batch):
    b, hs = batch
    ds = [to_dev(D) for _, _, D, _ in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, _, _, _ in b],
                                       [l for _, _, _, l in b], 20000, 1e-6, dtype="f32")
    for (p, G, D, lams), h, mo, inf in zip(b, hs, outs, infos):
        for j in (0, D.shape[1] - 1):
            single = h.lsqr(to_dev(D[:, j]), p.w, lams[j], 20000, 1e-6, dtype="f32", fmt="blocked")
            ref = h.lsqr(to_dev(D[:, j]), p.w, lams[j], 20000, 1e-10, dtype="f64")
            e_b = rel(mo[:, j].cpu().numpy(), ref.m.cpu().numpy())
            e_s = rel(single.m.cpu().numpy(), ref.m.cpu().numpy())
            assert e_b <= 2 * e_s + 1e-4, (e_b, e_s)


def test_repeat_call_is_bit_identical_and_itmax_zero(batch):
    b, hs = batch
    ds = [to_dev(D) for _, _, D, _ in b]
    args = ([p.w for p, _, _, _ in b], [l for _, _, _, l in b])
    o1, _, _ = pdst.lsqr_batched(hs, ds, *args, 50, 0.0, dtype="f32", tile_rows=8)
    o2, _, _ = pdst.lsqr_batched(hs, ds, *args, 50, 0.0, dtype="f32", tile_rows=8)
    for a, c in zip(o1, o2):
        assert np.array_equal(a.cpu().numpy(), c.cpu().numpy())
    o3, i3, _ = pdst.lsqr_batched(hs, ds, *args, 0, 1e-6, dtype="f32")
    assert all(not m.cpu().numpy().any() for m in o3)
    assert all(inf["iters"] == 0 for row in i3 for inf in row)


def test_bad_arguments():
    require_cuda()
    p = synth.custom(6, 6, 4, 8, 2, bend=0.1, seed=40)
    h = pdst.build_G_problem(p, dtypes=("f32",))
    import torch
    d = torch.zeros((h.m, 17), dtype=torch.float64, device="cuda")
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        pdst.lsqr_batched([h], [d], [1.0], [[0.1] * 17], 10, 1e-6, dtype="f32")
    d = torch.zeros((h.m, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        pdst.lsqr_batched([h], [d], [1.0], [[0.1, 0.2]], 10, 1e-6, dtype="f64")


# ------------------------------------------ the 16-right-hand-side fast paths
# With 9-16 right-hand sides (RS = 16) and nz = 8 or 16 the batched forward and
# adjoint run compile-time paths (two runs in flight; 4 x 4 outer products per
# lane), the ones the 64-system workload runs.  Each column is checked against
# the FP64 oracle directly: element by element at a fixed iteration count
# (FP64 values), and converged columns against the oracle's tol-1e-12
# solution (FP64 within 1e-4; FP32 within what the oracle itself reaches at
# the same tolerance, plus 1e-3).

def nzc_batch():
    probs = [synth.custom(14, 12, 8, 16, 5, bend=0.15, seed=51, w=1.0, lam=0.1),
             synth.custom(11, 13, 16, 15, 6, bend=0.15, seed=52, w=2.0, lam=0.05, dz_km=1.0),
             synth.custom(10, 9, 16, 12, 4, bend=0.1, seed=53, w=1.0, lam=0.1, dz_km=1.0)]
    nrhs = [16, 16, 13]
    out = []
    for p, R in zip(probs, nrhs):
        G = oracle.build_G_problem(p)
        cols, lams = [], []
        for j in range(R):
            m = synth.checkerboard(p.nx, p.ny, p.nz, 2 + (j % 7), 0.05) * (1 if j % 2 else -1)
            cols.append(oracle.rhs_for(p, G, m_model=m, noise=synth.rhs_noise(p.seed, p.m_rows, j)))
            lams.append(float(np.logspace(-3, 0, R)[j]))
        out.append((p, G, oracle.transpose(G), np.stack(cols, axis=1), lams))
    return out


@pytest.fixture(scope="module")
def nzc():
    require_cuda()
    b = nzc_batch()
    hs = [pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
          for p, _, _, _, _ in b]
    yield b, hs
    for h in hs:
        h.close()


@pytest.mark.parametrize("k", [1, 4, 8])
def test_nzc_paths_fixed_k_match_oracle(nzc, k):
    b, hs = nzc
    ds = [to_dev(D) for _, _, _, D, _ in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, *_ in b], [l for *_, l in b], k, 0.0,
                                       dtype="f64", tile_rows=2)
    for (p, G, GT, D, lams), mo, inf in zip(b, outs, infos):
        got = mo.cpu().numpy()
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, lams[j], D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k)
            assert inf[j]["iters"] == k
            assert rel(got[:, j], ref.x) < 1e-10, (p.nz, j, k)
            for key in ("rnorm", "arnorm", "anorm", "xnorm"):
                assert abs(inf[j][key] - getattr(ref, key)) <= 1e-10 * abs(getattr(ref, key)), key


def test_nzc_paths_converged_match_oracle(nzc):
    b, hs = nzc
    ds = [to_dev(D) for _, _, _, D, _ in b]
    w = [p.w for p, *_ in b]
    lams = [l for *_, l in b]
    o64, i64, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-10, dtype="f64")
    o32, i32, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32")
    for (p, G, GT, D, lj), m64, m32, inf64, inf32 in zip(b, o64, o32, i64, i32):
        for j in range(D.shape[1]):
            grid = (p.nx, p.ny, p.nz)
            ref = oracle.lsqr(G, GT, grid, p.w, lj[j], D[:, j], atol=1e-12, btol=1e-12,
                              itmax=50000)
            same = oracle.lsqr(G, GT, grid, p.w, lj[j], D[:, j], atol=1e-6, btol=1e-6,
                               itmax=50000)
            assert inf64[j]["istop"] in (1, 2) and inf32[j]["istop"] in (1, 2)
            assert rel(m64[:, j].cpu().numpy(), ref.x) <= 1e-4, (p.nz, j)
            e32 = rel(m32[:, j].cpu().numpy(), ref.x)
            e_or = rel(same.x, ref.x)
            assert e32 <= 2.0 * e_or + 1e-3, (p.nz, j, e32, e_or)


# ------------------------------------------------ batched with right scaling
# precond = 1: each system's handle scaling D (here the oracle's column norms,
# so both sides apply the same operator), pair (s, j) on
# [G D; w L D; lambda_j D] with no recurrence damping, m = D y (reading of the
# scaled form: the same minimiser as the damped problem).

def _set_oracle_scaling(b, hs):
    Ds = []
    for (p, G, GT, D, lams), h in zip(b, hs):
        c = oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam)
        Dc = 1.0 / np.sqrt(c)
        h.set_col_scaling(to_dev(Dc))
        Ds.append(Dc)
    return Ds


@pytest.mark.parametrize("k", [1, 5])
def test_scaled_batched_fixed_k_match_oracle(nzc, k):
    b, hs = nzc
    Ds = _set_oracle_scaling(b, hs)
    ds = [to_dev(D) for _, _, _, D, _ in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, *_ in b], [l for *_, l in b], k, 0.0,
                                       dtype="f64", tile_rows=8, precond=1)
    for (p, G, GT, D, lams), Dc, mo, inf in zip(b, Ds, outs, infos):
        got = mo.cpu().numpy()
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k, D=Dc, lam_rows=lams[j])
            assert inf[j]["iters"] == k
            assert rel(got[:, j], Dc * ref.x) < 1e-10, (p.nz, j, k)


def test_scaled_batched_converges_faster_to_the_same_minimiser(nzc):
    b, hs = nzc
    Ds = _set_oracle_scaling(b, hs)
    ds = [to_dev(D) for _, _, _, D, _ in b]
    w = [p.w for p, *_ in b]
    lams = [l for *_, l in b]
    o_s, i_s, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32", precond=1)
    o_u, i_u, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32")
    it_s = sum(inf["iters"] for row in i_s for inf in row)
    it_u = sum(inf["iters"] for row in i_u for inf in row)
    print(f"FP32 batched, tol 1e-6: scaled {it_s} iterations, unscaled {it_u}")
    assert it_s < it_u
    for (p, G, GT, D, lj), Dc, ms, inf in zip(b, Ds, o_s, i_s):
        for j in (0, D.shape[1] // 2, D.shape[1] - 1):
            grid = (p.nx, p.ny, p.nz)
            ref = oracle.lsqr(G, GT, grid, p.w, lj[j], D[:, j], atol=1e-12, btol=1e-12,
                              itmax=50000)
            same = oracle.lsqr(G, GT, grid, p.w, 0.0, D[:, j], atol=1e-6, btol=1e-6,
                               itmax=50000, D=Dc, lam_rows=lj[j])
            assert inf[j]["istop"] in (1, 2)
            e32 = rel(ms[:, j].cpu().numpy(), ref.x)
            e_or = rel(Dc * same.x, ref.x)
            assert e32 <= 2.0 * e_or + 1e-3, (p.nz, j, e32, e_or)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        fresh = pdst.build_G_problem(b[0][0], dtypes=("f32",), formats=("blocked",))
        pdst.lsqr_batched([fresh], [ds[0]], [1.0], [lams[0]], 10, 1e-6, dtype="f32", precond=1)


@pytest.mark.parametrize("k", [1, 5])
def test_scaled_batched_generic_paths_fixed_k_match_oracle(batch, k):
    """The scaled form on the generic paths (row stride 4 or 16 with nz = 8, 4
    and 3: the any-nz forward and adjoint), against the oracle's scaled LSQR."""
    b, hs = batch
    Ds = []
    for (p, G, D, lams), h in zip(b, hs):
        GT = oracle.transpose(G)
        Dc = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
        h.set_col_scaling(to_dev(Dc))
        Ds.append((GT, Dc))
    ds = [to_dev(D) for _, _, D, _ in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, _, _, _ in b],
                                       [l for _, _, _, l in b], k, 0.0, dtype="f64",
                                       tile_rows=4, precond=1)
    for (p, G, D, lams), (GT, Dc), mo, inf in zip(b, Ds, outs, infos):
        got = mo.cpu().numpy()
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k, D=Dc, lam_rows=lams[j])
            assert inf[j]["iters"] == k
            assert rel(got[:, j], Dc * ref.x) < 1e-10, (p.nz, j, k)


# ------------------------------------------ batched with the depth blocks
# precond = 2: each system's handle blocks P (here the oracle's, so both sides
# apply the same operator), pair (s, j) on [G P; w L P; lambda_j P] with no
# recurrence damping, m = P y.  The blocks are those of the system's own
# lambda; the other damping values of the batch are exact operator rows all
# the same, so every pair keeps its own minimiser.

def _set_oracle_blocks(b, hs):
    from oracle import blockprec
    Ps = []
    for (p, G, GT, *_), h in zip(b, hs):
        P = blockprec.block_precond(GT, (p.nx, p.ny, p.nz), p.w, p.lam)
        h.set_block_precond(to_dev(P), p.w, p.lam)
        Ps.append(P)
    return Ps


@pytest.mark.parametrize("k", [1, 5])
def test_block_batched_fixed_k_match_oracle(nzc, k):
    """The 16-right-hand-side paths (nz = 8 and 16) and 13 right-hand sides."""
    from oracle import blockprec
    b, hs = nzc
    Ps = _set_oracle_blocks(b, hs)
    ds = [to_dev(D) for _, _, _, D, _ in b]
    outs, infos, opts = pdst.lsqr_batched(hs, ds, [p.w for p, *_ in b], [l for *_, l in b], k,
                                          0.0, dtype="f64", tile_rows=8, precond=2)
    for (p, G, GT, D, lams), P, mo, inf in zip(b, Ps, outs, infos):
        got = mo.cpu().numpy()
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k, P=P, lam_rows=lams[j])
            assert inf[j]["iters"] == k
            assert rel(got[:, j], blockprec.apply_blocks(P, ref.x)) < 1e-10, (p.nz, j, k)


@pytest.mark.parametrize("k", [1, 5])
def test_block_batched_generic_paths_fixed_k_match_oracle(batch, k):
    """Row stride 4 or 16 with nz = 8, 4 and 3 (the any-nz adjoint), FP64 and
    FP32 (the FP32 bar is the FP32 single-system one)."""
    from oracle import blockprec
    b, hs = batch
    Ps = []
    for (p, G, D, lams), h in zip(b, hs):
        GT = oracle.transpose(G)
        P = blockprec.block_precond(GT, (p.nx, p.ny, p.nz), p.w, p.lam)
        h.set_block_precond(to_dev(P), p.w, p.lam)
        Ps.append((GT, P))
    ds = [to_dev(D) for _, _, D, _ in b]
    for dt, bar in (("f64", 1e-10), ("f32", 1e-4)):
        outs, infos, _ = pdst.lsqr_batched(hs, ds, [p.w for p, _, _, _ in b],
                                           [l for _, _, _, l in b], k, 0.0, dtype=dt,
                                           tile_rows=4, precond=2)
        for (p, G, D, lams), (GT, P), mo, inf in zip(b, Ps, outs, infos):
            got = mo.cpu().numpy()
            for j in range(D.shape[1]):
                ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, D[:, j], atol=0, btol=0,
                                  conlim=0, itmax=k, P=P, lam_rows=lams[j])
                assert inf[j]["iters"] == k
                assert rel(got[:, j], blockprec.apply_blocks(P, ref.x)) < bar, (dt, p.nz, j, k)


def test_block_batched_converges_to_the_minimiser_in_fewer_iterations(nzc):
    """FP32 batched with the device's own blocks against the oracle's
    unpreconditioned tol-1e-12 solutions, in fewer iterations than the
    column-norm form; precond = 2 without blocks is refused."""
    b, hs = nzc
    ds = [to_dev(D) for _, _, _, D, _ in b]
    w = [p.w for p, *_ in b]
    lams = [l for *_, l in b]
    for (p, *_), h in zip(b, hs):
        h.set_block_precond(None, p.w, p.lam)
    o_b, i_b, opts = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32", precond=2)
    _set_oracle_scaling(b, hs)
    o_c, i_c, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32", precond=1)
    it_b = sum(inf["iters"] for row in i_b for inf in row)
    it_c = sum(inf["iters"] for row in i_c for inf in row)
    print(f"FP32 batched, tol 1e-6: depth blocks {it_b} iterations, column norms {it_c}")
    assert it_b < it_c
    from oracle import blockprec
    for (p, G, GT, D, lj), mb, inf in zip(b, o_b, i_b):
        grid = (p.nx, p.ny, p.nz)
        P = blockprec.block_precond(GT, grid, p.w, p.lam)
        for j in (0, D.shape[1] // 2, D.shape[1] - 1):
            ref = oracle.lsqr(G, GT, grid, p.w, lj[j], D[:, j], atol=1e-12, btol=1e-12,
                              itmax=50000)
            same = oracle.lsqr(G, GT, grid, p.w, 0.0, D[:, j], atol=1e-6, btol=1e-6,
                               itmax=50000, P=P, lam_rows=lj[j])
            assert inf[j]["istop"] in (1, 2)
            e32 = rel(mb[:, j].cpu().numpy(), ref.x)
            e_or = rel(blockprec.apply_blocks(P, same.x), ref.x)
            assert e32 <= 2.0 * e_or + 1e-3, (p.nz, j, e32, e_or)
    with pytest.raises(pdst.PdstError, match="PDST_ERR_STATE"):
        fresh = pdst.build_G_problem(b[0][0], dtypes=("f32",), formats=("blocked",))
        pdst.lsqr_batched([fresh], [ds[0]], [1.0], [lams[0]], 10, 1e-6, dtype="f32", precond=2)


# ------------------------------------------------ deeper systems (nz > 16)
# A batch with a system of more than 16 depth nodes runs the adjoint kernels
# that hold 32 depths per lane, for all of its systems.

def wide_batch():
    probs = [synth.custom(9, 8, 20, 12, 4, bend=0.15, seed=61, w=1.0, lam=0.1, dz_km=1.0),
             synth.custom(10, 7, 8, 10, 3, bend=0.1, seed=62, w=2.0, lam=0.05),
             synth.custom(6, 6, 27, 8, 3, bend=0.15, seed=63, w=0.5, lam=0.2, dz_km=1.0)]
    nrhs = [16, 5, 3]
    out = []
    for p, R in zip(probs, nrhs):
        G = oracle.build_G_problem(p)
        cols, lams = [], []
        for j in range(R):
            m = synth.checkerboard(p.nx, p.ny, p.nz, 2 + (j % 5), 0.05) * (1 if j % 2 else -1)
            cols.append(oracle.rhs_for(p, G, m_model=m, noise=synth.rhs_noise(p.seed, p.m_rows, j)))
            lams.append(float(np.logspace(-3, 0, R)[j]) if R > 1 else p.lam)
        out.append((p, G, oracle.transpose(G), np.stack(cols, axis=1), lams))
    return out


@pytest.fixture(scope="module")
def wide():
    require_cuda()
    b = wide_batch()
    hs = [pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
          for p, *_ in b]
    yield b, hs
    for h in hs:
        h.close()


@pytest.mark.parametrize("k", [1, 4])
def test_wide_batch_fixed_k_match_oracle(wide, k):
    """nz = 20, 8 and 27 in one batch: unscaled and with the oracle's depth
    blocks, FP64, element by element against the oracle."""
    from oracle import blockprec
    b, hs = wide
    ds = [to_dev(D) for _, _, _, D, _ in b]
    w = [p.w for p, *_ in b]
    lams = [l for *_, l in b]
    outs, infos, _ = pdst.lsqr_batched(hs, ds, w, lams, k, 0.0, dtype="f64", tile_rows=4)
    for (p, G, GT, D, lj), mo, inf in zip(b, outs, infos):
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, lj[j], D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k)
            assert inf[j]["iters"] == k
            assert rel(mo[:, j].cpu().numpy(), ref.x) < 1e-10, (p.nz, j, k)
    Ps = []
    for (p, G, GT, *_), h in zip(b, hs):
        P = blockprec.block_precond(GT, (p.nx, p.ny, p.nz), p.w, p.lam)
        h.set_block_precond(to_dev(P), p.w, p.lam)
        Ps.append(P)
    outs, infos, _ = pdst.lsqr_batched(hs, ds, w, lams, k, 0.0, dtype="f64", tile_rows=4,
                                       precond=2)
    for (p, G, GT, D, lj), P, mo, inf in zip(b, Ps, outs, infos):
        for j in range(D.shape[1]):
            ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, D[:, j], atol=0, btol=0,
                              conlim=0, itmax=k, P=P, lam_rows=lj[j])
            assert rel(mo[:, j].cpu().numpy(), blockprec.apply_blocks(P, ref.x)) < 1e-10, \
                (p.nz, j, k)


def test_wide_batch_converged_fp32_and_limit(wide):
    b, hs = wide
    ds = [to_dev(D) for _, _, _, D, _ in b]
    w = [p.w for p, *_ in b]
    lams = [l for *_, l in b]
    for (p, *_), h in zip(b, hs):
        h.set_block_precond(None, p.w, p.lam)
    outs, infos, _ = pdst.lsqr_batched(hs, ds, w, lams, 20000, 1e-6, dtype="f32", precond=2)
    from oracle import blockprec
    for (p, G, GT, D, lj), mo, inf in zip(b, outs, infos):
        grid = (p.nx, p.ny, p.nz)
        P = blockprec.block_precond(GT, grid, p.w, p.lam)
        for j in (0, D.shape[1] - 1):
            ref = oracle.lsqr(G, GT, grid, p.w, lj[j], D[:, j], atol=1e-12, btol=1e-12,
                              itmax=50000)
            same = oracle.lsqr(G, GT, grid, p.w, 0.0, D[:, j], atol=1e-6, btol=1e-6,
                               itmax=50000, P=P, lam_rows=lj[j])
            assert inf[j]["istop"] in (1, 2)
            e32 = rel(mo[:, j].cpu().numpy(), ref.x)
            e_or = rel(blockprec.apply_blocks(P, same.x), ref.x)
            assert e32 <= 2.0 * e_or + 1e-3, (p.nz, j, e32, e_or)
    deep = synth.custom(4, 4, 34, 6, 2, bend=0.0, seed=64)
    hd = pdst.build_G_problem(deep, dtypes=("f32",), formats=("blocked",))
    dd = to_dev(np.zeros((hd.m, 1)))
    with pytest.raises(pdst.PdstError, match="PDST_ERR_LIMIT"):
        pdst.lsqr_batched([hd], [dd], [1.0], [[0.1]], 10, 1e-6, dtype="f32")
    hd.close()
