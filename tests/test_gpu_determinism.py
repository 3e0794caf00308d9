"""Bit-reproducibility on a system whose cells are split over several adjoint
work items (64 x 64 x 16: about 1,700 rows per cell, items of 512 rows).

The item that finishes such a cell depends on arrival order; its sum of
squares goes to the cell's slot and is added in cell order, so every
reduction, and so every iterate, has the same bits from run to run.
"""
import numpy as np
import pytest

from paper_2604_11920_b300 import pdst, synth
from gpu_util import require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mid():
    require_cuda()
    import torch
    p = synth.mid()
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("blocked",))
    d = torch.from_numpy(p.noise).cuda()
    yield p, h, d
    h.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_repeat_solves_identical(mid, dtype):
    p, h, d = mid
    runs = [h.lsqr(d, p.w, p.lam, 60, 0.0, dtype=dtype, fmt="blocked", conlim=1e300)
            for _ in range(3)]
    for r in runs[1:]:
        assert r.info["rnorm"] == runs[0].info["rnorm"]
        assert np.array_equal(r.m.cpu().numpy(), runs[0].m.cpu().numpy())
    g = h.lsqr(d, p.w, p.lam, 60, 0.0, dtype=dtype, fmt="blocked", conlim=1e300,
               use_graph=False)
    assert np.array_equal(g.m.cpu().numpy(), runs[0].m.cpu().numpy())


def test_sweep_identical_on_multi_item_cells(mid):
    p, h, d = mid
    lams = [0.01, 0.05, 0.3]
    sw = h.lsqr_damping_sweep(d, p.w, lams, 200, 1e-5, dtype="f32", fmt="blocked")
    for lam, r in zip(lams, sw):
        one = h.lsqr(d, p.w, lam, 200, 1e-5, dtype="f32", fmt="blocked")
        assert np.array_equal(r.m.cpu().numpy(), one.m.cpu().numpy()), lam


def test_batched_repeat_identical(mid):
    import torch
    p, h, d = mid
    D = torch.stack([d, 0.5 * d, -d, 2.0 * d], dim=1).contiguous()
    lams = [[p.lam, 0.01, 0.1, 1.0]]
    o1, _, _ = pdst.lsqr_batched([h], [D], [p.w], lams, 40, 0.0, dtype="f32", tile_rows=8)
    o2, _, _ = pdst.lsqr_batched([h], [D], [p.w], lams, 40, 0.0, dtype="f32", tile_rows=8)
    assert np.array_equal(o1[0].cpu().numpy(), o2[0].cpu().numpy())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_launch_modes_give_the_same_bits(mid, dtype):
    """The graph replay launches each sweep with programmatic dependent launch
    (its blocks scheduled while the kernel before it finishes); the profiled
    replay launches the same kernels plainly between event nodes, and profile
    mode 1 one at a time with the scalar step in line.  Same arithmetic in the
    same order, so the iterates and estimates are identical bit for bit, with
    the depth blocks as well."""
    p, h, d = mid
    h.set_block_precond(None, p.w, p.lam)
    for precond in (0, 2):
        kw = dict(dtype=dtype, fmt="blocked", conlim=1e300, precond=precond)
        base = h.lsqr(d, p.w, p.lam, 40, 0.0, **kw)
        for extra in ({"profile": 2}, {"profile": 1}, {"use_graph": False}):
            r = h.lsqr(d, p.w, p.lam, 40, 0.0, **kw, **extra)
            assert r.info["iters"] == base.info["iters"] == 40
            assert r.info["rnorm"] == base.info["rnorm"], (precond, extra)
            assert np.array_equal(r.m.cpu().numpy(), base.m.cpu().numpy()), (precond, extra)
