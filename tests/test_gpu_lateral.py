"""Laterally varying depth kernels: a kernel table per horizontal cell, so G
is a general sparse matrix with the pattern of Eq. 5 but no l (x) Kdz
structure.  The device assembly matches the oracle bit for bit, and the solve
reaches the oracle's minimiser (nothing downstream relies on separability)."""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lateral():
    require_cuda()
    p = synth.tiny_lateral()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"))
    return p, G, GT, d, h


def test_lateral_G_bit_exact(lateral):
    p, G, GT, d, h = lateral
    ptr, idx, val = h.export_csr("f64")
    assert np.array_equal(ptr, G.ptr) and np.array_equal(idx, G.idx)
    assert np.array_equal(val, G.val)
    _, _, v32 = h.export_csr("f32")
    assert np.array_equal(v32, G.val.astype(np.float32).astype(np.float64))
    cptr, cidx, cval = h.export_csc("f64")
    assert np.array_equal(cptr, GT.ptr) and np.array_equal(cidx, GT.idx)
    assert np.array_equal(cval, GT.val)
    # the per-cell table was used: the separable table gives other values
    hs = pdst.build_G_problem(p, dtypes=("f64",), kdz_cells=None)
    assert not np.array_equal(hs.export_csr("f64")[2], val)
    hs.close()


@pytest.mark.parametrize("fmt", ["element", "blocked"])
def test_lateral_lsqr_matches_oracle(lateral, fmt):
    p, G, GT, d, h = lateral
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-12, btol=1e-12,
                      itmax=50000)
    k8 = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0, btol=0, conlim=0,
                     itmax=8)
    r8 = h.lsqr(to_dev(d), p.w, p.lam, 8, 0.0, fmt=fmt, conlim=1e300)
    assert rel(r8.m.cpu().numpy(), k8.x) < 1e-10
    res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-10, fmt=fmt)
    assert res.info["istop"] in (1, 2)
    assert rel(res.m.cpu().numpy(), ref.x) <= 1e-4


def test_lateral_bad_table_rejected(lateral):
    p, G, GT, d, h = lateral
    bad = p.kdz_cells.copy()
    bad[3, 1, 2] = np.nan
    with pytest.raises(pdst.PdstError):
        pdst.build_G_problem(p, dtypes=("f64",), kdz_cells=bad)
    with pytest.raises(ValueError):
        pdst.build_G_problem(p, dtypes=("f64",), kdz_cells=bad[:-1])


# ------------------------------------------------ bilinear node coefficients (Eq. 1)

@pytest.fixture(scope="module")
def bilinear():
    require_cuda()
    p = synth.tiny_bilinear()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"))
    return p, G, GT, d, h


def test_bilinear_G_bit_exact(bilinear):
    p, G, GT, d, h = bilinear
    ptr, idx, val = h.export_csr("f64")
    assert np.array_equal(ptr, G.ptr) and np.array_equal(idx, G.idx)
    assert np.array_equal(val, G.val)
    cptr, cidx, cval = h.export_csc("f64")
    assert np.array_equal(cptr, GT.ptr) and np.array_equal(cidx, GT.idx)
    assert np.array_equal(cval, GT.val)
    hc = pdst.build_G_problem(p, dtypes=("f64",), interp=0)
    assert hc.nnz < G.nnz          # the cell form touches fewer columns per row
    hc.close()


def test_bilinear_lsqr_matches_oracle(bilinear):
    p, G, GT, d, h = bilinear
    ref = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=1e-12, btol=1e-12,
                      itmax=50000)
    res = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-10, fmt="blocked")
    assert res.info["istop"] in (1, 2)
    assert rel(res.m.cpu().numpy(), ref.x) <= 1e-4
    r32 = h.lsqr(to_dev(d), p.w, p.lam, 50000, 1e-6, dtype="f32", fmt="blocked")
    assert r32.info["istop"] in (1, 2)


def test_bilinear_needs_two_nodes_per_axis(bilinear):
    p, G, GT, d, h = bilinear
    with pytest.raises(pdst.PdstError):
        pdst.build_G(1, 4, 2, 1.0, 2.0, p.ctrl[:3], p.row_period[:3], p.n_periods, p.kdz,
                     dtypes=("f64",), interp=1)
