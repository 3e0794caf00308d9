"""GPU parity of the G assembly (Eq. 5-7) against the FP64 oracle.

Indices must match exactly; FP64 values bit for bit (both sides evaluate the
same recipe with one rounding per operation); FP32 values are the exact
round-to-nearest casts of the FP64 values; BF16 values the exact
round-to-nearest-even casts.
"""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_bf16_rne, to_dev

pytestmark = pytest.mark.gpu


def edge_problem():
    """Ragged case: nz = 3 (not a multiple of 4), 13 x 7 cells of 1.5 km, bent
    rays, plus a zero-length ray, a ray mostly outside the grid and a ray on a
    cell edge."""
    p = synth.custom(13, 7, 3, 17, 5, bend=0.15, seed=21, dx_km=1.5)
    extra = np.array([[4.0, 4.0, 4.0, 4.0, 4.0, 4.0],          # zero length: empty row
                      [-5.0, -3.0, 30.0, -1.0, 40.0, 20.0],     # mostly outside: clamped
                      [0.0, 3.0, 9.75, 3.0, 19.5, 3.0]])        # along y = 2 dx
    p.ctrl = np.vstack([p.ctrl, extra])
    p.row_period = np.concatenate([p.row_period, np.array([0, 2, 4], np.int32)])
    return p


CASES = {"tiny": synth.tiny, "edge": edge_problem,
         "ragged_nz8": lambda: synth.custom(9, 11, 8, 12, 7, bend=0.15, seed=5)}


@pytest.mark.parametrize("name", sorted(CASES))
def test_csr_csc_bit_exact(name):
    require_cuda()
    p = CASES[name]()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "bf16"))
    assert (h.m, h.n, h.nnz) == (G.n_rows, G.n_cols, G.nnz)
    ptr, idx, val = h.export_csr("f64")
    assert np.array_equal(ptr, G.ptr)
    assert np.array_equal(idx, G.idx)
    assert np.array_equal(val, G.val)
    cptr, cidx, cval = h.export_csc("f64")
    assert np.array_equal(cptr, GT.ptr)
    assert np.array_equal(cidx, GT.idx)
    assert np.array_equal(cval, GT.val)
    _, _, v32 = h.export_csr("f32")
    assert np.array_equal(v32, G.val.astype(np.float32).astype(np.float64))
    _, _, t32 = h.export_csc("f32")
    assert np.array_equal(t32, GT.val.astype(np.float32).astype(np.float64))
    _, _, vbf = h.export_csr("bf16")
    assert np.array_equal(vbf, to_bf16_rne(G.val))
    h.close()


def test_blocked_only_handle_exports_same_matrix():
    require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    h = pdst.build_G_problem(p, formats=("blocked",))
    ptr, idx, val = h.export_csr("f64")
    assert np.array_equal(ptr, G.ptr) and np.array_equal(idx, G.idx)
    assert np.array_equal(val, G.val)
    cptr, cidx, _ = h.export_csc("f64")
    assert np.array_equal(cptr, GT.ptr) and np.array_equal(cidx, GT.idx)


def test_empty_system():
    require_cuda()
    p = synth.custom(4, 4, 2, 2, 1, bend=0.0, seed=1)
    h = pdst.build_G(p.nx, p.ny, p.nz, p.dx_km, p.dz_km, np.zeros((0, 6)),
                     np.zeros(0, np.int32), p.n_periods, p.kdz)
    assert h.m == 0 and h.nnz == 0 and h.n == 32
    ptr, _, _ = h.export_csr("f64")
    assert ptr.tolist() == [0]


def test_bad_inputs_rejected():
    require_cuda()
    p = synth.custom(4, 4, 2, 5, 2, bend=0.1, seed=2)
    bad = p.ctrl.copy()
    bad[3, 2] = np.nan
    with pytest.raises(pdst.PdstError, match="non-finite"):
        pdst.build_G(p.nx, p.ny, p.nz, p.dx_km, p.dz_km, bad, p.row_period, p.n_periods, p.kdz)
    per = p.row_period.copy()
    per[0] = 7
    with pytest.raises(pdst.PdstError, match="period index"):
        pdst.build_G(p.nx, p.ny, p.nz, p.dx_km, p.dz_km, p.ctrl, per, p.n_periods, p.kdz)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("fmt", ["element", "blocked"])
def test_apply_G_matches_oracle(dtype, fmt):
    torch = require_cuda()
    for p in (synth.tiny(), edge_problem()):
        G = oracle.build_G_problem(p)
        if dtype == "f32":
            G.val = G.val.astype(np.float32).astype(np.float64)
        elif dtype == "bf16":
            G.val = to_bf16_rne(G.val)
        GT = oracle.transpose(G)
        h = pdst.build_G_problem(p, dtypes=(dtype,), formats=(fmt,))
        rng = np.random.default_rng(4)
        x = rng.standard_normal(h.n)
        y = torch.zeros(h.m, dtype=torch.float64, device="cuda")
        h.apply_G(to_dev(x), y, dtype=dtype)
        assert rel(y.cpu().numpy(), oracle.spmv(G, x)) < 1e-13
        u = rng.standard_normal(h.m)
        z = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        h.apply_G(to_dev(u), z, trans=True, dtype=dtype)
        assert rel(z.cpu().numpy(), oracle.spmv(GT, u)) < 1e-13


def test_full_size_64x64x16_sampled_rows():
    """64x64x16 grid, 171,360 rows (the benchmark system): 3,000 sampled rows
    rebuilt one by one by the oracle match the GPU rows bit for bit, and the
    GPU transpose is exactly the transpose of the GPU CSR."""
    require_cuda()
    import scipy.sparse as sp
    p = synth.mid()
    h = pdst.build_G_problem(p, dtypes=("f64",))
    ptr, idx, val = h.export_csr("f64")
    rows = np.sort(np.random.default_rng(8).choice(p.m_rows, 3000, replace=False))
    G = oracle.build_G(p.nx, p.ny, p.nz, p.dx_km, p.ctrl[rows], p.row_period[rows], p.kdz)
    for i, r in enumerate(rows):
        lo, hi = ptr[r], ptr[r + 1]
        assert np.array_equal(idx[lo:hi], G.idx[G.ptr[i]:G.ptr[i + 1]])
        assert np.array_equal(val[lo:hi], G.val[G.ptr[i]:G.ptr[i + 1]])
    cptr, cidx, cval = h.export_csc("f64")
    T = sp.csr_matrix((val, idx, ptr), shape=(h.m, h.n)).T.tocsr()
    T.sort_indices()
    assert np.array_equal(cptr, T.indptr) and np.array_equal(cidx, T.indices)
    assert np.array_equal(cval, T.data)
    assert h.nnz == int(ptr[-1]) and np.all(np.diff(ptr) % p.nz == 0)
