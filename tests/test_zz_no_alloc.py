"""pdst_lsqr_noalloc, the allocation-free solve, against pdst_lsqr and the oracle.

Callers that must not allocate device memory while they run (a serving or
plugin host that owns all device memory, a process under a hard memory cap,
a loop that cannot take cudaFree's device-wide synchronisation) use this entry
point: its scratch is one static device array in the library.  The test calls
it through the C ABI twice in a row -- the array keeps the previous call's
contents, so the second call checks that nothing stale leaks in -- and
compares each result with pdst_lsqr's: the same kernels run in the same
order, so the models and the reported fields agree bit for bit.  One more
case runs the column-scaled operator with lambda rows appended (which moves
every later carve of the array), and one compares a fixed-k run with the FP64
oracle directly.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

FIELDS = ("iters", "istop", "rnorm", "arnorm", "anorm", "acond", "xnorm", "bnorm")


def _same(got, ref):
    assert np.array_equal(got.m.cpu().numpy(), ref.m.cpu().numpy())
    for key in FIELDS:
        assert got.info[key] == ref.info[key], key


def test_noalloc_matches_lsqr_on_two_calls_in_a_row():
    torch = require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"))
    cases = [(to_dev(d), dict(dtype="f64", fmt="element"), 400, 1e-8),
             (to_dev(-0.5 * d), dict(dtype="f32", fmt="blocked"), 300, 1e-6)]
    for dd, form, itmax, tol in cases:
        ref = h.lsqr(dd, p.w, p.lam, itmax, tol, **form)
        out = torch.full((h.n,), float("nan"), dtype=torch.float64, device="cuda")
        got = h.lsqr_noalloc(dd, p.w, p.lam, itmax, tol, out, **form)
        assert got.info["iters"] > 0
        _same(got, ref)
    h.close()


def test_noalloc_scaled_with_lambda_rows_and_oracle():
    """precond = 1 with lambda > 0 appends the lambda D rows (M = m + 2n):
    equal to pdst_lsqr bit for bit, and at a fixed iteration count equal to
    the oracle's scaled LSQR within the FP64 fixed-k bar."""
    torch = require_cuda()
    p = synth.tiny()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    h = pdst.build_G_problem(p, dtypes=("f64",))
    D = 1.0 / np.sqrt(oracle.aug_colnorm2(GT, p.nx, p.ny, p.nz, p.w, p.lam))
    h.set_col_scaling(to_dev(D))
    dd = to_dev(d)
    for fmt in ("element", "blocked"):
        ref = h.lsqr(dd, p.w, p.lam, 500, 1e-8, fmt=fmt, precond=1)
        out = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        _same(h.lsqr_noalloc(dd, p.w, p.lam, 500, 1e-8, out, fmt=fmt, precond=1), ref)
    k = 6
    o = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, 0.0, d, atol=0, btol=0, conlim=0, itmax=k,
                    D=D, lam_rows=p.lam)
    out = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    got = h.lsqr_noalloc(dd, p.w, p.lam, k, 0.0, out, fmt="blocked", precond=1, conlim=1e300)
    assert got.info["iters"] == k
    assert rel(got.m.cpu().numpy(), D * o.x) < 1e-10
    with pytest.raises(pdst.PdstError, match="PDST_ERR_ARG"):
        h.lsqr_noalloc(dd, p.w, p.lam, 10, 1e-6, out, refine=2)
    h.close()


def test_noalloc_rejects_a_system_beyond_its_scratch():
    torch = require_cuda()
    p = synth.custom(400, 400, 8, 6, 1, bend=0.0, seed=4)   # 1.28 M unknowns, 15 rays
    h = pdst.build_G_problem(p, dtypes=("f64",))
    d = torch.zeros(h.m, dtype=torch.float64, device="cuda")
    out = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    with pytest.raises(pdst.PdstError, match="PDST_ERR_LIMIT"):
        h.lsqr_noalloc(d, 1.0, 0.1, 10, 1e-6, out)
    h.close()
