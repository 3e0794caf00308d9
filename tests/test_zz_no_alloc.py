"""pdst_lsqr_noalloc, the allocation-free solve, against pdst_lsqr.

Callers that must not allocate device memory while they run (a serving or
plugin host that owns all device memory, a process under a hard memory cap,
a loop that cannot take cudaFree's device-wide synchronisation) use this entry
point: its scratch is one static device array in the library.  The test calls
it through the C ABI twice in a row -- the array keeps the previous call's
contents, so the second call checks that nothing stale leaks in -- and
compares each result with pdst_lsqr's within the tolerance of the fixed-k
parity tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import pdst, synth
from gpu_util import rel, require_cuda, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-10


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
        assert got.info["iters"] == ref.info["iters"] > 0
        assert got.info["istop"] == ref.info["istop"]
        assert rel(got.m.cpu().numpy(), ref.m.cpu().numpy()) <= TOL
        for key in ("rnorm", "arnorm", "anorm", "xnorm"):
            assert abs(got.info[key] - ref.info[key]) <= TOL * abs(ref.info[key])
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
