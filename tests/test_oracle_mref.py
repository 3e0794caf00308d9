"""The stored oracle solution of the 64 x 64 x 16 workload
(tests/golden/mid_mref.npy, written by tests/golden/make_mref.py, which
calls only the oracle) is what it claims to be: the metadata names this
system, and the solution satisfies the normal equations of the regularised
problem, A^T r = 0 with A = [G; w L; lambda I], to the stopping tolerance
(true residuals from the oracle's products, not LSQR's estimates)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.slow
def test_mid_mref_solves_the_normal_equations():
    meta = json.load(open(os.path.join(GOLDEN, "mid_mref.json")))
    m_ref = np.load(os.path.join(GOLDEN, "mid_mref.npy"))
    p = synth.mid(meta["seed"])
    assert (meta["w"], meta["lambda"]) == (p.w, p.lam) and meta["istop"] in (1, 2)
    G = oracle.build_G_problem(p)
    assert G.nnz == meta["nnz"] and m_ref.shape == (p.n,)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    grid = (p.nx, p.ny, p.nz)
    r = np.concatenate([d, np.zeros(p.n)]) - oracle.apply_A(G, grid, p.w, m_ref)
    atr = oracle.apply_At(GT, grid, p.w, r) - p.lam * p.lam * m_ref
    rn = np.sqrt(r @ r + p.lam ** 2 * (m_ref @ m_ref))
    ratio = np.linalg.norm(atr) / (meta["anorm"] * rn)
    assert ratio < 1e-10, ratio
    # the zero model is far from it: the check has teeth
    atr0 = oracle.apply_At(GT, grid, p.w, np.concatenate([d, np.zeros(p.n)]))
    assert np.linalg.norm(atr0) / (meta["anorm"] * np.linalg.norm(d)) > 1e-3
