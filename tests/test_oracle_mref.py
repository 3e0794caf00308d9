"""The stored oracle solutions of the 64 x 64 x 16 and the paper-shaped
workloads (tests/golden/<workload>_mref.npy, written by
tests/golden/make_mref.py, which calls only the oracle) are what they claim
to be: the metadata names the system, and the solution satisfies the normal
equations of the regularised problem, A^T r = 0 with A = [G; w L; lambda I],
to the stopping tolerance (true residuals from the oracle's products, not
LSQR's estimates); the oracle's own ladder reaches the benchmark's 1e-4."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2604_11920_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.slow
@pytest.mark.parametrize("workload", ["mid", "paper"])
def test_mref_solves_the_normal_equations(workload):
    meta = json.load(open(os.path.join(GOLDEN, f"{workload}_mref.json")))
    m_ref = np.load(os.path.join(GOLDEN, f"{workload}_mref.npy"))
    p = {"mid": synth.mid, "paper": synth.paper_shaped}[workload](meta["seed"])
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
    # the ladder: iterations grow and the error falls with the tolerance
    lad = meta["ladder"]
    assert all(a["iters"] <= b["iters"] for a, b in zip(lad, lad[1:]))
    assert any(r["model_error"] <= 1e-4 for r in lad)
