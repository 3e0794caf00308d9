#!/usr/bin/env python
"""Write the FP64 oracle's reference solution of a benchmark workload.

The stored vector is the oracle LSQR (Paige & Saunders 1982, run on the
oracle's own G of Eq. 5-7) at atol = btol = 1e-12 on a seeded workload:

* mid: the 64 x 64 x 16 system (generator seed 1: 120 stations, 7,140 pairs
  x 24 periods, Bezier rays, Gaussian blobs, 2 % noise, w = 2, lambda = 0.05);
* paper: the paper-shaped 20 x 37 x 18 system (seed 3: 229 stations, 26,106
  pairs x 14 periods, bilinear coefficients; the same noise and weights).

It is the m_ref against which the benchmark and the accuracy tests measure
||m - m_ref|| / ||m_ref||.  Only the oracle and the input generator run here.

    python tests/golden/make_mref.py [mid|paper]   # ~25 / ~40 min on 8 cores

The same run also records the oracle's own accuracy ladder: for each
tolerance t of LADDER, the iteration at which a solve with atol = btol = t
stops (S1 or S2) and the relative model error of that iterate against the
final solution -- what the oracle needs to come within 1e-4 of it.

Outputs beside this script: <workload>_mref.npy (the n FP64 values) and
<workload>_mref.json (seed, tolerance, iterations, stopping reason,
estimates, the ladder).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2604_11920_b300 import synth  # noqa: E402

TOL = 1e-12
WORKLOADS = {"mid": (synth.mid, 1, "mid_64x64x16"), "paper": (synth.paper_shaped, 3, "paper_20x37x18")}
LADDER = (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10)


def main(workload="mid"):
    gen, SEED, name = WORKLOADS[workload]
    oracle.build()
    p = gen(SEED)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    t0 = time.perf_counter()
    r = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=TOL, btol=TOL,
                    conlim=1e8, itmax=200000, checkpoints=LADDER)
    secs = time.perf_counter() - t0
    np.save(os.path.join(HERE, f"{workload}_mref.npy"), r.x)
    nref = float(np.linalg.norm(r.x))
    ladder = [{"tol": t, "iters": int(r.ck_itn[c]),
               "model_error": float(np.linalg.norm(r.ck_x[c] - r.x) / nref)}
              for c, t in enumerate(LADDER)]
    meta = {"workload": name, "seed": SEED, "w": p.w, "lambda": p.lam,
            "atol": TOL, "btol": TOL, "conlim": 1e8, "iters": r.itn, "istop": r.istop,
            "rnorm": r.rnorm, "arnorm": r.arnorm, "anorm": r.anorm, "acond": r.acond,
            "xnorm": r.xnorm, "bnorm": r.bnorm, "nnz": G.nnz, "rows": G.n_rows,
            "cols": G.n_cols, "oracle_threads": oracle.num_threads(),
            "oracle_seconds": round(secs, 1), "ladder": ladder,
            "rhs": "d = G m_true + 0.02 RMS(G m_true) z with the oracle's G (oracle.rhs_for)"}
    with open(os.path.join(HERE, f"{workload}_mref.json"), "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    print(json.dumps(meta))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "mid")
