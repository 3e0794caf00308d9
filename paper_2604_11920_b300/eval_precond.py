"""Evaluate the learned scaling on held-out systems against column-norm
scaling and no scaling: LSQR iterations to tol, time to tol and model error
against an FP64 reference solve (FP32 values, FP64 scalars in all three).

Usage:  python -m paper_2604_11920_b300.eval_precond --mid 20 --large 2 \\
            --model paper_2604_11920_b300/precond_mlp.json
The summary is added to the model file under "eval".
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import pdst, synth
from .train_precond import DEFAULT_OUT, learned_scaling, load_params, make_rhs


def run_one(p, params, ref_tol=1e-10):
    import torch
    h = pdst.build_G_problem(p, dtypes=("f64", "f32"), formats=("element", "blocked"))
    d = make_rhs(h, p)
    ref = h.lsqr(d, p.w, p.lam, 50000, ref_tol, dtype="f64")
    out = {"seed": p.seed, "size": p.name, "ref_iters": ref.info["iters"]}

    def timed(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.lsqr(d, p.w, p.lam, 20000, p.tol, dtype="f32", fmt="blocked", **kw)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(r.m - ref.m) / torch.linalg.norm(ref.m))
        return {"iters": r.info["iters"], "istop": r.info["istop"],
                "s": time.perf_counter() - t0, "model_error": err}

    out["none"] = timed(precond=0)
    h.set_col_scaling_power(p.w, p.lam, 1.0)
    out["colnorm"] = timed(precond=1)
    learned_scaling(h, p, params)
    out["learned"] = timed(precond=1)
    h.close()
    return out


def summarise(rows):
    s = {}
    for key in ("none", "colnorm", "learned"):
        s[key] = {"mean_iters": float(np.mean([r[key]["iters"] for r in rows])),
                  "mean_s": float(np.mean([r[key]["s"] for r in rows])),
                  "mean_model_error": float(np.mean([r[key]["model_error"] for r in rows]))}
    return s


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mid", type=int, default=20)
    ap.add_argument("--large", type=int, default=2)
    ap.add_argument("--first-seed", type=int, default=20000)
    ap.add_argument("--model", default=DEFAULT_OUT)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    params = load_params(args.model)
    rows_mid, rows_large = [], []
    for i in range(args.mid):
        r = run_one(synth.mid(args.first_seed + i), params)
        rows_mid.append(r)
        print(json.dumps(r), flush=True)
    for i in range(args.large):
        r = run_one(synth.large(args.first_seed + i), params)
        rows_large.append(r)
        print(json.dumps(r), flush=True)
    ev = {"held_out_seeds": [args.first_seed, args.first_seed + max(args.mid, args.large) - 1],
          "mid": {"systems": rows_mid, "summary": summarise(rows_mid) if rows_mid else None},
          "large": {"systems": rows_large, "summary": summarise(rows_large) if rows_large else None}}
    with open(args.model) as fh:
        rec = json.load(fh)
    rec["eval"] = ev
    with open(args.model, "w") as fh:
        json.dump(rec, fh)
    print(json.dumps({"mid": ev["mid"]["summary"], "large": ev["large"]["summary"]}))


if __name__ == "__main__":
    main()
