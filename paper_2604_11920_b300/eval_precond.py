"""Evaluate the learned scaling on held-out systems against column-norm
scaling and no scaling, with the per-cell depth-block preconditioner beside
them (the benchmark's chosen form).

Per system: a tight reference solution (the training script's recipe), then
(1) the accuracy-matched metric of the benchmark -- LSQR iterations and time of
the two-phase FP32 solve to within 1e-4 of the reference, with column-norm and
with learned scaling (the refinement tolerance the loosest rung of the ladder
that gets there); (2) one FP32 solve to tol 1e-6 with no scaling, column-norm
and learned scaling: iterations, time and model error.  FP64 scalars
throughout.

Usage:  python -m paper_2604_11920_b300.eval_precond --mid 10 --large 2 \\
            --model paper_2604_11920_b300/precond_mlp.json
The summary is added to the model file under "eval".
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import pdst, synth
from .train_precond import (DEFAULT_OUT, accuracy_cost, learned_scaling, load_params, make_rhs,
                            reference, relerr)


def run_one(p, params):
    import torch
    h = pdst.build_G_problem(p, dtypes=("f64", "f32", "df64"), formats=("blocked",))
    d = make_rhs(h, p)
    m_ref = reference(h, p, d)
    out = {"seed": p.seed, "size": p.name}

    def timed(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.lsqr(d, p.w, p.lam, 200000, p.tol, dtype="f32", fmt="blocked", **kw)
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    def set_form(form):
        if form == "colnorm":
            h.set_col_scaling_power(p.w, p.lam, 1.0)
        elif form == "learned":
            learned_scaling(h, p, params)
        elif form == "blocks":
            h.set_block_precond(None, p.w, p.lam)

    for form, pc in (("colnorm", 1), ("learned", 1), ("blocks", 2)):
        set_form(form)
        it, rt = accuracy_cost(h, p, d, m_ref, precond=pc)
        acc = {"iters": it, "refine_tol": rt, "s": None, "model_error": None}
        if it is not None:
            set_form(form)   # the scaling is part of the timed step
            r, t = timed(precond=pc, refine=3, refine_dtype="f32", refine_tol=rt)
            acc.update(s=t, model_error=relerr(r.m, m_ref))
        out[f"acc_{form}"] = acc
    for form, pc in (("none", 0), ("colnorm", 1), ("learned", 1), ("blocks", 2)):
        set_form(form)
        r, t = timed(precond=pc)
        out[form] = {"iters": r.info["iters"], "istop": r.info["istop"], "s": t,
                     "model_error": relerr(r.m, m_ref)}
    h.close()
    return out


def summarise(rows):
    s = {}
    for key in ("none", "colnorm", "learned", "blocks"):
        s[key] = {"mean_iters": float(np.mean([r[key]["iters"] for r in rows])),
                  "mean_s": float(np.mean([r[key]["s"] for r in rows])),
                  "mean_model_error": float(np.mean([r[key]["model_error"] for r in rows]))}
    for key in ("acc_colnorm", "acc_learned", "acc_blocks"):
        ok = [r[key] for r in rows if r[key]["iters"] is not None]
        s[key] = {"reached": len(ok), "of": len(rows),
                  "mean_iters": float(np.mean([a["iters"] for a in ok])) if ok else None,
                  "mean_s": float(np.mean([a["s"] for a in ok])) if ok else None}
    return s


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mid", type=int, default=10)
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
