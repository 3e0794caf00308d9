#!/usr/bin/env python
"""Benchmark: LSQR time-to-tolerance of the regularised traveltime solve.

Workload (default): the 64 x 64 x 16 system (65,536 unknowns; 120 stations,
7,140 pairs x 24 periods = 171,360 rows; Bezier rays; Gaussian-blob model,
2 % noise; w = 2, lambda = 0.05; tol 1e-6), synthetic inputs from the seeded
generator.  One step = one LSQR solve to tolerance on the device-resident G
(forward product, adjoint product, FP64 recurrence and x/w update, all in the
library's kernels, replayed from a CUDA graph).  The G assembly is timed
separately (`build_G_s`).

Reported beside the headline: the plain FP64 GPU LSQR on the same system (FP64
values and vectors, element CSR/CSC, no scaling, graph on), the model error of
both against an FP64 reference solve, a per-kernel roofline from CUDA events,
the end-to-end time through the host entry point, and the FP64 CPU oracle
timed on this machine's cores on a bounded sample.

`--impl reference` times the FP64 CPU oracle alone (the comparison arm).
Multi-GPU (torchrun): every rank solves its own system (seed + rank); no data
moves between ranks ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR time-to-tol (s) & SpMV/SpMV^T HBM GB/s vs plain FP64 GPU LSQR, 1xB300"

FORMS = {
    # name: (dtype, format, precond); precond 1 = column-norm, 2 = learned scaling
    "f64-element": ("f64", "element", 0),
    "f64-blocked": ("f64", "blocked", 0),
    "df64-blocked": ("df64", "blocked", 0),
    "f32-element": ("f32", "element", 0),
    "f32-blocked": ("f32", "blocked", 0),
    "f32-blocked-colnorm": ("f32", "blocked", 1),
    "bf16-blocked-colnorm": ("bf16", "blocked", 1),
    "f32-blocked-learned": ("f32", "blocked", 2),
}
PLAIN = "f64-element"
MODEL_PATH = os.path.join(ROOT, "paper_2604_11920_b300", "precond_mlp.json")
DEFAULT_FORM = "f32-blocked-learned" if os.path.exists(MODEL_PATH) else "f32-blocked-colnorm"
ACC_TARGET = 1e-4                     # relative model error vs the FP64 reference
TOL_LADDER = (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10)
REFINE_DTYPE = "f32"                  # refinement sweeps of the reduced-precision forms
REF_TOL = 1e-12                       # FP64 reference solve (stops earlier on S4-S6 if need be)
VALUE_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "df64": 8}
VEC_BYTES = {"f64": 8, "f32": 4, "bf16": 4, "df64": 8}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pdst", "reference"], default="pdst")
    ap.add_argument("--workload", choices=["mid", "tiny", "large", "paper"], default="mid")
    ap.add_argument("--form", choices=sorted(FORMS), default=DEFAULT_FORM)
    ap.add_argument("--cpu-sample-iters", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-workload section (64 systems x 16 right-hand sides)")
    ap.add_argument("--batched-systems", type=int, default=64)
    ap.add_argument("--only-batched", action="store_true",
                    help="print the batched-workload section alone")
    ap.add_argument("--no-lsmr", action="store_true", help="skip the LSMR section")
    ap.add_argument("--no-sweep", action="store_true", help="skip the damping-sweep section")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy-matched ladder (skipped by default on "
                         "--workload large, whose FP64 ladder takes tens of minutes)")
    ap.add_argument("--accuracy", action="store_true",
                    help="run the accuracy-matched ladder on --workload large too")
    ap.add_argument("--ref-tol", type=float, default=None,
                    help="tolerance of the FP64 reference solve (default 1e-12; 1e-10 "
                         "on --workload large)")
    ap.add_argument("--only-solve", action="store_true",
                    help="time the chosen form only (for profiler runs)")
    ap.add_argument("--ncu-case", action="store_true",
                    help="small profiler case: build G in the chosen form only and run 3 "
                         "LSQR iterations with plain launches (no timing)")
    args = ap.parse_args()
    if args.workload == "large" and not args.accuracy:
        args.no_accuracy = True
    if args.ref_tol is None:
        args.ref_tol = 1e-10 if args.workload == "large" else REF_TOL
    return args


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks: the slowest replica sets the job time."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def make_problem(name, rank):
    from paper_2604_11920_b300 import synth
    return {"mid": synth.mid, "tiny": synth.tiny, "large": synth.large,
            "paper": synth.paper_shaped}[name](
        seed={"mid": 1, "tiny": 0, "large": 2, "paper": 3}[name] + 1000 * rank)


def workload_desc(p):
    extra = ", bilinear node coefficients" if getattr(p, "interp", 0) else ""
    return (f"{p.nx}x{p.ny}x{p.nz} grid ({p.n} unknowns), {p.stations.shape[0]} stations, "
            f"{p.pairs.shape[0]} pairs x {p.n_periods} periods = {p.m_rows} rows, "
            f"w={p.w}, lambda={p.lam}, tol={p.tol}{extra}")


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, enabled: bool = True):
        self.idx = device_index
        self.proc = None
        self.path = None
        self.enabled = enabled

    def __enter__(self):
        if not self.enabled:
            return self
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p > 0.3 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


# ------------------------------------------------------------- roofline

def algorithmic_bytes(h, p, dtype, fmt, scaled):
    """Bytes each kernel must move once per launch: matrix arrays read once,
    vectors read/written once, gathered vectors counted once (L2-resident)."""
    vb, xb = VALUE_BYTES[dtype], VEC_BYTES[dtype]
    m, n, nnz, nz = h.m, h.n, h.nnz, p.nz
    U, H = nnz // nz, p.nx * p.ny
    M = m + n + (n if scaled else 0)
    if fmt == "element":
        fwd_idx = 4 * nnz + 8 * (m + 1)
        adj_idx = 4 * nnz + 8 * (n + 1)
    else:
        fwd_idx = 4 * U + 8 * (m + 1)
        adj_idx = 4 * U + 8 * (H + 1) + 4 * H
    fwd = vb * nnz + fwd_idx + 2 * xb * M + xb * n
    adj = vb * nnz + adj_idx + xb * M + 2 * xb * n + (xb * n + 8 * n if scaled else 0)
    upd = xb * n + 8 * n * 3
    return {"fwd": fwd, "adj": adj, "upd": upd}


def dram_traffic_record(kernel, form, workload):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"```json\n(.*?)\n```", open(path).read(), re.S)
    if not m:
        return None
    try:
        rec = json.loads(m.group(1))
    except json.JSONDecodeError:
        return None
    src = os.path.join(ROOT, "paper_2604_11920_b300", "csrc", "lsqr.cu")
    digest = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    for r in rec.get("records", []):
        if (r.get("kernel") == kernel and r.get("form") == form and r.get("workload") == workload
                and r.get("lsqr_cu_sha1") == digest):
            return r.get("bytes_per_launch")
    return None


# ------------------------------------------------------------------ arms

def run_ncu_case(args):
    """Three LSQR iterations of the chosen form with plain launches: the case
    profiled by ncu (one k_fwd and one k_adj launch per iteration)."""
    import torch

    from paper_2604_11920_b300 import pdst
    torch.cuda.set_device(0)
    p = make_problem(args.workload, 0)
    dtype, fmt, precond = FORMS[args.form]
    h = pdst.build_G_problem(p, dtypes=(dtype,), formats=(fmt,))
    d = torch.from_numpy(p.noise).cuda()
    if precond:   # learned and column-norm scaling run the same kernels
        h.set_col_scaling(None, p.w, p.lam)
    r = h.lsqr(d, p.w, p.lam, 3, 0.0, dtype=dtype, fmt=fmt, precond=1 if precond else 0,
               use_graph=False)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.form, "iters": r.info["iters"], "nnz": h.nnz}))
    h.close()


def run_pdst(args, rank, world):
    import torch

    from paper_2604_11920_b300 import pdst

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    pdst.load()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    p = make_problem(args.workload, rank)
    dtype, fmt, precond = FORMS[args.form]
    dtypes = sorted({"f64", "df64", "f32", dtype})   # f32, df64: the refinement sweeps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = pdst.build_G_problem(p, dtypes=tuple(dtypes))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0

    # right-hand side d = G m_true + 2 % noise (input synthesis on the device)
    mt = torch.from_numpy(p.m_true).cuda()
    gm = torch.empty(h.m, dtype=torch.float64, device="cuda")
    h.apply_G(mt, gm, dtype="f64")
    rms = torch.sqrt(torch.mean(gm * gm))
    d = gm + p.noise_frac * rms * torch.from_numpy(p.noise).cuda()
    itmax = p.itmax
    params = None
    if precond == 2:
        from paper_2604_11920_b300.train_precond import learned_scaling, load_params
        params = load_params(MODEL_PATH)

    def set_scaling(pc):
        if pc == 1:
            h.set_col_scaling_power(p.w, p.lam, 1.0)
        elif pc == 2:
            learned_scaling(h, p, params)     # features + MLP, inside the step

    def solve(form, tol=p.tol, **kw):
        dt, fm, pc = FORMS[form]
        set_scaling(pc)
        return h.lsqr(d, p.w, p.lam, itmax, tol, dtype=dt, fmt=fm, precond=1 if pc else 0, **kw)

    def timed(form, steps, warmup, **kw):
        for _ in range(warmup):
            solve(form, **kw)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        e0.record(stream)
        for _ in range(steps):
            r = solve(form, **kw)
            launches += r.info["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
        return ms, r, launches

    with ClockSampler(dev, enabled=not args.no_clocks) as clk:
        ms, res, launches = timed(args.form, args.steps, args.warmup)
    clocks = clk.summary()
    if args.only_solve:
        if rank == 0:
            print(json.dumps({"form": args.form, "ms_per_solve": ms, "iters": res.info["iters"],
                              "istop": res.info["istop"]}))
        return

    out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype, "data": "synthetic (seeded generator; no dataset)"}
    m_chosen = res.m.clone()
    it_chosen = res.info["iters"]

    # plain FP64 GPU LSQR on the same system
    if args.form != PLAIN:
        ms_plain, res_plain, _ = timed(PLAIN, max(1, min(args.steps, 3)), 1)
    else:
        ms_plain, res_plain = ms, res
    m_plain = res_plain.m.clone()
    # FP64 reference solution: plain form at tol REF_TOL (its iteration count is reported)
    ref = h.lsqr(d, p.w, p.lam, 200000, args.ref_tol, dtype="f64", fmt="element")

    def relerr(a):
        return float(torch.linalg.norm(a - ref.m) / torch.linalg.norm(ref.m))

    # time to reach the FP64 reference within ACC_TARGET.  Plain FP64: loosest
    # tolerance of the ladder that gets there.  Reduced-precision forms: one
    # solve stalls near the FP32 accuracy limit (large-residual problem), so
    # they run two-phase: the form's solve to tol, then refinement sweeps on the
    # FP64 residual (FP32 values; each sweep starts from the exact residual, so
    # the FP32 operator only slows the contraction) with the loosest tolerance
    # of the ladder that gets there; double-float sweeps reported beside.
    def to_accuracy(form, refine_dtype=REFINE_DTYPE):
        dt, fm, pc = FORMS[form]
        err = None
        for t in TOL_LADDER:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if dt == "f64":
                set_scaling(pc)
                r = h.lsqr(d, p.w, p.lam, 100000, t, dtype=dt, fmt=fm, precond=1 if pc else 0)
            else:
                set_scaling(pc)
                r = h.lsqr(d, p.w, p.lam, 100000, p.tol, dtype=dt, fmt=fm,
                           precond=1 if pc else 0, refine=3, refine_dtype=refine_dtype,
                           refine_tol=t)
            e1.record(stream)
            torch.cuda.synchronize()
            err = relerr(r.m)
            if err <= ACC_TARGET:
                if dt != "f64":
                    return {"refine_tol": t, "refine_dtype": refine_dtype,
                            "s": e0.elapsed_time(e1) / 1e3, "iters": r.info["iters"],
                            "sweeps": r.info["sweeps"], "model_error": err}
                return {"tol": t,
                        "s": e0.elapsed_time(e1) / 1e3, "iters": r.info["iters"],
                        "sweeps": r.info["sweeps"], "model_error": err}
        return {"s": None, "iters": None, "model_error": err}

    if args.no_accuracy:
        accuracy_matched = None
    else:
        acc_chosen = to_accuracy(args.form)
        acc_plain = to_accuracy(PLAIN)
        accuracy_matched = {"target_model_error": ACC_TARGET, "chosen": acc_chosen,
                            "plain_fp64": acc_plain,
                            "speedup": (acc_plain["s"] / acc_chosen["s"])
                            if acc_plain["s"] and acc_chosen["s"] else None}
        # the column-norm form as well: the learned scaling is trained for the
        # FP32 solve, not for the refinement sweeps
        if args.form != "f32-blocked-colnorm":
            acc_cn = to_accuracy("f32-blocked-colnorm")
            accuracy_matched["f32-blocked-colnorm"] = acc_cn
            if acc_plain["s"] and acc_cn["s"]:
                accuracy_matched["speedup_colnorm"] = acc_plain["s"] / acc_cn["s"]
        # the same two-phase solve with double-float refinement sweeps
        acc_df = to_accuracy(args.form, "df64")
        accuracy_matched["df64_refinement"] = acc_df
        if acc_plain["s"] and acc_df["s"]:
            accuracy_matched["speedup_df64_refinement"] = acc_plain["s"] / acc_df["s"]

    # LSMR (the paper's solver) on the same sweeps: chosen form and plain FP64
    lsmr_sec = None
    if not args.no_lsmr:
        ms_l, res_l, _ = timed(args.form, max(1, min(args.steps, 3)), 1, method="lsmr")
        ms_lp, res_lp, _ = timed(PLAIN, 1, 1, method="lsmr")
        lsmr_sec = {"chosen": {"s": ms_l / 1e3, "iters": res_l.info["iters"],
                               "istop": res_l.info["istop"],
                               "model_error_vs_fp64_ref": relerr(res_l.m)},
                    "plain_fp64": {"s": ms_lp / 1e3, "iters": res_lp.info["iters"],
                                   "model_error_vs_fp64_ref": relerr(res_lp.m)},
                    "speedup_vs_plain_fp64": ms_lp / ms_l}

    # damping sweep: 8 damping values from one bidiagonalisation vs 8 solves
    sweep_sec = None
    if not args.no_sweep:
        lams = [float(10.0 ** (-3 + 3 * i / 7)) for i in range(8)]   # logspace(-3, 0, 8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sw = h.lsqr_damping_sweep(d, p.w, lams, itmax, p.tol, dtype="f32", fmt="blocked")
        torch.cuda.synchronize()
        t_sweep = time.perf_counter() - t0
        t0 = time.perf_counter()
        sep = [h.lsqr(d, p.w, lm, itmax, p.tol, dtype="f32", fmt="blocked") for lm in lams]
        torch.cuda.synchronize()
        t_sep = time.perf_counter() - t0
        sweep_sec = {"lambdas": lams, "form": "f32-blocked (no scaling)",
                     "sweep_s": t_sweep, "separate_s": t_sep, "speedup": t_sep / t_sweep,
                     "iters": [r.info["iters"] for r in sw],
                     "identical_to_separate": all(
                         bool(torch.equal(a.m, b.m)) for a, b in zip(sw, sep))}

    # per-kernel device time (events around each launch, same solve)
    prof = solve(args.form, profile=True)
    pi = max(prof.info["profiled_iters"], 1)
    kms = {"fwd": prof.info["fwd_ms"] / pi, "adj": prof.info["adj_ms"] / pi,
           "upd": prof.info["upd_ms"] / pi}
    ab = algorithmic_bytes(h, p, dtype, fmt, precond > 0)
    dom = max(("fwd", "adj"), key=lambda k: kms[k])
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    peak = peaks.get("hbm_gbs", 6400.0)
    achieved = ab[dom] / (kms[dom] * 1e-3) / 1e9
    kernel_name = {"fwd": "k_fwd", "adj": "k_adj"}[dom]
    out["roofline"] = {"bound": "hbm", "kernel": kernel_name, "achieved": round(achieved, 1),
                       "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                       "traffic": dram_traffic_record(kernel_name, args.form, args.workload),
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"
                       if "hbm_gbs" in peaks else "fallback 6400 GB/s",
                       "algorithmic_bytes_per_launch": ab[dom],
                       "avg_launch_ms": round(kms[dom], 5)}
    spmv_gbs = {k: round(ab[k] / (kms[k] * 1e-3) / 1e9, 1) for k in ("fwd", "adj")}

    # end to end through the host entry point (pinned host d and m)
    e2e = None
    if not args.no_e2e:
        dh = torch.empty(h.m, dtype=torch.float64, pin_memory=True)
        dh.copy_(d.cpu())
        mh = torch.empty(h.n, dtype=torch.float64, pin_memory=True)
        dn, mn = dh.numpy(), mh.numpy()
        dt_, fm_, pc_ = FORMS[args.form]
        set_scaling(pc_)
        h.lsqr_host(dn, p.w, p.lam, itmax, p.tol, m_out=mn, dtype=dt_, fmt=fm_, precond=min(pc_, 1))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            set_scaling(pc_)
            h.lsqr_host(dn, p.w, p.lam, itmax, p.tol, m_out=mn, dtype=dt_, fmt=fm_,
                        precond=min(pc_, 1))
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * h.m,
               "d2h_bytes_per_step": 8 * h.n}

    out.update({
        "reference": {"form": PLAIN, "tol": args.ref_tol, "iters": ref.info["iters"],
                      "istop": ref.info["istop"]},
        "config": {"workload": workload_desc(p), "form": args.form,
                   "plain_form": PLAIN, "nnz": h.nnz,
                   "l2_policy": "inputs larger than L2 (G values+indices "
                                f"{(VALUE_BYTES[dtype] * 2 * h.nnz) / 1e9:.2f} GB > 126 MB)",
                   "step": "one LSQR solve to tol on device-resident G (graph replay)",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "iters": it_chosen,
        "istop": res.info["istop"],
        "model_error_vs_fp64_ref": relerr(m_chosen),
        "plain_fp64": {"s": ms_plain / 1e3, "iters": res_plain.info["iters"],
                       "model_error_vs_fp64_ref": relerr(m_plain)},
        "speedup_vs_plain_fp64": ms_plain / ms,
        "accuracy_matched": accuracy_matched,
        "lsmr": lsmr_sec,
        "damping_sweep": sweep_sec,
        "kernel_ms_per_iter": {k: round(v, 5) for k, v in kms.items()},
        "spmv_gbs": spmv_gbs,
        "build_G_s": build_s,
        "iters_per_s": it_chosen / (ms / 1e3),
    })

    h.close()
    if not args.no_batched:
        out["batched"] = batched_section(args.batched_systems)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, args.cpu_sample_iters, res_plain.info["iters"])
    if rank == 0:
        print(json.dumps(out))


def batched_section(nsys=64, steps=2):
    """The batched workload: nsys uneven systems (grids 24x24x8 .. 64x64x16),
    16 right-hand sides each sharing G (8 checkerboards at the system's
    lambda, the blob model at 8 damping values 1e-3..1), FP32 values, tol 1e-6,
    solved by pdst_lsqr_batched.  Compared with one-at-a-time FP32 solves of the
    same pairs on a sample of systems, scaled by stored entries x pairs."""
    import numpy as np
    import torch

    from paper_2604_11920_b300 import pdst, synth
    ps = synth.batched(nsys)
    hs, ds, lams = [], [], []
    for p in ps:
        h = pdst.build_G_problem(p, dtypes=("f32",), formats=("blocked",))
        cols = []
        for j, (model, lam) in enumerate(synth.batched_rhs_models(p)):
            gm = torch.empty(h.m, dtype=torch.float64, device="cuda")
            h.apply_G(torch.from_numpy(model).cuda(), gm, dtype="f32")
            rms = torch.sqrt(torch.mean(gm * gm))
            z = torch.from_numpy(synth.rhs_noise(p.seed, p.m_rows, j)).cuda()
            cols.append(gm + p.noise_frac * rms * z)
        ds.append(torch.stack(cols, dim=1).contiguous())
        lams.append([lam for _, lam in synth.batched_rhs_models(p)])
        hs.append(h)
    w = [p.w for p in ps]
    nnz = [h.nnz for h in hs]
    outs, infos, opts = pdst.lsqr_batched(hs, ds, w, lams, 2000, 1e-6, dtype="f32")  # + tune
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        outs, infos, opts2 = pdst.lsqr_batched(hs, ds, w, lams, 2000, 1e-6, dtype="f32")
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / steps
    iters = [inf["iters"] for row in infos for inf in row]
    conv = sum(inf["istop"] in (1, 2) for row in infos for inf in row)
    # one-at-a-time reference on a sample of systems (largest, median, smallest)
    order = np.argsort(nnz)
    sample = sorted({int(order[-1]), int(order[len(order) // 2]), int(order[0])})
    t_single, work_single = 0.0, 0
    for s in sample:
        for j in range(ds[s].shape[1]):
            dj = ds[s][:, j].contiguous()
            hs[s].lsqr(dj, w[s], lams[s][j], 2000, 1e-6, dtype="f32", fmt="blocked")
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            hs[s].lsqr(dj, w[s], lams[s][j], 2000, 1e-6, dtype="f32", fmt="blocked")
            torch.cuda.synchronize()
            t_single += time.perf_counter() - t1
        work_single += nnz[s] * ds[s].shape[1]
    total_work = sum(n * d.shape[1] for n, d in zip(nnz, ds))
    t_seq_est = t_single * total_work / work_single
    for h in hs:
        h.close()
    return {"workload": f"{nsys} systems (grids 24x24x8..64x64x16), 16 right-hand sides each, "
                        "FP32 values, tol 1e-6",
            "total_nnz": int(sum(nnz)), "pairs": len(iters), "converged_pairs": conv,
            "batch_s": t_batch, "solves_per_s": len(iters) / t_batch,
            "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
            "chosen_tile_rows": opts["chosen_tile_rows"], "autotune_fwd_ms": opts["tune_ms"][:3],
            "gpu_launches": opts2["kernel_launches"],
            "one_at_a_time_estimate_s": t_seq_est,
            "speedup_vs_one_at_a_time": t_seq_est / t_batch,
            "one_at_a_time_sample": f"systems {sample} ({sum(ds[s].shape[1] for s in sample)} "
                                    "single solves), scaled by stored entries x right-hand sides"}


def cpu_baseline(p, sample_iters, iters_to_tol):
    """FP64 CPU oracle on this machine's cores: a bounded sample of LSQR
    iterations on the same system, scaled to the FP64 iteration count."""
    import oracle
    oracle.build()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    t0 = time.perf_counter()
    r = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=0.0, btol=0.0, conlim=0.0,
                    itmax=sample_iters)
    t = time.perf_counter() - t0
    per_it = t / max(r.itn, 1)
    return {"value": per_it * iters_to_tol, "unit": "s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{r.itn} FP64 oracle LSQR iterations on the same system in {t:.2f} s, "
                      f"scaled to the {iters_to_tol} iterations the FP64 solve needs to reach tol",
            "s_per_iter": per_it}


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = make_problem(args.workload, 0)
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    grid = (p.nx, p.ny, p.nz)
    # iteration count to tolerance of the oracle itself (untimed, once)
    full = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=p.tol, btol=p.tol, itmax=p.itmax)
    sample = args.cpu_sample_iters
    for _ in range(args.warmup):
        oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0.0, btol=0.0, conlim=0.0, itmax=3)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0.0, btol=0.0, conlim=0.0, itmax=sample)
        times.append((time.perf_counter() - t0) / r.itn)
    per_it = statistics.mean(times)
    value = per_it * full.itn
    cb = {"value": value, "unit": "s", "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"{sample} FP64 oracle LSQR iterations per step, scaled to the oracle's "
                    f"own {full.itn} iterations to tol"}
    print(json.dumps({"metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": per_it * sample * 1e3, "higher_is_better": False,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic (seeded generator; no dataset)",
                      "config": {"workload": workload_desc(p), "form": "oracle-f64"},
                      "impl": "reference", "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "pdst":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.ncu_case:
            run_ncu_case(args)
        elif args.only_batched:
            import torch
            torch.cuda.set_device(0)
            print(json.dumps(batched_section(args.batched_systems, steps=args.steps)))
        else:
            run_pdst(args, rank, world)
    finally:
        if world > 1 and args.impl == "pdst":
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
