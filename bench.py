#!/usr/bin/env python
"""Benchmark: LSQR time-to-tolerance of the regularised traveltime solve.

Workload (default): the 64 x 64 x 16 system (65,536 unknowns; 120 stations,
7,140 pairs x 24 periods = 171,360 rows; Bezier rays; Gaussian-blob model,
2 % noise; w = 2, lambda = 0.05), synthetic inputs from the seeded generator.

One step = one solve of the chosen form (FP32 values and vectors, FP64
scalars, the per-cell depth-block preconditioner computed inside the step:
each cell's nz x nz block of the normal matrix, its Cholesky factor R_h and
the solve on [G P; w L P; lambda P], P_h = R_h^-1) to within 1e-4
relative model error of the FP64 oracle's converged solution (stored in
tests/golden by a script that calls only the oracle): the FP32 solve to tol
1e-6, then refinement sweeps with FP32 values on the FP64 residual, their
tolerance the loosest rung of a fixed ladder that reaches the target (found
once, untimed).  Every step runs in the library's kernels on device-resident
G, replayed from CUDA graphs.  The G assembly is timed separately.

Reported beside the headline: the plain FP64 GPU LSQR (FP64 values and
vectors, element CSR/CSC, no scaling) at the same target and its own
per-kernel roofline; column-norm and learned diagonal scalings and the FP64
form with depth blocks at the same target; both forms at
tol 1e-6 (one solve); LSMR; the damping sweep; the batched workload; compact
records of the paper-shaped and 100 x 100 x 20 systems; the per-kernel
roofline of the chosen form from CUDA events; the end-to-end time through
the host entry point; and the FP64 CPU oracle timed on this machine's cores
on a bounded sample, scaled to the iterations the oracle itself needs.

`--impl reference` times the FP64 CPU oracle alone (the comparison arm).
Multi-GPU (torchrun): every rank solves its own system (seed + 1000 rank);
no data moves between ranks ("replicas only").
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
    # name: (dtype, format, scaling); scaling 1 = column-norm, 2 = learned (both
    # right-diagonal: the library's precond 1), 3 = per-cell depth blocks (precond 2)
    "f64-element": ("f64", "element", 0),
    "f64-blocked": ("f64", "blocked", 0),
    "df64-blocked": ("df64", "blocked", 0),
    "f32-element": ("f32", "element", 0),
    "f32-blocked": ("f32", "blocked", 0),
    "f32-blocked-colnorm": ("f32", "blocked", 1),
    "bf16-blocked-colnorm": ("bf16", "blocked", 1),
    "f32-blocked-learned": ("f32", "blocked", 2),
    "f32-blocked-block": ("f32", "blocked", 3),
    "bf16-blocked-block": ("bf16", "blocked", 3),
    "f64-blocked-block": ("f64", "blocked", 3),
}
LIB_PRECOND = {0: 0, 1: 1, 2: 1, 3: 2}   # scaling code of FORMS -> pdst_lsqr_opts.precond
PLAIN = "f64-element"
MODEL_PATH = os.path.join(ROOT, "paper_2604_11920_b300", "precond_mlp.json")
# the chosen form: FP32 values with FP64 scalars and the per-cell depth-block
# preconditioner (column-norm and learned diagonal scalings are measured beside
# it on the same target)
DEFAULT_FORM = "f32-blocked-block"
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
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the compact paper-shaped and 100x100x20 sections of the "
                         "default (64x64x16) run")
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

def algorithmic_bytes(h, p, dtype, fmt, scaled, blocks=False):
    """Bytes each kernel must move once per launch: matrix arrays read once,
    vectors read/written once, gathered vectors counted once (L2-resident);
    with depth blocks the adjoint also reads every cell's nz x nz block once."""
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
    if blocks:
        adj += xb * H * nz * nz - 8 * n   # the blocks replace the diagonal scaling vector
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
    if precond == 3:
        h.set_block_precond(None, p.w, p.lam)
    elif precond:   # learned and column-norm scaling run the same kernels
        h.set_col_scaling(None, p.w, p.lam)
    r = h.lsqr(d, p.w, p.lam, 3, 0.0, dtype=dtype, fmt=fmt, precond=LIB_PRECOND[precond],
               use_graph=False)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.form, "iters": r.info["iters"], "nnz": h.nnz}))
    h.close()


def load_mref(workload, seed):
    """The FP64 oracle's converged solution of a workload, stored by a
    committed script that calls only the oracle (tests/golden/make_mref.py);
    None when there is none for this workload and seed."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_mref.npy")
    meta_path = path[:-4] + ".json"
    if not (os.path.exists(path) and os.path.exists(meta_path)):
        return None, None
    meta = json.load(open(meta_path))
    if meta.get("seed") != seed:
        return None, None
    return np.load(path), meta


class System:
    """One device-resident system of the benchmark with its right-hand side
    (synthesised on the device with the library's FP64 product) and the
    solve forms of FORMS."""

    def __init__(self, p, dtypes, formats=("element", "blocked"), params=None):
        import torch

        from paper_2604_11920_b300 import pdst
        self.p = p
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.h = pdst.build_G_problem(p, dtypes=tuple(sorted(set(dtypes))), formats=formats)
        torch.cuda.synchronize()
        self.build_s = time.perf_counter() - t0
        mt = torch.from_numpy(p.m_true).cuda()
        gm = torch.empty(self.h.m, dtype=torch.float64, device="cuda")
        self.h.apply_G(mt, gm, dtype="f64")
        rms = torch.sqrt(torch.mean(gm * gm))
        self.d = gm + p.noise_frac * rms * torch.from_numpy(p.noise).cuda()
        self.params = params

    def set_scaling(self, pc):
        if pc == 1:
            self.h.set_col_scaling_power(self.p.w, self.p.lam, 1.0)
        elif pc == 3:
            self.h.set_block_precond(None, self.p.w, self.p.lam)
        elif pc == 2:
            from paper_2604_11920_b300.train_precond import learned_scaling
            learned_scaling(self.h, self.p, self.params)   # features + MLP, inside the step

    def solve(self, form, tol=None, itmax=None, **kw):
        """One solve of `form`, its scaling computed first (part of the step)."""
        dt, fm, pc = FORMS[form]
        self.set_scaling(pc)
        return self.h.lsqr(self.d, self.p.w, self.p.lam, itmax or self.p.itmax,
                           self.p.tol if tol is None else tol, dtype=dt, fmt=fm,
                           precond=LIB_PRECOND[pc], **kw)

    def acc_kw(self, form, t):
        """Solve arguments of the accuracy-matched form at ladder rung t: the
        plain FP64 form solves to tol t; reduced-precision forms run two-phase
        (their solve to the workload's tol, then refinement sweeps with FP32
        values on the FP64 residual to tol t)."""
        dt = FORMS[form][0]
        if dt == "f64":
            return {"tol": t, "itmax": 200000}
        return {"itmax": 200000, "refine": 3, "refine_dtype": REFINE_DTYPE, "refine_tol": t}

    def close(self):
        self.h.close()


def event_time(stream, fn):
    """Device time of fn() on `stream` (CUDA events, synchronised on both sides)."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def stream_ceiling(nbytes, stream, reps=5):
    """Device time of one plain sequential read of `nbytes` (pdst_stream_read
    over a buffer of that size, L2 flushed before each read by writing 256 MB):
    the rate at which this GPU streams the sweep's value bytes with no gather
    and no dependent load, the context for the sweeps' own fraction of peak."""
    import torch

    from paper_2604_11920_b300 import pdst
    nbytes -= nbytes % 16
    buf = torch.rand(nbytes // 4, device="cuda", dtype=torch.float32)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    best = None
    for i in range(reps + 1):
        flush.fill_(float(i))
        t, _ = event_time(stream, lambda: pdst.stream_read(buf, stream))
        if i > 0:
            best = t if best is None else min(best, t)
    del buf, flush
    return {"what": "pdst_stream_read (16-byte streaming loads, 8 blocks per SM) over a "
                    f"buffer of the sweep's value bytes, L2 flushed, best of {reps}",
            "bytes": nbytes, "ms": best * 1e3, "gbs": nbytes / best / 1e9}


def relerr_to(m_ref):
    import torch

    def f(m):
        return float(torch.linalg.norm(m - m_ref) / torch.linalg.norm(m_ref))
    return f


def calibrate(S, form, relerr, stream):
    """Loosest rung of TOL_LADDER at which `form` reaches ACC_TARGET (one timed
    solve per rung); None if no rung does."""
    err = None
    for t in TOL_LADDER:
        s, r = event_time(stream, lambda: S.solve(form, **S.acc_kw(form, t)))
        err = relerr(r.m)
        if err <= ACC_TARGET:
            return {"tol": t, "s": s, "iters": r.info["iters"], "sweeps": r.info["sweeps"],
                    "model_error": err}
    return {"tol": None, "s": None, "model_error": err}


def kernel_roofline(S, form, peak, iters=64, mode=2):
    """Per-kernel device time over `iters` iterations and the HBM fraction of
    each sweep on its algorithmic bytes.  mode 2: the CUDA-graph replay the
    timed steps run, with event nodes around each kernel; mode 1: each kernel
    launched alone between two events (includes its launch latency)."""
    dt, fm, pc = FORMS[form]
    prof = S.solve(form, itmax=iters, tol=0.0, profile=mode, conlim=1e300)
    pi = max(prof.info["profiled_iters"], 1)
    kms = {"fwd": prof.info["fwd_ms"] / pi, "adj": prof.info["adj_ms"] / pi,
           "upd": prof.info["upd_ms"] / pi}
    ab = algorithmic_bytes(S.h, S.p, dt, fm, pc > 0, blocks=pc == 3)
    gbs = {k: ab[k] / (kms[k] * 1e-3) / 1e9 for k in ("fwd", "adj")}
    return {"kernel_ms_per_iter": {k: round(v, 5) for k, v in kms.items()},
            "gbs": {k: round(v, 1) for k, v in gbs.items()},
            "frac_of_hbm": {k: round(v / peak, 4) for k, v in gbs.items()},
            "bytes": ab, "iters_profiled": pi}


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

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = ("MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks
                else "fallback 6400 GB/s")

    p = make_problem(args.workload, rank)
    dtype, fmt, precond = FORMS[args.form]
    params = None
    if precond == 2 or os.path.exists(MODEL_PATH):
        from paper_2604_11920_b300.train_precond import load_params
        params = load_params(MODEL_PATH) if os.path.exists(MODEL_PATH) else None
    S = System(p, {"f64", "f32", "bf16", dtype}, params=params)
    h = S.h

    # ---- the reference solution: the oracle's, stored; else the GPU's FP64 solve
    m_ref_np, ref_meta = load_mref(args.workload, p.seed)
    if m_ref_np is not None:
        m_ref = torch.from_numpy(m_ref_np).cuda()
        ref_desc = {"source": "FP64 CPU oracle (stored, tests/golden)", "tol": ref_meta["atol"],
                    "iters": ref_meta["iters"], "istop": ref_meta["istop"]}
    else:
        ref = h.lsqr(S.d, p.w, p.lam, 200000, args.ref_tol, dtype="f64", fmt="element")
        m_ref = ref.m.clone()
        ref_desc = {"source": "GPU plain FP64 solve (no oracle solution stored for this "
                              "workload)", "tol": args.ref_tol, "iters": ref.info["iters"],
                    "istop": ref.info["istop"]}
    relerr = relerr_to(m_ref)

    # ---- headline: time to within ACC_TARGET of the reference, chosen form
    headline_acc = not args.no_accuracy
    cal = calibrate(S, args.form, relerr, stream) if headline_acc else None
    if cal is not None and cal["tol"] is not None:
        kw = S.acc_kw(args.form, cal["tol"])
        step_desc = (f"one solve to within {ACC_TARGET:g} relative model error of the "
                     f"reference: {dtype} solve to tol {p.tol:g}, then refinement sweeps with "
                     f"FP32 values on the FP64 residual to tol {cal['tol']:g} (loosest rung of "
                     "the tolerance ladder that reaches it); scaling computed inside the step")
        metric_kind = "time_to_1e-4"
    else:
        kw = {}
        step_desc = f"one LSQR solve to tol {p.tol:g} on device-resident G (graph replay)"
        metric_kind = f"time_to_tol_{p.tol:g}"

    def timed(form, steps, warmup, **skw):
        for _ in range(warmup):
            S.solve(form, **skw)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        e0.record(stream)
        for _ in range(steps):
            r = S.solve(form, **skw)
            launches += r.info["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
        return ms, r, launches

    with ClockSampler(dev, enabled=not args.no_clocks) as clk:
        ms, res, launches = timed(args.form, args.steps, args.warmup, **kw)
    clocks = clk.summary()
    if args.only_solve:
        if rank == 0:
            print(json.dumps({"form": args.form, "ms_per_solve": ms, "iters": res.info["iters"],
                              "istop": res.info["istop"], "model_error": relerr(res.m)}))
        return
    headline_err = relerr(res.m)
    out = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype, "data": "synthetic (seeded generator; no dataset)"}

    # ---- the plain FP64 form at the same accuracy, with its own roofline
    plain_roof = kernel_roofline(S, PLAIN, peak)
    chosen_roof = kernel_roofline(S, args.form, peak)
    chosen_isolated = kernel_roofline(S, args.form, peak, mode=1)
    accuracy = {"target_model_error": ACC_TARGET, "reference": ref_desc,
                "chosen": {"form": args.form, "s": ms / 1e3, "iters": res.info["iters"],
                           "sweeps": res.info["sweeps"], "model_error": headline_err,
                           "calibration": cal}}
    if headline_acc:
        pcal = calibrate(S, PLAIN, relerr, stream)
        if pcal["tol"] is not None:
            ms_p, res_p, _ = timed(PLAIN, 2, 0, **S.acc_kw(PLAIN, pcal["tol"]))
            accuracy["plain_fp64"] = {"form": PLAIN, "tol": pcal["tol"], "s": ms_p / 1e3,
                                      "iters": res_p.info["iters"],
                                      "model_error": relerr(res_p.m),
                                      "kernels": plain_roof}
            accuracy["speedup_vs_plain_fp64"] = ms_p / ms
        else:
            accuracy["plain_fp64"] = {"form": PLAIN, "tol": None, "calibration": pcal,
                                      "kernels": plain_roof}
        # the other forms at the same target, for comparison: the diagonal
        # scalings (column norms, learned), BF16 values for the first solve (the
        # refinement sweeps stay FP32) and the depth blocks in FP64 (one solve)
        for other in ("f32-blocked-block", "f64-blocked-block", "f32-blocked-colnorm",
                      "f32-blocked-learned", "bf16-blocked-colnorm"):
            if other == args.form or (other.endswith("learned") and params is None):
                continue
            oc = calibrate(S, other, relerr, stream)
            if oc["tol"] is not None:
                ms_o, res_o, _ = timed(other, 2, 0, **S.acc_kw(other, oc["tol"]))
                accuracy[other] = {"s": ms_o / 1e3, "tol": oc["tol"],
                                   "iters": res_o.info["iters"], "model_error": relerr(res_o.m)}
            else:
                accuracy[other] = {"s": None, "calibration": oc}

    # ---- time to the workload's tolerance (one solve), chosen and plain
    ms_c6, res_c6, _ = timed(args.form, max(1, min(args.steps, 3)), 1)
    ms_p6, res_p6, _ = timed(PLAIN, max(1, min(args.steps, 3)), 1)
    tol_sec = {"tol": p.tol,
               "chosen": {"s": ms_c6 / 1e3, "iters": res_c6.info["iters"],
                          "istop": res_c6.info["istop"], "model_error": relerr(res_c6.m)},
               "plain_fp64": {"s": ms_p6 / 1e3, "iters": res_p6.info["iters"],
                              "model_error": relerr(res_p6.m), "kernels": plain_roof},
               "speedup_vs_plain_fp64": ms_p6 / ms_c6}

    # ---- LSMR (the paper's solver) on the same sweeps: chosen form and plain FP64
    lsmr_sec = None
    if not args.no_lsmr:
        ms_l, res_l, _ = timed(args.form, max(1, min(args.steps, 3)), 1, method="lsmr")
        ms_lp, res_lp, _ = timed(PLAIN, 1, 1, method="lsmr")
        lsmr_sec = {"tol": p.tol,
                    "chosen": {"s": ms_l / 1e3, "iters": res_l.info["iters"],
                               "istop": res_l.info["istop"], "model_error": relerr(res_l.m)},
                    "plain_fp64": {"s": ms_lp / 1e3, "iters": res_lp.info["iters"],
                                   "model_error": relerr(res_lp.m), "kernels": plain_roof},
                    "speedup_vs_plain_fp64": ms_lp / ms_l}

    # ---- damping sweep: 8 damping values from one bidiagonalisation vs 8 solves
    sweep_sec = None
    if not args.no_sweep:
        lams = [float(10.0 ** (-3 + 3 * i / 7)) for i in range(8)]   # logspace(-3, 0, 8)
        t_sweep, sw = event_time(stream, lambda: h.lsqr_damping_sweep(
            S.d, p.w, lams, p.itmax, p.tol, dtype="f32", fmt="blocked"))
        t_sep, sep = event_time(stream, lambda: [
            h.lsqr(S.d, p.w, lm, p.itmax, p.tol, dtype="f32", fmt="blocked") for lm in lams])
        sweep_sec = {"lambdas": lams, "form": "f32-blocked (no scaling)",
                     "sweep_s": t_sweep, "separate_s": t_sep, "speedup": t_sep / t_sweep,
                     "iters": [r.info["iters"] for r in sw],
                     "identical_to_separate": all(
                         bool(torch.equal(a.m, b.m)) for a, b in zip(sw, sep))}

    # ---- roofline of the dominant sweep of the chosen form
    kms = chosen_roof["kernel_ms_per_iter"]
    dom = max(("fwd", "adj"), key=lambda k: kms[k])
    kernel_name = {"fwd": "k_fwd", "adj": "k_adj"}[dom]
    ab = chosen_roof["bytes"]
    achieved = ab[dom] / (kms[dom] * 1e-3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": kernel_name, "achieved": round(achieved, 1),
                       "timing": "CUDA event nodes around each kernel inside the graph replay "
                                 f"({chosen_roof['iters_profiled']} iterations)",
                       "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                       "traffic": dram_traffic_record(kernel_name, args.form, args.workload),
                       "peak_source": peak_src, "algorithmic_bytes_per_launch": ab[dom],
                       "avg_launch_ms": kms[dom], "other_sweep": {
                           "kernel": {"fwd": "k_adj", "adj": "k_fwd"}[dom],
                           "frac": chosen_roof["frac_of_hbm"]["adj" if dom == "fwd" else "fwd"]}}
    sc = stream_ceiling(VALUE_BYTES[dtype] * h.nnz, stream)
    sc["frac_of_peak"] = round(sc["gbs"] / peak, 4)
    sc["sweep_frac_of_ceiling"] = round(achieved / sc["gbs"], 4)
    out["roofline"]["stream_ceiling"] = sc

    # ---- end to end through the host entry point (pinned host d and m)
    e2e = None
    if not args.no_e2e:
        dh = torch.empty(h.m, dtype=torch.float64, pin_memory=True)
        dh.copy_(S.d.cpu())
        mh = torch.empty(h.n, dtype=torch.float64, pin_memory=True)
        dn, mn = dh.numpy(), mh.numpy()
        dt_, fm_, pc_ = FORMS[args.form]
        hkw = dict(kw)
        itmax_h = hkw.pop("itmax", p.itmax)
        tol_h = hkw.pop("tol", p.tol)

        def host_step():
            S.set_scaling(pc_)
            h.lsqr_host(dn, p.w, p.lam, itmax_h, tol_h, m_out=mn, dtype=dt_, fmt=fm_,
                        precond=LIB_PRECOND[pc_], **hkw)
        host_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * h.m,
               "d2h_bytes_per_step": 8 * h.n,
               "model_error": relerr(torch.from_numpy(mn.copy()).cuda())}

    out.update({
        "config": {"workload": workload_desc(p), "form": args.form, "metric_kind": metric_kind,
                   "plain_form": PLAIN, "nnz": h.nnz,
                   "l2_policy": "inputs larger than L2 (G values+indices "
                                f"{(VALUE_BYTES[dtype] * 2 * h.nnz) / 1e9:.2f} GB > 126 MB)",
                   "step": step_desc, "reference": ref_desc["source"],
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "iters": res.info["iters"],
        "istop": res.info["istop"],
        "model_error_vs_reference": headline_err,
        "accuracy_matched": accuracy,
        "time_to_tol": tol_sec,
        "lsmr": lsmr_sec,
        "damping_sweep": sweep_sec,
        "kernels": chosen_roof,
        "kernels_isolated_launches": {k: chosen_isolated[k] for k in
                                      ("kernel_ms_per_iter", "gbs", "frac_of_hbm")},
        "build_G_s": S.build_s,
        "iters_per_s": res.info["iters"] / (ms / 1e3),
    })
    S.close()
    if not args.no_batched:
        out["batched"] = batched_section(args.batched_systems)
    if not args.no_extra_workloads and args.workload == "mid":
        out["workloads"] = {w: workload_section(w, args.form, params, peak, stream)
                            for w in ("paper", "large")}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, args.workload, args.cpu_sample_iters, metric_kind)
    if rank == 0:
        print(json.dumps(out))


def workload_section(name, form, params, peak, stream, steps=2):
    """Compact record of another workload in the default run: one warm-up and
    `steps` timed solves to the workload's tol of the chosen form and of the
    plain FP64 form, the per-kernel roofline of both, and the model error
    against the oracle's stored solution where there is one (the
    paper-shaped system), else against a tight GPU solve (100 x 100 x 20: FP64
    values with depth blocks at tol 1e-10; its oracle checks, on sampled rows
    and true residual norms, are in the full-size tests).  Only the value
    copies the section uses are built."""
    import torch
    p = make_problem(name, 0)
    S = System(p, {"f64", "f32"}, params=params)
    m_ref_np, meta = load_mref(name, p.seed)

    def solve_t(f, **kw):
        times, r = [], None
        S.solve(f, **kw)
        for _ in range(steps):
            s, r = event_time(stream, lambda: S.solve(f, **kw))
            times.append(s)
        return statistics.mean(times), r

    s_c, r_c = solve_t(form)
    s_p, r_p = solve_t(PLAIN)
    if m_ref_np is not None:
        relerr = relerr_to(torch.from_numpy(m_ref_np).cuda())
        ref = {"source": "FP64 CPU oracle (stored, tests/golden)", "tol": meta["atol"]}
    else:
        # no oracle solution at this size: a tight GPU solve (FP64 values, depth
        # blocks, tol 1e-10), so that both forms' errors at the workload's tol mean
        # distance to the minimiser
        r_ref = S.solve("f64-blocked-block", tol=1e-10, itmax=200000)
        relerr = relerr_to(r_ref.m)
        ref = {"source": "GPU FP64 solve with depth blocks at tol 1e-10 (not the oracle)",
               "iters": r_ref.info["iters"], "istop": r_ref.info["istop"]}
    sec = {"workload": workload_desc(p), "nnz": S.h.nnz, "build_G_s": S.build_s,
           "reference": ref,
           "time_to_tol": {"tol": p.tol,
                           "chosen": {"form": form, "s": s_c, "iters": r_c.info["iters"],
                                      "model_error": relerr(r_c.m)},
                           "plain_fp64": {"s": s_p, "iters": r_p.info["iters"],
                                          "model_error": relerr(r_p.m)},
                           "speedup_vs_plain_fp64": s_p / s_c},
           "kernels": {"chosen": kernel_roofline(S, form, peak),
                       "plain_fp64": kernel_roofline(S, PLAIN, peak)}}
    for k in ("chosen", "plain_fp64"):
        sec["kernels"][k].pop("bytes", None)
    acc_forms = (("chosen", form), ("plain_fp64", PLAIN)) if m_ref_np is not None else \
        (("chosen", form),)   # the plain form's ladder would take minutes at this size
    acc = {}
    for key, f in acc_forms:
        c = calibrate(S, f, relerr, stream)
        if c["tol"] is not None:
            s, r = solve_t(f, **S.acc_kw(f, c["tol"]))
            acc[key] = {"s": s, "tol": c["tol"], "iters": r.info["iters"],
                        "model_error": relerr(r.m)}
        else:
            acc[key] = {"s": None, "calibration": c}
    if "plain_fp64" in acc and acc["chosen"]["s"] and acc["plain_fp64"]["s"]:
        acc["speedup_vs_plain_fp64"] = acc["plain_fp64"]["s"] / acc["chosen"]["s"]
    sec["accuracy_matched"] = acc
    S.close()
    return sec


def batched_section(nsys=64, steps=2, itmax=6000, sample_every=1):
    """The batched workload: nsys uneven systems (grids 24x24x8 .. 64x64x16),
    16 right-hand sides each sharing G (8 checkerboards at the system's
    lambda, the blob model at 8 damping values 1e-3..1), FP32 values, FP64
    scalars, the per-cell depth-block preconditioner of each system (built
    with the system's lambda; lambda_j P rows per pair), tol 1e-6, solved by
    pdst_lsqr_batched.  Compared with one-at-a-time solves of the same pairs
    in the same form (same blocks, same lambda_j rows), all 16 pairs of every
    `sample_every`-th system measured (by default every system, so every pair
    is measured and the scaling below is 1; a sparser sample is scaled to the
    batch by stored entries x iterations); and with the same batch under
    column-norm scaling (one timed call)."""
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
        h.set_col_scaling(None, p.w, p.lam)      # column norms with the system's lambda
        h.set_block_precond(None, p.w, p.lam)    # depth blocks with the system's lambda
        hs.append(h)
    w = [p.w for p in ps]
    nnz = [h.nnz for h in hs]
    # column-norm scaling: one autotuned call, then one timed call
    pdst.lsqr_batched(hs, ds, w, lams, itmax, 1e-6, dtype="f32", precond=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, infos_c, _ = pdst.lsqr_batched(hs, ds, w, lams, itmax, 1e-6, dtype="f32", precond=1)
    torch.cuda.synchronize()
    t_colnorm = time.perf_counter() - t0
    outs, infos, opts = pdst.lsqr_batched(hs, ds, w, lams, itmax, 1e-6, dtype="f32",
                                          precond=2)   # + autotune
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        outs, infos, opts2 = pdst.lsqr_batched(hs, ds, w, lams, itmax, 1e-6, dtype="f32",
                                               precond=2)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / steps
    iters = [inf["iters"] for row in infos for inf in row]
    conv = [inf["istop"] in (1, 2) for row in infos for inf in row]
    recipe_names = [f"checkerboard b={b}" for b in (2, 3, 4, 5, 6, 7, 8)] + ["-checkerboard b=8"]
    recipe_names += [f"blobs lambda={l:.3g}" for l in np.logspace(-3.0, 0.0, 8)]
    per_recipe = {nm: {"converged": int(sum(infos[s][j]["istop"] in (1, 2) for s in range(nsys))),
                       "iters_mean": float(np.mean([infos[s][j]["iters"] for s in range(nsys)]))}
                  for j, nm in enumerate(recipe_names)}
    # one-at-a-time solves of every pair of the sampled systems (by default all
    # of them), measured; one untimed solve per system first (graph capture)
    sample = list(range(0, nsys, sample_every))
    t_single, work_single, it_single = 0.0, 0, 0
    for s in sample:
        d0 = ds[s][:, 0].contiguous()
        hs[s].lsqr(d0, w[s], lams[s][0], itmax, 1e-6, dtype="f32", fmt="blocked", precond=2)
        for j in range(ds[s].shape[1]):
            dj = ds[s][:, j].contiguous()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r = hs[s].lsqr(dj, w[s], lams[s][j], itmax, 1e-6, dtype="f32", fmt="blocked",
                           precond=2)
            torch.cuda.synchronize()
            t_single += time.perf_counter() - t1
            work_single += nnz[s] * r.info["iters"]
            it_single += r.info["iters"]
    total_work = sum(nnz[s] * infos[s][j]["iters"] for s in range(nsys)
                     for j in range(ds[s].shape[1]))
    t_seq_est = t_single * total_work / work_single
    total_nnz_iters = total_work
    for h in hs:
        h.close()
    iters_c = [inf["iters"] for row in infos_c for inf in row]
    return {"workload": f"{nsys} systems (grids 24x24x8..64x64x16), 16 right-hand sides each, "
                        "FP32 values, FP64 scalars, per-cell depth-block preconditioner per "
                        f"system, tol 1e-6, itmax {itmax}",
            "total_nnz": int(sum(nnz)), "pairs": len(iters), "converged_pairs": int(sum(conv)),
            "per_recipe": per_recipe,
            "batch_s": t_batch, "solves_per_s": len(iters) / t_batch,
            "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
            "entries_x_iters_per_s": total_nnz_iters / t_batch,
            "chosen_tile_rows": opts["chosen_tile_rows"], "autotune_iter_ms": opts["tune_ms"][:3],
            "gpu_launches": opts2["kernel_launches"],
            "one_at_a_time": {"measured_s": t_single, "solves": len(sample) * 16,
                              "systems": sample, "iters": it_single,
                              "scaled_to_batch_s": t_seq_est,
                              "scaling": ("none: every pair measured" if len(sample) == nsys else
                                          "measured time x (batch stored entries x iterations) / "
                                          "(sample stored entries x iterations)")},
            "speedup_vs_one_at_a_time": t_seq_est / t_batch,
            "column_norm_scaling": {"batch_s": t_colnorm, "iters_mean": float(np.mean(iters_c)),
                                    "converged_pairs": int(sum(inf["istop"] in (1, 2)
                                                               for row in infos_c
                                                               for inf in row))}}


def oracle_iters_to_target(workload, seed):
    """Iterations the oracle itself needs to come within ACC_TARGET of its
    converged solution: the loosest rung of its stored ladder (one oracle run,
    tests/golden) that gets there, with that rung; (None, None) if unknown."""
    _, meta = load_mref(workload, seed)
    if not meta:
        return None, None
    for rung in meta.get("ladder", []):
        if rung["iters"] > 0 and rung["model_error"] <= ACC_TARGET:
            return rung["iters"], rung
    return None, None


def time_oracle_iters(p, sample_iters, repeats=1, warmup=0):
    """Seconds per FP64 oracle LSQR iteration on this machine's cores: the
    mean over `repeats` bounded samples of `sample_iters` iterations."""
    import oracle
    oracle.build()
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    grid = (p.nx, p.ny, p.nz)
    for _ in range(warmup):
        oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0.0, btol=0.0, conlim=0.0, itmax=3)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        r = oracle.lsqr(G, GT, grid, p.w, p.lam, d, atol=0.0, btol=0.0, conlim=0.0,
                        itmax=sample_iters)
        times.append((time.perf_counter() - t0) / max(r.itn, 1))
    return statistics.mean(times), oracle.num_threads(), (G, GT, d)


def oracle_value(p, workload, per_it, system, metric_kind):
    """The oracle's time on the benchmark's metric: seconds per iteration x the
    iterations the oracle needs (to within ACC_TARGET of its solution for the
    accuracy-matched metric, else to the workload's tol, found by one untimed
    oracle solve)."""
    if metric_kind == "time_to_1e-4":
        its, rung = oracle_iters_to_target(workload, p.seed)
        if its is not None:
            return per_it * its, (f"the {its} iterations the oracle needs to come within "
                                  f"{ACC_TARGET:g} of its converged solution (its stopping "
                                  f"rule at tol {rung['tol']:g}; stored ladder)")
    import oracle
    G, GT, d = system
    full = oracle.lsqr(G, GT, (p.nx, p.ny, p.nz), p.w, p.lam, d, atol=p.tol, btol=p.tol,
                       itmax=p.itmax)
    return per_it * full.itn, f"the oracle's own {full.itn} iterations to tol {p.tol:g}"


def cpu_baseline(p, workload, sample_iters, metric_kind):
    """FP64 CPU oracle on this machine's cores: a bounded sample of LSQR
    iterations on the same system, scaled to the iterations the oracle needs
    for the benchmark's metric."""
    per_it, cores, system = time_oracle_iters(p, sample_iters)
    value, what = oracle_value(p, workload, per_it, system, metric_kind)
    return {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"{sample_iters} FP64 oracle LSQR iterations on the same system "
                      f"({per_it * 1e3:.1f} ms each), scaled to {what}",
            "s_per_iter": per_it}


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, timed on the host cores, on the
    benchmark's metric: each step a bounded sample of oracle iterations,
    scaled to the iterations the oracle needs."""
    if rank != 0:
        return
    p = make_problem(args.workload, 0)
    metric_kind = ("time_to_1e-4" if not args.no_accuracy and
                   oracle_iters_to_target(args.workload, p.seed)[0] else
                   f"time_to_tol_{p.tol:g}")
    sample = args.cpu_sample_iters
    per_it, cores, system = time_oracle_iters(p, sample, repeats=args.steps,
                                              warmup=args.warmup)
    value, what = oracle_value(p, args.workload, per_it, system, metric_kind)
    cb = {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
          "sample": f"{sample} FP64 oracle LSQR iterations per step ({per_it * 1e3:.1f} ms "
                    f"each), scaled to {what}"}
    print(json.dumps({"metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": per_it * sample * 1e3, "higher_is_better": False,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic (seeded generator; no dataset)",
                      "config": {"workload": workload_desc(p), "form": "oracle-f64",
                                 "metric_kind": metric_kind},
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
