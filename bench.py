#!/usr/bin/env python
"""Benchmark: PAGD time steps per second on the FCH 256^2 workload.

Workload (the configuration the headline metric is quoted on): FCH 2D,
256 x 256 Fourier collocation on [0, 4 pi]^2, W(u) = (u^2 - 1)^2 / 4, eps = 0.1,
eta1 = eta2 = eps, u0 = -0.3 + 0.05 U(-1, 1), fully implicit BDF2 solved by PAGD
with the averaged Newton preconditioner, FP32 iterations with FP64 base, norms
and acceptance, dt = 1e-3, residual tolerance ||d||_inf <= 1e-8.  The linear
IMEX scheme LBDF2 is timed beside it.

One "step" is one time step: the whole hot path (guess, preconditioner
constants, PAGD iterations to the tolerance, FP64 acceptance check).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: replicas only (independent instances, no collective on the data
path); value = all ranks' steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2204_07247_gb300 import inputs as I  # noqa: E402
from paper_2204_07247_gb300 import replicas as R  # noqa: E402

METRIC = "time steps/s at residual<=1e-8"
UNIT = "steps/s"
# algorithmic HBM bytes per grid point per PAGD residual evaluation of the
# fused passes (FP32-mixed: PFC 52, FCH 75; FP64 doubles them)
BYTES_PER_POINT_EVAL = {("pfc", "fp32_mixed"): 52, ("fch", "fp32_mixed"): 75,
                        ("pfc", "fp64"): 104, ("fch", "fp64"): 150}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# algorithmic HBM bytes per grid point per PAGD residual evaluation of the
# iteration passes as laid out here (PFC, FP32-mixed): row pass 24.1 B (read the
# direction's half spectrum, delta_i, delta_{i-1}, the FP32 base; write delta,
# the nonlinear term's half spectrum) + column pass 24.2 B (read it, the two
# spectral states and C0; write a state and the direction's half spectrum); 3D
# adds the middle passes (read + write one half spectrum each way, 16.1 B)
ITER_BYTES_2D_PFC = 48.3
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per time step of
# the dominant kernel, from one ncu capture of a short launch of the same
# kernel build on the same workload; the roofline's traffic is this times the
# steps of one timed launch (the per-step traffic is flat once the working set
# is resident).  Workloads without a capture report null.
TRAFFIC_PER_STEP = {"fch2d_256_bdf2_fp32mixed": 5.07e6}
# per batch step (all members).  The 3D figure is the capture of one 128^3
# member (2 steps) scaled by points to 256^3, for two members: a lower bound,
# as part of the 128^3 working set stays in L2
BATCH_TRAFFIC_PER_STEP = {"pfc2d_batch96_128_256_512_mp_fp32mixed": 10.42e9,
                          "pfc3d_256_bdf2_fp32mixed_x2": 2 * 8 * 0.9835e9}
ITER_BYTES_3D_PFC = 64.4


def flush_l2(torch):
    buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    buf.fill_(1.0)  # larger than the 129 MB L2
    del buf


def bench_batch(torch, pagd, bw, steps, warm, plain_steps, bytes_per_eval, peak, rank=0, world=1, dist=None):
    """One batched launch per chunk over all members of bw (the batched form),
    and each member alone through the single-instance kernel (the plain form).
    With N ranks each advances a disjoint shard of the members (strong scaling)."""
    members = R.shard(bw.members, rank, world)
    if not members:  # more ranks than members: this rank only joins the collectives
        R.max_over_ranks(0.0, dist, "cuda")
        R.sum_over_ranks(0.0, dist, "cuda")
        R.max_over_ranks(0.0, dist, "cuda")
        return None
    sol, u0s = [], []
    for w in members:
        S = pagd.solver_for(w)
        u0s.append(torch.from_numpy(w.u0(w.seeds[0])).cuda())
        S.set_state(u0s[-1])
        sol.append(S)
    B = pagd.Batch(sol)
    # the launch shape chosen by timing (before, and outside, the timed region)
    from paper_2204_07247_gb300 import autotune
    schedule = autotune.tune_batch(torch, B, u0s, bw.dt, bw.tol, steps=2)
    del u0s
    B.run(bw.dt, warm, bw.tol)
    flush_l2(torch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    its, res, status = B.run(bw.dt, steps, bw.tol)
    e1.record()
    torch.cuda.synchronize()
    ms = R.max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    launch = B.launch_info()
    npts = np.array([int(np.prod(w.n)) for w in members], dtype=np.float64)
    evals = its.sum(axis=1).astype(np.float64)
    nbytes = R.sum_over_ranks(float((evals * npts).sum()) * bytes_per_eval, dist, "cuda")
    achieved = nbytes / (ms / 1000.0) / 1e9 / world  # per GPU
    # plain form: the same members one at a time, a bounded number of steps each
    plain_ms = 0.0
    for w in members:
        S = pagd.solver_for(w)
        S.set_state(torch.from_numpy(w.u0(w.seeds[0])).cuda())
        S.run(w.dt, warm, w.tol)
        torch.cuda.synchronize()
        e0.record()
        S.run(w.dt, plain_steps, w.tol)
        e1.record()
        torch.cuda.synchronize()
        plain_ms += e0.elapsed_time(e1)
    plain_ms = R.max_over_ranks(plain_ms, dist, "cuda")
    m = len(bw.members)
    return {
        "workload": bw.name, "members": m, "steps": steps, "ms": ms,
        "member_steps_per_s": m * steps / (ms / 1000.0), "batch_steps_per_s": steps / (ms / 1000.0),
        "iters_per_step": float(its.mean()), "max_iters": int(its.max()), "max_resid": float(res.max()),
        "all_ok": bool(np.all(status == 0)),
        "gpu_launches": (len(members) if launch["sequential"] else 1) * math.ceil(steps / 4096),
        "scaling": "strong" if world > 1 else "weak",
        "schedule": schedule,
        "launch": {**launch, "strategy": "member after member through the single-instance kernel (every member "
                                         "alone fills every warp of the launch)" if launch["sequential"]
                   else "one batched launch per chunk"},
        "plain_member_steps_per_s": m * plain_steps / (plain_ms / 1000.0),
        "plain_sample": f"each member alone, {plain_steps} steps after {warm} warm-up steps",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     # DRAM bytes per launch: one member's steps when the members run one after
                     # the other, else every member's
                     "traffic": (BATCH_TRAFFIC_PER_STEP[bw.name] * steps / math.ceil(steps / 4096)
                                 / (len(bw.members) if launch["sequential"] else 1)
                                 if bw.name in BATCH_TRAFFIC_PER_STEP else None),
                     "kernel": "pagd_kernel<float>" if launch["sequential"] else "pagd_batch_kernel<float>",
                     "bytes_model": f"{bytes_per_eval} B per point per residual evaluation of the "
                                    f"iteration passes x sum over members of points x evaluations "
                                    f"({nbytes / 1e9:.1f} GB); base evaluations not counted"},
    }


def timed_run(torch, S, dt, steps, tol):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    its, res = S.run(dt, steps, tol)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), its


def bench_pgd_vs_pagd(torch, pagd, w, steps):
    """Table 2 analogue on the workload: the same kernels with sweeping friction
    (PAGD, Algorithm 2) and with lambda = 0 (PGD, Algorithm 1), from the same
    state after the same warm-up; transform pairs per step = evaluations x real
    fields per pass (PFC 1, FCH 2)."""
    pairs = 1 if w.model == "pfc" else 2
    out = {"workload": w.name, "steps": steps}
    for name, accel in (("pagd", 1), ("pgd", 0)):
        S = pagd.solver_for(w, accel=accel, max_iter=5000)
        S.set_state(torch.from_numpy(w.u0(1)).cuda())
        S.run(w.dt, 3, w.tol)
        ms, its = timed_run(torch, S, w.dt, steps, w.tol)
        out[name] = {"steps_per_s": steps / (ms / 1000.0), "iters_per_step": float(np.mean(its)),
                     "fft_pairs_per_step": pairs * float(np.mean(its))}
    out["iteration_ratio_pgd_over_pagd"] = out["pgd"]["iters_per_step"] / out["pagd"]["iters_per_step"]
    return out


def bench_cost_to_accuracy(torch, pagd, w, T_end, dts, ref_refine=8):
    """Table 4 analogue: fully implicit (PAGD) and linear IMEX schemes at equal
    final time T_end, error in the relative L2 norm against a reference run of
    the implicit scheme at dt_min / ref_refine, and the device time of each run."""
    def run(scheme, dt, precision):
        S = pagd.solver_for(w, scheme=scheme, precision=precision)
        S.set_state(torch.from_numpy(w.u0(1)).cuda())
        n = int(round(T_end / dt))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        S.run(dt, n, w.tol if scheme in ("bdf2", "mp") else 0.0, out)
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    imp, imex = w.scheme, {"bdf2": "lbdf2", "mp": "lmp"}[w.scheme]
    ref, _ = run(imp, min(dts) / ref_refine, "fp64")
    rn = float(torch.linalg.norm(ref))
    rows = []
    for dt in dts:
        for scheme, prec in ((imp, w.precision), (imex, "fp64")):
            u, ms = run(scheme, dt, prec)
            rows.append({"scheme": scheme, "precision": prec, "dt": dt, "ms": ms,
                         "rel_l2_error": float(torch.linalg.norm(u - ref)) / rn})
    return {"workload": w.name, "T": T_end, "reference": f"{imp} fp64 at dt {min(dts) / ref_refine:g}",
            "runs": rows}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_steps_per_s(w, budget_s=15.0, max_steps=20, warm=0, threads=1, final=None):
    """The FP64 CPU oracle as it stands on a bounded sample of the workload:
    `warm` untimed steps, then up to max_steps timed steps of the same
    trajectory (fewer once budget_s is spent); `threads` host threads share
    its line transforms.  final (a dict, optional) receives the oracle's last
    state and its step count from u0."""
    from oracle import oracle as O
    O.set_threads(threads)
    P = O.Problem(O.PFC if w.model == "pfc" else O.FCH, w.n, w.L, w.eps, w.eta1, w.eta2, w.tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2, "lmp": O.LMP}[w.scheme],
                  s=w.s, eta=w.eta, max_iter=w.max_iter)
    un = w.u0(1)
    unm1 = un.copy()
    for k in range(warm):
        r = O.pagd_step(P, k, un, unm1, w.dt, w.dt, w.tol)
        unm1, un = un, r.u
    t0 = time.perf_counter()
    nst = 0
    its = []
    while nst < max_steps:
        r = O.pagd_step(P, warm + nst, un, unm1, w.dt, w.dt, w.tol)
        its.append(r.iters)
        unm1, un = un, r.u
        nst += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    if final is not None:
        final["u"], final["steps"] = un, warm + nst
    return nst / dt, nst, float(np.mean(its)), dt


def gpu_rel_l2_vs_oracle(torch, pagd, w, u_oracle, nsteps, seed=1):
    """|u_gpu - u_oracle|_2 / |u_oracle|_2 after nsteps steps from u0 (full
    fields: the oracle state comes from the CPU-baseline run)."""
    S = pagd.solver_for(w)
    S.set_state(torch.from_numpy(w.u0(seed)).cuda())
    out = S.empty_field()
    S.run(w.dt, nsteps, w.tol, out)
    u = out.cpu().numpy()
    return float(np.linalg.norm(u - u_oracle) / np.linalg.norm(u_oracle))


def reference_fixture(name):
    p = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        return json.load(fh)


def gpu_vs_reference(torch, pagd, w):
    """The plain GPU trajectory from u0 against the oracle's stored reference
    trajectory (tests/golden, written by oracle/reference_runs.py): relative L2
    error at each checkpoint from the two sketches, with the oracle's own
    tolerance floor and twin-run amplification beside it."""
    rec = reference_fixture(w.name)
    if rec is None:
        return None
    S = pagd.solver_for(w)
    S.set_state(torch.from_numpy(w.u0(rec["seed"])).cuda())
    out = S.empty_field()
    done, rows = 0, {}
    for step in sorted(int(k) for k in rec["states"]):
        S.run(w.dt, step - done, w.tol, out)
        done = step
        ref = rec["states"][str(step)]
        est = I.sketch_rel_l2(I.sketch(out.cpu().numpy(), rec["sketch"]["count"], rec["sketch"]["seed"]),
                              ref["sketch"], ref["sumsq"])
        rows[str(step)] = {"rel_l2_est": est,
                           "oracle_tol_floor": rec.get("tol_floor", {}).get("rel_l2", {}).get(str(step)),
                           "twin_amplification": rec.get("twin", {}).get("amplification", {}).get(str(step))}
    return {"reference": f"tests/golden/oracle_{w.name}.json (FP64 oracle, seed {rec['seed']})",
            "estimator": f"{rec['sketch']['count']}-projection sketch", "checkpoints": rows}


def batch_vs_reference(torch, pagd, names):
    """Members with a stored oracle reference trajectory (tests/golden), run
    together as one batch from u0 through the reference's checkpoints: the
    relative L2 error at each (sketch estimate) beside the oracle's own
    tolerance floor."""
    recs = [reference_fixture(n) for n in names]
    recs = [r for r in recs if r is not None]
    if not recs:
        return None
    ws = [I.Workload(r["workload"], r["model"], tuple(r["n"]), tuple(r["L"]), r["eps"], r["eta1"], r["eta2"],
                     r["tau"], r["M"], r["scheme"], "fp32_mixed", r["dt"], 0, r["tol"], r["mean"], r["amp"],
                     (r["seed"],), r["s"], tuple(r["eta"])) for r in recs]
    sols = []
    for r, w in zip(recs, ws):
        S = pagd.solver_for(w)
        S.set_state(torch.from_numpy(w.u0(r["seed"])).cuda())
        sols.append(S)
    B = pagd.Batch(sols) if len(sols) > 1 else None
    out = {r["workload"]: {} for r in recs}
    done = 0
    for step in sorted({int(k) for r in recs for k in r["states"]}):
        if B is not None:
            B.run(ws[0].dt, step - done, ws[0].tol)
        else:
            sols[0].run(ws[0].dt, step - done, ws[0].tol)
        done = step
        for r, S in zip(recs, sols):
            if str(step) not in r["states"]:
                continue
            ref = r["states"][str(step)]
            u = S.get_state()[0].cpu().numpy()
            out[r["workload"]][str(step)] = {
                "rel_l2_est": I.sketch_rel_l2(I.sketch(u, r["sketch"]["count"], r["sketch"]["seed"]), ref["sketch"],
                                              ref["sumsq"]),
                "oracle_tol_floor": r.get("tol_floor", {}).get("rel_l2", {}).get(str(step))}
    return {"reference": "tests/golden (FP64 oracle)", "form": "batched" if B is not None else "plain",
            "members": out}


def bench_pfc64(torch, pagd, warm, cores, cpu=True):
    """PFC 2D 64^2 MP FP64 (100 steps): GPU steps/s, its error against the
    oracle over the whole run, and the oracle timed in full on the host."""
    w = I.PFC64
    S = pagd.solver_for(w)
    S.set_state(torch.from_numpy(w.u0(1)).cuda())
    S.run(w.dt, warm, w.tol)
    S.set_state(torch.from_numpy(w.u0(1)).cuda())
    flush_l2(torch)
    out = S.empty_field()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    its, res = S.run(w.dt, w.steps, w.tol, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    row = {"workload": w.name, "steps": w.steps, "ms": ms, "steps_per_s": w.steps / (ms / 1000.0),
           "iters_per_step": float(np.mean(its)), "max_resid": float(np.max(res)), "gpu_launches": 1,
           "roofline": {"bound": "latency", "note": "64^2 FP64: 4096 points per phase, far below the "
                        "machine's parallelism; bound by the device barriers and the per-unit latency"}}
    if cpu:
        from oracle import oracle as O
        fin = {}
        v1, n1, oits, sec1 = oracle_steps_per_s(w, budget_s=60.0, max_steps=w.steps, threads=1, final=fin)
        row["cpu_baseline"] = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"the whole run ({n1} steps, {sec1:.1f} s), FP64 C oracle, 1 thread"}
        row["oracle_iters_per_step"] = oits
        if fin["steps"] == w.steps:
            u = out.cpu().numpy()
            row["rel_l2_vs_oracle"] = float(np.linalg.norm(u - fin["u"]) / np.linalg.norm(fin["u"]))
        O.set_threads(cores)
        vN, nN, _, secN = oracle_steps_per_s(w, budget_s=30.0, max_steps=w.steps, threads=cores)
        row["cpu_baseline"]["all_cores_value"] = vN
        row["cpu_baseline"]["all_cores"] = cores
    row["vs_reference_trajectory"] = gpu_vs_reference(torch, pagd, w)
    return row


def _oracle_problem(w, n=None, L=None):
    from oracle import oracle as O
    return O.Problem(O.PFC if w.model == "pfc" else O.FCH, n or w.n, L or w.L, w.eps, w.eta1, w.eta2, w.tau,
                     scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2, "lmp": O.LMP}[w.scheme],
                     s=w.s, eta=w.eta, max_iter=w.max_iter)


def oracle_batch_baseline(bw, steps=2, threads=1):
    """The oracle on the batch's members, one of each grid size (the sizes are
    equal shares of the batch), `steps` steps each: member steps per second."""
    from oracle import oracle as O
    O.set_threads(threads)
    picked, seen = [], set()
    for m in bw.members:
        if m.n not in seen:
            seen.add(m.n)
            picked.append(m)
    tot, done = 0.0, 0
    for m in picked:
        P = _oracle_problem(m)
        un = m.u0(m.seeds[0])
        unm1 = un.copy()
        t0 = time.perf_counter()
        for k in range(steps):
            r = O.pagd_step(P, k, un, unm1, bw.dt, bw.dt, bw.tol)
            unm1, un = un, r.u
        tot += time.perf_counter() - t0
        done += steps
    return {"value": done / tot, "unit": "member steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} steps of one member of each size ({', '.join(str(m.n) for m in picked)}), "
                      f"{tot:.1f} s, FP64 C oracle, {threads} threads on its line transforms"}


def oracle_3d_measured(w, threads=1, steps=1):
    """The oracle on the full 3D workload, `steps` steps from u0 of the
    first seed, timed: member steps per second (a bounded sample; one 256^3
    step is tens of seconds on the host cores)."""
    from oracle import oracle as O
    O.set_threads(threads)
    P = _oracle_problem(w)
    un = w.u0(w.seeds[0])
    unm1 = un.copy()
    its = []
    t0 = time.perf_counter()
    for k in range(steps):
        r = O.pagd_step(P, k, un, unm1, w.dt, w.dt, w.tol)
        its.append(r.iters)
        unm1, un = un, r.u
    t = time.perf_counter() - t0
    return {"value": steps / t, "unit": "member steps/s", "cores": threads, "kind": "oracle",
            "sample": f"measured: the first {steps} step(s) of {w.n} from u0 ({its} PAGD evaluations, {t:.1f} s), "
                      f"FP64 C oracle, {threads} threads on its line transforms"}


def run_reference(args, w, rank):
    if rank != 0:
        return 0
    # a bounded sample: at most 3 warm-up and 10 timed oracle steps (~2.3 s
    # each at 256^2 on one host core), so the run ends within a minute or so
    K = max(1, min(args.steps, 10))
    W = max(0, min(args.warmup, 3))
    cores = host_cores()
    v, nst, its, secs = oracle_steps_per_s(w, budget_s=60.0, max_steps=K, warm=W, threads=cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": nst, "warmup": W, "ms_per_step": 1000.0 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "model": w.model, "grid": list(w.n), "scheme": w.scheme,
                   "dt": w.dt, "tol": w.tol, "oracle_iters_per_step": its},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"steps {W + 1}..{W + nst} of the workload after {W} untimed "
                                   f"warm-up steps, FP64 C oracle, {cores} threads on its line "
                                   f"transforms"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


FORMS = ("single", "batched", "pfc3d")


def form_solvers(torch, pagd, form, w, grid=None):
    """Solvers (state set) and a runner for one form: the single-instance
    workload w, the 96-member batch, or the two-seed 3D batch (grid: the 3D
    members at grid^3 with the same spacing, for a capture that must stay
    small)."""
    if form == "single":
        S = pagd.solver_for(w)
        S.set_state(torch.from_numpy(w.u0(1)).cuda())
        return [S], (lambda k: S.run(w.dt, k, w.tol)), w.dt
    if form == "batched":
        members = I.PFC_BATCH96.members
    else:
        w3 = I.PFC3D256
        if grid:
            w3 = dataclasses.replace(w3, n=(grid,) * 3, L=tuple(l * grid / n for l, n in zip(w3.L, w3.n)))
        members = [w3, dataclasses.replace(w3, seeds=(w3.seeds[1],))]
    sol = []
    for m in members:
        S = pagd.solver_for(m)
        S.set_state(torch.from_numpy(m.u0(m.seeds[0])).cuda())
        sol.append(S)
    B = pagd.Batch(sol)
    m0 = members[0]
    return sol, (lambda k: B.run(m0.dt, k, m0.tol)), m0.dt


def profile_form(torch, pagd, form, w, steps, warm, trace, grid=None):
    """One warm-up launch, then one launch of `steps` steps (the launch an ncu
    capture with -s 1 -c 1 takes); with trace, print its phase breakdown."""
    import collections
    sol, run, _ = form_solvers(torch, pagd, form, w, grid)
    run(warm)
    if trace:
        sol[0].set_trace(True)
    out = run(steps)
    torch.cuda.synchronize()
    if not trace:
        print("ok", flush=True)
        return 0
    batch = form != "single"
    masks, t = sol[0].get_trace(raw=True)
    its = out[0]
    agg = collections.defaultdict(lambda: [0, 0.0])
    for m, d in zip(masks[1:], np.diff(t)):
        name = ("+".join(pagd.PHASES[p] for p in range(32) if m >> p & 1) if batch
                else pagd.PHASES[m & 0xFFFF] + ("/inc" if m >> 16 & 1 else ""))
        agg[name][0] += 1
        agg[name][1] += d
    tot = t[-1]
    print(f"{form}: {steps} steps, {tot / steps:.1f} us/step, {(len(t) - 1) / steps:.1f} phases/step, "
          f"{float(np.mean(its)):.2f} evaluations/step")
    for k, (n, sec) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"  {k:24s} per step {n / steps:6.2f}  mean {sec / n:9.2f} us  share {100 * sec / tot:5.1f}%")
    return 0


# algorithmic HBM bytes per grid point of one FP32 iteration pass (PFC): the
# row and column passes as in ITER_BYTES_2D_PFC, each middle pass reading and
# writing one half spectrum
PASS_BYTES_PFC = {"RI": 24.1, "CI": 24.2, "MF": 8.05, "MI": 8.05}


def pass_rooflines(torch, pagd, w, peak, count=20, warm=3, lib=None):
    """Each FP32 iteration pass of the PFC FP32-mixed workload w on its own
    (pagd_pass_probe: `count` repetitions in one launch after `warm` steps,
    barrier included, CUDA events): device time, algorithmic bytes
    (PASS_BYTES_PFC x points) over that time, and the fraction of the
    measured HBM peak."""
    S = pagd.solver_for(w, lib=lib)
    S.set_state(torch.from_numpy(w.u0(w.seeds[0])).cuda())
    S.run(w.dt, warm, w.tol)
    npts = int(np.prod(w.n))
    out = {"workload": w.name, "count": count, "barrier_us": S.barrier_probe(count),
           "bytes_per_point": dict(PASS_BYTES_PFC), "unit": "GB/s", "peak": peak,
           "source": "pagd_pass_probe, one launch per pass, CUDA events"}
    for p in (("RI", "CI", "MF", "MI") if len(w.n) == 3 else ("RI", "CI")):
        us = S.pass_probe(p, count)
        achieved = PASS_BYTES_PFC[p] * npts / (us * 1e-6) / 1e9 if us > 0 else None
        out[p] = {"us": us, "achieved": achieved, "frac": achieved / peak if achieved else None}
    return out


def probe_pass(torch, pagd, w, which, count, warm, grid=None):
    """One iteration pass of w repeated `count` times in one launch (after a
    warm-up launch of `warm` steps): device time per pass with and without the
    barrier, and the pass's algorithmic bytes over that time."""
    if grid and len(w.n) == 3:
        w = dataclasses.replace(w, n=(grid,) * 3, L=tuple(l * grid / n for l, n in zip(w.L, w.n)))
    S = pagd.solver_for(w)
    S.set_state(torch.from_numpy(w.u0(w.seeds[0])).cuda())
    S.run(w.dt, warm, w.tol)
    us = S.pass_probe(which, count)
    bar = S.barrier_probe(count)
    npts = int(np.prod(w.n))
    out = {"workload": w.name, "grid": list(w.n), "pass": which, "count": count, "us_per_pass": us,
           "barrier_us": bar, "launch": S.launch_info()}
    if w.model == "pfc" and w.precision == "fp32_mixed":
        nbytes = PASS_BYTES_PFC[which] * npts
        out["bytes_per_pass"] = nbytes
        out["GBps_with_barrier"] = nbytes / (us * 1e-6) / 1e9
        out["GBps_without_barrier"] = nbytes / ((us - bar) * 1e-6) / 1e9
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=I.FCH256.name,
                    choices=sorted(I.WORKLOADS) + [m.name for m in I.PFC_BATCH96.members])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and 3D lines")
    ap.add_argument("--no-studies", action="store_true", help="skip the PGD and cost-to-accuracy studies")
    ap.add_argument("--profile", choices=FORMS, help="one warm-up launch and one launch of --steps steps of "
                    "a form, then exit (the launch for ncu -s 1 -c 1)")
    ap.add_argument("--trace", choices=FORMS, help="print the phase trace of --steps steps of a form")
    ap.add_argument("--profile-grid", type=int, default=None,
                    help="with --profile / --trace pfc3d / --probe-pass: 3D members at this grid^3, same spacing")
    ap.add_argument("--probe-pass", choices=("RI", "CI", "MF", "MI"),
                    help="time one iteration pass of --workload run on its own (--steps repetitions in one "
                         "launch, after --warmup steps; the launch for ncu -s 1 -c 1), then exit")
    args = ap.parse_args()
    w = I.WORKLOADS.get(args.workload) or {m.name: m for m in I.PFC_BATCH96.members}[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, w, rank)

    import torch
    from paper_2204_07247_gb300 import pagd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")

    W = max(3, args.warmup)
    K = max(1, args.steps)
    if args.profile or args.trace:
        return profile_form(torch, pagd, args.profile or args.trace, w, K, W, bool(args.trace), args.profile_grid)
    if args.probe_pass:
        return probe_pass(torch, pagd, w, args.probe_pass, K, W, args.profile_grid)
    S = pagd.solver_for(w)
    u0 = torch.from_numpy(w.u0(1 + rank)).cuda()
    S.set_state(u0)
    out = torch.empty_like(u0)
    S.run(w.dt, W, w.tol, out)  # warm-up steps (continue the same trajectory)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush.fill_(1.0)  # larger than the 129 MB L2: evicts what the warm-up left there
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    its, res = S.run(w.dt, K, w.tol, out)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    value = world * K / (ms / 1000.0)
    evals = int(np.sum(its))

    # end to end through the host-buffer entry point (copies inside the timed region)
    S2 = pagd.solver_for(w)
    u0h = torch.from_numpy(w.u0(1 + rank)).pin_memory().numpy()
    S2.run_host(u0h, w.dt, W, w.tol)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    uh, its2, _ = S2.run_host(u0h, w.dt, K, w.tol)
    t_e2e = time.perf_counter() - t0
    if dist:
        t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    n_pts = int(np.prod(w.n))
    e2e = {"value": world * K / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * n_pts / K, "d2h_bytes_per_step": (8 * n_pts + 16 * K + 64) / K}

    # the other schemes side by side (MP fully implicit, the IMEX LBDF2 / LMP),
    # same workload, device and step count
    side = {}
    for scheme, prec, tol in (("mp", w.precision, w.tol), ("lbdf2", "fp64", 0.0), ("lmp", "fp64", 0.0)):
        S3 = pagd.solver_for(w, scheme=scheme, precision=prec)
        S3.set_state(u0)
        S3.run(w.dt, W, tol)
        torch.cuda.synchronize()
        e0.record()
        its3, _ = S3.run(w.dt, K, tol)
        e1.record()
        torch.cuda.synchronize()
        side[scheme] = {"steps_per_s": K / (e0.elapsed_time(e1) / 1000.0),
                        "iters_per_step": float(np.mean(its3)), "precision": prec}
    imex_sps = side["lbdf2"]["steps_per_s"]

    # what binds the step: device barriers per step x the measured cost of one
    # (an empty phase of the same launch plan), from a short traced run
    S4 = pagd.solver_for(w)
    S4.set_state(u0)
    S4.run(w.dt, W, w.tol)
    S4.set_trace(True)
    its4, _ = S4.run(w.dt, 20, w.tol)
    names4, t4 = S4.get_trace()
    S4.set_trace(False)
    phases_per_step = (len(names4) - 1) / 20.0
    barrier_us = S4.barrier_probe(2000)

    # the batched form (PFC, 96 members of 128^2 / 256^2 / 512^2) and the 3D
    # workload (PFC 256^3, two seeds in one batch), each timed on its own
    peak, peak_kind = measured_peaks()
    extra = {}
    if not args.no_studies and rank == 0:
        extra["pgd_vs_pagd"] = bench_pgd_vs_pagd(torch, pagd, w, 100)
        extra["cost_to_accuracy"] = bench_cost_to_accuracy(torch, pagd, w, 0.064,
                                                           [4e-3, 2e-3, 1e-3, 5e-4])
    if not args.no_forms and rank == 0:
        extra["pfc64"] = bench_pfc64(torch, pagd, W, host_cores(), cpu=not args.no_cpu_baseline)
    if not args.no_forms and rank == 0:
        # learned initial iterate (FCH 512^2): train on solver trajectories, then
        # PAGD from the network's proposal vs from the extrapolation
        from paper_2204_07247_gb300 import learned
        extra["learned"] = learned.run_study(torch, I.FCH512, list(range(1000, 1016)), [2000, 2001], [0, 1, 2, 3],
                                             96, 16, 600, batched_seeds=list(range(4, 12)))
    if not args.no_forms:
        extra["batched"] = bench_batch(torch, pagd, I.PFC_BATCH96, I.PFC_BATCH96.steps, W, 20,
                                       ITER_BYTES_2D_PFC, peak, rank, world, dist)
        w3 = I.PFC3D256
        bw3 = I.BatchWorkload(w3.name + "_x2", [w3, dataclasses.replace(w3, seeds=(w3.seeds[1],))],
                              w3.dt, w3.steps, w3.tol)
        extra["pfc3d"] = bench_batch(torch, pagd, bw3, w3.steps, W, w3.steps, ITER_BYTES_3D_PFC, peak, rank,
                                     world, dist)
        if rank == 0:
            firsts = ["pfc2d_128_mp_fp32mixed_i0", "pfc2d_256_mp_fp32mixed_i32", "pfc2d_512_mp_fp32mixed_i64"]
            if extra["batched"]:
                extra["batched"]["vs_reference_trajectory"] = batch_vs_reference(torch, pagd, firsts)
            if extra["pfc3d"]:
                extra["pfc3d"]["vs_reference_trajectory"] = {
                    "at_64^3_same_spacing": batch_vs_reference(torch, pagd, ["pfc3d_64_bdf2_fp32mixed"]),
                    "at_256^3": batch_vs_reference(torch, pagd, [w3.name])}
                # each iteration pass alone, after the timed region: reported, never fatal to the line
                try:
                    extra["pfc3d"]["roofline"]["passes"] = pass_rooflines(torch, pagd, w3, peak)
                except Exception as e:  # pragma: no cover - reported in the JSON line
                    extra["pfc3d"]["roofline"]["passes"] = {"error": f"{type(e).__name__}: {e}"}
        if rank == 0 and not args.no_cpu_baseline:
            # secondary baselines: a failure here is reported, never fatal to the line
            for key, fn in (("batched", lambda: oracle_batch_baseline(I.PFC_BATCH96, 2, host_cores())),
                            ("pfc3d", lambda: oracle_3d_measured(w3, host_cores(), 1))):
                if extra[key]:
                    try:
                        extra[key]["cpu_baseline"] = fn()
                    except Exception as e:  # pragma: no cover - reported in the JSON line
                        extra[key]["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    bpp = BYTES_PER_POINT_EVAL[(w.model, w.precision)]
    launches = math.ceil(K / 4096)
    achieved = bpp * n_pts * evals / launches / ((ms / 1000.0) / launches) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": TRAFFIC_PER_STEP[w.name] * K / launches if w.name in TRAFFIC_PER_STEP else None,
            "peak_kind": peak_kind,
            "kernel": "pagd_kernel<float>",
            "bytes_model": f"{bpp} B per grid point per residual evaluation x {n_pts} points x "
                           f"{evals} evaluations",
            "frac_is": "a lower bound: the 256^2 working set stays in L2, HBM is not the binding resource",
            "binding": {"kind": "latency", "phases_per_step": phases_per_step,
                        "barrier_us": barrier_us,
                        "barrier_share": phases_per_step * barrier_us / (1000.0 * ms / K),
                        "phase_us_mean": 1000.0 * ms / K / phases_per_step,
                        "note": "every phase ends in a device-wide barrier; a phase's work is one "
                                "row pair or column per warp (128 / 129 units on 152 SMs), so its "
                                "time is the latency of one unit plus the barrier"}}
    cpu = None
    rel_short = None
    if not args.no_cpu_baseline:
        # all host cores on the oracle's line transforms, and one core beside it
        cores = host_cores()
        fin = {}
        v, nst, oits, secs = oracle_steps_per_s(w, budget_s=15.0, max_steps=20, threads=cores, final=fin)
        rel_short = {"steps": fin["steps"],
                     "rel_l2": gpu_rel_l2_vs_oracle(torch, pagd, w, fin["u"], fin["steps"])}
        v1, nst1, _, secs1 = oracle_steps_per_s(w, budget_s=8.0, max_steps=20, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {nst} steps of the same workload ({secs:.1f} s), FP64 C oracle, "
                         f"{cores} threads on its line transforms, {oits:.1f} PAGD iterations/step",
               "single_thread_value": v1,
               "single_thread_sample": f"first {nst1} steps ({secs1:.1f} s), 1 thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, "model": w.model, "grid": list(w.n),
                   "domain": [round(x, 6) for x in w.L], "scheme": w.scheme,
                   "precision": w.precision, "dt": w.dt, "tol": w.tol, "form": "plain",
                   "parallelism": f"replicas{world}", "l2": "flushed before the timed run; "
                   "the 256^2 working set (~6 MB) is L2-resident across steps by design",
                   "iters_per_step": evals / K, "max_resid": float(np.max(res)),
                   "imex_lbdf2_steps_per_s": imex_sps, "schemes_side_by_side": side},
        "rel_l2_vs_oracle": rel_short,
        "vs_reference_trajectory": gpu_vs_reference(torch, pagd, w),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": ck,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
