"""Reference states of the benchmark workloads from the FP64 CPU oracle, and the
conditioning study that says how closely any other arithmetic can follow them.

TEST INFRASTRUCTURE ONLY.  This script calls nothing but the oracle
(``oracle.py`` / ``pagd_oracle.c``) and the seeded input generators
(``paper_2204_07247_gb300/inputs.py``); it writes one small JSON text fixture
per workload to ``tests/golden/oracle_<workload>.json``, which the GPU parity
tests and the benchmark read.  No value in those files comes from the CUDA
library.

Per workload (model, grid, scheme, dt, tol and u0 as the workload defines them)
it records, at a few checkpoint steps of the fixed-step trajectory from
u0 (seed = the workload's first seed):
  * the sum of squares, mass h^d sum u and discrete energy E_N of u^n, and the
    projections of u^n onto inputs.SKETCH_COUNT seeded U(-1, 1) fields (so that
    a test can estimate |u_test - u^n|_2 / |u^n|_2 without the full field);
  * the PAGD iteration counts per step (Algorithm 2, the oracle's own counting);
  * twin run: the relative L2 distance between the trajectory and one started
    from u0 + 1e-7 |u0|_rms w (w a zero-mean seeded U(-1, 1) field), divided by
    the initial relative distance: the amplification of a perturbation of u0
    by the dynamics of the discrete scheme (Sec. 3.1.1);
  * tolerance floor: the relative L2 distance between the trajectory at the
    workload's PAGD tolerance and one at tol / 100: how far two solves that
    both meet the stopping rule of Algorithm 2 drift apart over the run.  Any
    implementation that stops at the same tolerance but not at the same iterate
    (another precision, another summation order) differs from the oracle by
    about this much.

Usage: python oracle/reference_runs.py [--only NAME ...] [--threads N] [--force]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2204_07247_gb300 import inputs as I  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")
TWIN_REL = 1e-7
TWIN_SEED = 0x7A1E0000


def problem(w: I.Workload) -> O.Problem:
    return O.Problem(O.PFC if w.model == "pfc" else O.FCH, tuple(w.n), tuple(w.L), w.eps, w.eta1, w.eta2, w.tau,
                     w.M, scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2, "lmp": O.LMP}[w.scheme],
                     s=w.s, eta=tuple(w.eta), max_iter=w.max_iter)


def trajectory(P: O.Problem, u0: np.ndarray, dt: float, tol: float, checkpoints):
    """Fixed-step run; returns {step: u^step} at the checkpoints and the
    per-step iteration counts."""
    want = set(checkpoints)
    last = max(checkpoints)
    un, unm1 = u0.copy(), u0.copy()
    out, iters = {}, []
    for n in range(last):
        if P.scheme in (O.BDF2, O.MP):
            r = O.pagd_step(P, n, un, unm1, dt, dt, tol)
            if r.status != O.OK:
                raise RuntimeError(f"oracle step {n} failed with status {r.status}")
            unew, it = r.u, r.iters
        else:
            unew, it = O.imex_step(P, n, un, unm1, dt, dt), 0
        unm1, un = un, unew
        iters.append(int(it))
        if n + 1 in want:
            out[n + 1] = un.copy()
    return out, iters


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def twin_field(u0: np.ndarray) -> np.ndarray:
    w = I.noisy_field(u0.shape, 0.0, 1.0, TWIN_SEED)
    w -= w.mean()  # same mass
    return u0 + TWIN_REL * math.sqrt(float(np.mean(u0 * u0))) * w


def run_workload(w: I.Workload, checkpoints, seed: int, twin: bool = True, floor: bool = True,
                 twin_checkpoints=None) -> dict:
    P = problem(w)
    u0 = w.u0(seed)
    t0 = time.time()
    states, iters = trajectory(P, u0, w.dt, w.tol, checkpoints)
    t_main = time.time() - t0
    rec = {
        "workload": w.name, "seed": seed, "model": w.model, "n": list(w.n), "L": list(w.L), "eps": w.eps,
        "eta1": w.eta1, "eta2": w.eta2, "tau": w.tau, "M": w.M, "scheme": w.scheme, "dt": w.dt, "tol": w.tol,
        "s": w.s, "eta": list(w.eta), "mean": w.mean, "amp": w.amp,
        "generated_by": "oracle/reference_runs.py (FP64 C oracle)",
        "sketch": {"seed": I.SKETCH_SEED, "count": I.SKETCH_COUNT},
        "oracle_seconds": t_main,
        "iters": iters,
        "states": {},
    }
    for n, u in sorted(states.items()):
        rec["states"][str(n)] = {
            "sumsq": float(np.sum(u * u)), "mass": O.mass(P, u), "energy": O.energy(P, u),
            "sketch": [float(x) for x in I.sketch(u)],
        }
    if twin:
        tc = twin_checkpoints or checkpoints
        u0t = twin_field(u0)
        if twin_checkpoints and set(twin_checkpoints) != set(checkpoints):
            states, _ = trajectory(P, u0, w.dt, w.tol, tc)
        tw, _ = trajectory(P, u0t, w.dt, w.tol, tc)
        d0 = rel_l2(u0t, u0)
        rec["twin"] = {"perturbation_rel_l2": d0,
                       "rel_l2": {str(n): rel_l2(tw[n], states[n]) for n in sorted(tw)},
                       "amplification": {str(n): rel_l2(tw[n], states[n]) / d0 for n in sorted(tw)}}
    if floor and P.scheme in (O.BDF2, O.MP):
        fl, _ = trajectory(P, u0, w.dt, w.tol * 1e-2, checkpoints)
        rec["tol_floor"] = {"tol_ref": w.tol * 1e-2,
                            "rel_l2": {str(n): rel_l2(states[n], fl[n]) for n in sorted(fl)}}
    return rec


def pfc3d_small(w: I.Workload, n: int) -> I.Workload:
    """The 3D workload at n^3 with the same spacing (for its conditioning)."""
    return dataclasses.replace(w, name=f"pfc3d_{n}_bdf2_fp32mixed", n=(n, n, n),
                               L=tuple(Li * n / ni for Li, ni in zip(w.L, w.n)))


def jobs():
    bw = I.PFC_BATCH96
    firsts, seen = [], set()
    for m in bw.members:
        if m.n not in seen:
            seen.add(m.n)
            firsts.append(m)
    J = [
        ("pfc2d_64_mp_fp64", lambda: run_workload(I.PFC64, [1, 10, 100], 1)),
        ("fch2d_256_bdf2_fp32mixed", lambda: run_workload(I.FCH256, [1, 10, 25, 100, 1000], 1)),
    ]
    for m in firsts:
        J.append((m.name, (lambda m=m: run_workload(m, [1, 10, 100, 500], m.seeds[0]))))
    w3 = pfc3d_small(I.PFC3D256, 64)
    J.append((w3.name, lambda: run_workload(w3, [1, 10, 200], 1, floor=True)))
    J.append((I.PFC3D256.name, lambda: run_workload(I.PFC3D256, [1, 2], 1, twin=False, floor=False)))
    return J


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    O.set_threads(a.threads)
    os.makedirs(GOLDEN, exist_ok=True)
    for name, fn in jobs():
        if a.only and name not in a.only:
            continue
        path = os.path.join(GOLDEN, f"oracle_{name}.json")
        if os.path.exists(path) and not a.force:
            print("exists:", path, flush=True)
            continue
        t0 = time.time()
        rec = fn()
        rec["threads"] = a.threads
        with open(path + ".tmp", "w") as f:
            json.dump(rec, f, indent=1)
        os.replace(path + ".tmp", path)
        print(f"{name}: {time.time() - t0:.0f} s -> {path}", flush=True)


if __name__ == "__main__":
    main()
