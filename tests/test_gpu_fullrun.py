"""Full-length GPU parity against the FP64 oracle's reference trajectories.

``oracle/reference_runs.py`` (oracle only) wrote, for every benchmark workload,
the oracle's state at a few checkpoint steps of the fixed-step trajectory from
u0 as a sketch: its projections onto seeded U(-1, 1) fields, its sum of squares,
mass and energy (``tests/golden/oracle_<workload>.json``).  These tests run
the CUDA path over the same steps from the same u0 (plain solver, and the
batched launch where the workload is batched) and estimate
|u_gpu - u_oracle|_2 / |u_oracle|_2 from the two sketches (128 projections:
the estimate is within about 25% of the true value with high probability, so
the bounds carry a factor 1.5).

Bounds (relative L2 on u): the configured targets, 1e-9 for FP64 and 1e-6 for
FP32-mixed, or, where larger, twice the fixture's tolerance floor: the
distance between two oracle trajectories that both meet the PAGD stopping rule
(tol and tol / 100).  Any solve that stops at the same tolerance but not at the
same iterate (FP32 iterations, another summation order) drifts from the oracle
by about that much; the floor is measured, not assumed, and the bound in use
is printed.  Mass: 1e-12 relative at every checkpoint."""
import glob
import json
import math
import os

import numpy as np
import pytest

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIXTURES = sorted(os.path.basename(p)[len("oracle_"):-len(".json")]
                  for p in glob.glob(os.path.join(GOLD, "oracle_*.json")))
SKETCH_MARGIN = 1.5


def load(name):
    with open(os.path.join(GOLD, f"oracle_{name}.json")) as f:
        return json.load(f)


def workload_of(rec, precision):
    return I.Workload(rec["workload"], rec["model"], tuple(rec["n"]), tuple(rec["L"]), rec["eps"], rec["eta1"],
                      rec["eta2"], rec["tau"], rec["M"], rec["scheme"], precision, rec["dt"], 0, rec["tol"],
                      rec["mean"], rec["amp"], (rec["seed"],), rec["s"], tuple(rec["eta"]))


def precision_of(name):
    return "fp64" if name.endswith("fp64") else "fp32_mixed"


def bound(rec, step, precision):
    target = 1e-9 if precision == "fp64" else 1e-6
    floor = rec.get("tol_floor", {}).get("rel_l2", {}).get(str(step), 0.0)
    return max(target, 2.0 * floor)


def check_state(rec, step, u, precision, errs):
    ref = rec["states"][str(step)]
    got = I.sketch(u, rec["sketch"]["count"], rec["sketch"]["seed"])
    err = I.sketch_rel_l2(got, ref["sketch"], ref["sumsq"])
    cellvol = float(np.prod([Li / ni for Li, ni in zip(rec["L"], rec["n"])]))
    mass = float(np.sum(u)) * cellvol
    b = bound(rec, step, precision)
    errs.append((step, err, b))
    assert abs(mass - ref["mass"]) <= 1e-12 * abs(ref["mass"]), (step, mass, ref["mass"])
    assert err <= SKETCH_MARGIN * b, f"step {step}: rel L2 {err:.3e} > {SKETCH_MARGIN} x {b:.3e} ({errs})"


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    t.cuda.set_device(0)
    return t


@pytest.mark.parametrize("name", FIXTURES)
def test_plain_trajectory_matches_oracle_reference(torch, name):
    rec = load(name)
    precision = precision_of(name)
    w = workload_of(rec, precision)
    S = pagd.solver_for(w)
    S.set_state(torch.from_numpy(w.u0(rec["seed"])).cuda())
    out = S.empty_field()
    done, errs = 0, []
    for step in sorted(int(k) for k in rec["states"]):
        its, res = S.run(w.dt, step - done, w.tol, out)
        assert all(res <= w.tol)
        done = step
        check_state(rec, step, out.cpu().numpy(), precision, errs)
    print(name, precision, [(s, f"{e:.2e}", f"{b:.1e}") for s, e, b in errs])


BATCHED = [n for n in FIXTURES if n.startswith("pfc2d_") and "_mp_fp32mixed_i" in n]


@pytest.mark.skipif(not BATCHED, reason="no batch-member fixtures")
def test_batched_members_match_oracle_reference(torch):
    """The first member of each grid size of the uneven PFC batch (128^2,
    256^2, 512^2) over its full 500 steps, advanced together in one batched
    launch per checkpoint interval."""
    recs = [load(n) for n in BATCHED]
    ws = [workload_of(r, "fp32_mixed") for r in recs]
    sols = []
    for r, w in zip(recs, ws):
        S = pagd.solver_for(w)
        S.set_state(torch.from_numpy(w.u0(r["seed"])).cuda())
        sols.append(S)
    B = pagd.Batch(sols)
    steps = sorted({int(k) for r in recs for k in r["states"]})
    done = 0
    errs = {r["workload"]: [] for r in recs}
    for step in steps:
        its, res, status = B.run(ws[0].dt, step - done, ws[0].tol)
        assert np.all(status == 0) and np.all(res <= ws[0].tol)
        done = step
        for r, S in zip(recs, sols):
            if str(step) in r["states"]:
                un, _, _ = S.get_state()
                check_state(r, step, un.cpu().numpy(), "fp32_mixed", errs[r["workload"]])
    print({k: [(s, f"{e:.2e}") for s, e, _ in v] for k, v in errs.items()})
