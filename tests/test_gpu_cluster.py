"""Cluster-resident PAGD iterations on the GPU (csrc/cluster.cuh): square
2D grids of 64^2, 128^2 and 256^2 run the iterations of each base point in
one thread-block cluster of n/16 CTAs (distributed shared memory, cluster
barriers).  Against the same solver with every phase device-wide
(PAGD_CLUSTER=0) and against the FP64 oracle: FP64 agrees to rounding with
the same iteration counts (within one), FP32-mixed within 1e-6 relative L2."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

pytestmark = pytest.mark.gpu

CASES = [
    ("fch", (256, 256), "bdf2", "fp32_mixed", 1e-3, -0.3, 1e-8, 3),
    ("fch", (128, 128), "mp", "fp32_mixed", 1e-3, -0.3, 1e-8, 4),
    ("pfc", (128, 128), "mp", "fp32_mixed", 0.1, 0.1, 1e-8, 4),
    ("pfc", (64, 64), "mp", "fp64", 0.1, 0.07, 1e-10, 6),
    ("fch", (64, 64), "bdf2", "fp64", 1e-3, -0.3, 1e-10, 4),
]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    t.cuda.set_device(0)
    return t


def _solver(case, cluster):
    model, n, scheme, prec = case[:4]
    L = (4 * math.pi,) * 2 if model == "fch" else (n[0] * math.pi / 4,) * 2
    args = (0.1, 0.1, 0.1, 0.0) if model == "fch" else (0.1,)
    old = os.environ.get("PAGD_CLUSTER")
    os.environ["PAGD_CLUSTER"] = cluster
    try:
        S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=prec)
    finally:
        if old is None:
            del os.environ["PAGD_CLUSTER"]
        else:
            os.environ["PAGD_CLUSTER"] = old
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args, scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    return S, P


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1][0]}-{c[2]}-{c[3]}")
def test_cluster_iterations_match_device_wide_and_oracle(torch, case):
    model, n, scheme, prec, dt, mean, tol, steps = case
    u0 = I.noisy_field(n, mean, 0.05, 51)
    outs, its = {}, {}
    for cl in ("1", "0"):
        S, P = _solver(case, cl)
        S.set_state(torch.from_numpy(u0).cuda())
        out = S.empty_field()
        it, res = S.run(dt, steps, tol, out)
        assert all(res <= tol)
        info = S.launch_info()
        if cl == "1":
            assert info["cluster"] == n[0] // 16
            assert info["grid"] % info["cluster"] == 0 and info["grid"] >= info["cluster"]
        else:
            assert info["cluster"] == 0
        outs[cl], its[cl] = out.cpu().numpy(), list(it)
    ref, oits = O.run(P, u0, dt, steps, tol)
    e_cl = np.linalg.norm(outs["1"] - outs["0"]) / np.linalg.norm(outs["0"])
    e_or = np.linalg.norm(outs["1"] - ref) / np.linalg.norm(ref)
    if prec == "fp64":
        assert e_cl <= 1e-12 and e_or <= 1e-12, (e_cl, e_or)
        assert all(abs(a - b) <= 1 for a, b in zip(its["1"], oits)), (its["1"], oits)
    else:
        assert e_cl <= 1e-6 and e_or <= 1e-6, (e_cl, e_or)
    assert abs(outs["1"].mean() - u0.mean()) <= 1e-12 * abs(u0.mean())


def test_cluster_trace_counts_every_evaluation(torch):
    """The loop records its column and row passes in the phase trace: the R1 and
    RI records still equal the evaluations the run reports."""
    case = CASES[0]
    S, _ = _solver(case, "1")
    S.set_state(torch.from_numpy(I.noisy_field(case[1], case[5], 0.05, 52)).cuda())
    S.run(case[4], 2, case[6])
    S.set_trace(True)
    its, _ = S.run(case[4], 5, case[6])
    names, t = S.get_trace()
    S.set_trace(False)
    assert np.all(np.diff(t) >= 0)
    assert names.count("R1") + names.count("RI") == int(np.sum(its))
    assert names.count("CI") == names.count("RI")
