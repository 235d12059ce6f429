"""Cluster-resident iterations (csrc/cluster.cuh) against the device-wide
phase sequence, on the CPU emulation of the kernels.

The two paths run the same PAGD iterations (Algorithm 2) with the same
arithmetic per point and the same decisions after each evaluation; only the
data movement differs (distributed shared memory and cluster barriers instead
of global memory and device barriers), and columns 0 and n/2 of the half
spectrum share one complex transform.  FP64 runs must agree to rounding with
identical iteration counts; FP32-mixed runs to well below the stopping
tolerance, also with identical counts."""
import math
import os

import numpy as np
import pytest

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

CASES = [
    ("fch", (64, 64), "bdf2", "fp32_mixed", 1e-3, -0.3, 1e-8),
    ("fch", (64, 64), "mp", "fp64", 1e-3, -0.3, 1e-10),
    ("pfc", (64, 64), "mp", "fp32_mixed", 0.1, 0.1, 1e-8),
    ("pfc", (64, 64), "bdf2", "fp64", 0.1, 0.07, 1e-10),
    ("fch", (128, 128), "bdf2", "fp32_mixed", 1e-3, -0.3, 1e-8),
]


def _run(case, cluster, steps):
    model, n, scheme, prec, dt, mean, tol = case
    L = (4 * math.pi,) * 2 if model == "fch" else (n[0] * math.pi / 4,) * 2
    args = (0.1, 0.1, 0.1, 0.0) if model == "fch" else (0.1,)
    old = os.environ.get("PAGD_CLUSTER")
    os.environ["PAGD_CLUSTER"] = cluster
    try:
        S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=prec, lib=pagd.load_emulation())
    finally:
        if old is None:
            del os.environ["PAGD_CLUSTER"]
        else:
            os.environ["PAGD_CLUSTER"] = old
    S.set_state(I.noisy_field(n, mean, 0.05, 7))
    out = S.empty_field()
    its, res = S.run(dt, steps, tol, out)
    return S, out, its, res


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1][0]}-{c[2]}-{c[3]}")
def test_cluster_iterations_match_device_wide_phases(case):
    steps = 2 if case[1][0] > 64 else 4
    S1, u1, it1, r1 = _run(case, "1", steps)
    S0, u0, it0, r0 = _run(case, "0", steps)
    assert S1.launch_info()["cluster"] == case[1][0] // 16
    assert S0.launch_info()["cluster"] == 0
    assert list(it1) == list(it0)
    assert all(r1 <= case[6])
    err = np.linalg.norm(u1 - u0) / np.linalg.norm(u0)
    assert err <= (1e-13 if case[3] == "fp64" else 1e-7), err
