"""GPU parity of the solver knobs of Table 1 and Algorithms 1 / 2: PGD
(accel = 0, Algorithm 1), the literal MP preconditioner (theta_mode = 1), a
non-default sweeping friction list and step size, each against the FP64 oracle
run with the same knobs on the same seeded inputs.  FP64 runs must match the
oracle's iterates (1e-12 relative L2 on u after several steps) and its
iteration counts (within one, from summation order at the stopping test);
FP32-mixed runs 1e-6 relative L2."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    t.cuda.set_device(0)
    return t


@pytest.fixture(scope="module")
def lib():
    return pagd.load()


KNOBS = {
    "pgd": dict(accel=0),
    "theta_literal": dict(theta_mode=1),
    "eta_list": dict(eta=(0.3, 0.9, 1.7)),
    "eta_one_s": dict(eta=(1.2,), s=0.6),
}

PROBLEMS = [
    ("pfc", (32, 32), (16 * math.pi,) * 2, (0.25,), 0.5, 0.1),
    ("fch", (64, 64), (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0), 0.01, -0.3),
]


def _oracle(model, n, L, args, scheme, kn):
    return O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args,
                     scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme], **kn)


@pytest.mark.parametrize("knob", sorted(KNOBS))
@pytest.mark.parametrize("prob", PROBLEMS, ids=lambda p: p[0])
@pytest.mark.parametrize("scheme", ["bdf2", "mp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_knob_matches_oracle(torch, lib, knob, prob, scheme, precision):
    model, n, L, args, dt, mean = prob
    kn = KNOBS[knob]
    if knob == "theta_literal" and scheme != "mp":
        pytest.skip("theta_mode only changes the MP preconditioner")
    tol = 1e-10 if precision == "fp64" else 1e-8
    S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib, **kn)
    P = _oracle(model, n, L, args, scheme, kn)
    u0 = I.noisy_field(n, mean, 0.05, 41)
    S.set_state(torch.from_numpy(u0).cuda())
    out = S.empty_field()
    nst = 4
    its, res = S.run(dt, nst, tol, out)
    ref, oits = O.run(P, u0, dt, nst, tol)
    u = out.cpu().numpy()
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert all(res <= tol)
    if precision == "fp64":
        assert err <= 1e-12, err
        assert all(abs(a - b) <= 1 for a, b in zip(its, oits)), (list(its), oits)
    else:
        assert err <= 1e-6, err
    assert abs(u.mean() - u0.mean()) <= 1e-12 * abs(u0.mean())


def test_pgd_takes_more_iterations_than_pagd_on_gpu(torch, lib):
    """Table 2's finding on the GPU path: the same hard FCH steps take more
    residual evaluations with PGD (Algorithm 1) than with PAGD (Algorithm 2),
    and the two reach the same discrete solution."""
    n, L, args = (64, 64), (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0)
    u0 = torch.from_numpy(I.noisy_field(n, -0.3, 0.05, 42)).cuda()
    outs, counts = [], []
    for accel in (1, 0):
        S = pagd.Solver("fch", n, L, *args, scheme="bdf2", accel=accel, lib=lib)
        S.set_state(u0)
        out = S.empty_field()
        its, _ = S.run(0.05, 3, 1e-11, out)
        outs.append(out.cpu().numpy())
        counts.append(int(np.sum(its)))
    assert counts[0] < counts[1], counts
    assert np.abs(outs[0] - outs[1]).max() <= 1e-9
