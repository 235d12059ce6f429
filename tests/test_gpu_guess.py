"""GPU parity of pagd_step_with_guess against the FP64 oracle: a guess close to
the solution is kept and the step equals the oracle's step from that guess; a
poor guess falls back to the extrapolation (Sec. 3.4.2) and the step equals the
oracle's plain step.  FCH 256^2 (the bench workload) and PFC 64^2."""
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("w,bound", [(I.FCH256, 1e-6), (I.PFC64, 1e-9)])
def test_step_with_guess_matches_oracle(torch, w, bound):
    P = O.Problem(O.PFC if w.model == "pfc" else O.FCH, w.n, w.L, w.eps, w.eta1, w.eta2, w.tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[w.scheme])
    u0 = w.u0(1)
    tight = O.pagd_step(P, 0, u0, u0, w.dt, w.dt, 1e-12).u
    good = tight + 1e-7 * I.noisy_field(w.n, 0.0, 1.0, 9) + 0.2
    bad = I.noisy_field(w.n, w.mean, 0.3, 11)
    for g, expect_used in ((good, True), (bad, False)):
        S = pagd.solver_for(w)
        S.set_state(dev(torch, u0))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        its, res, used = S.step_with_guess(out, dev(torch, g), w.dt, w.tol)
        assert used == expect_used
        ref = O.pagd_step(P, 0, u0, u0, w.dt, w.dt, w.tol, guess=g if used else None)
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref.u) <= bound * np.linalg.norm(ref.u)
        assert res <= w.tol
        assert abs(got.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
