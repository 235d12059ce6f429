"""Adaptive time stepping (pagd_run_adaptive, Algorithm 3) and R(v) = M Lap mu
(pagd_rhs) on the CPU emulation harness against the oracle: the same accepted
step sizes, the same rejections and the same final state (FP64).  No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

CASES = [
    ("fch", "bdf2", (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0), -0.3, 0.05, 1e-4, 1e-2),
    ("fch", "mp", (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.1), -0.3, 0.05, 1e-4, 1e-2),
    ("pfc", "lbdf2", (8 * math.pi,) * 2, (0.25, 0.0, 0.0, 0.0), 0.1, 2.0, 1e-2, 0.5),
    ("pfc", "mp", (8 * math.pi, 16 * math.pi), (0.25, 0.0, 0.0, 0.0), 0.1, 2.0, 1e-2, 0.5),
]


@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


@pytest.mark.parametrize("case", CASES)
def test_adaptive_matches_oracle(emu, case):
    model, scheme, L, args, mean, T, dmin, dmax = case
    n = (16, 16) if L[0] == L[1] else (16, 32)
    S = pagd.Solver(model, n, L, *args, scheme=scheme, lib=emu)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args,
                  scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2}[scheme])
    u0 = I.noisy_field(n, mean, 0.05, 4)
    v = I.noisy_field(n, mean, 0.3, 5)
    ref_r = O.rhs(P, v)
    assert np.abs(S.rhs(v) - ref_r).max() <= 1e-13 * np.abs(ref_r).max()
    S.set_state(u0)
    out = S.empty_field()
    t, dts, its, rej = S.run_adaptive(T, dmin, dmax, 1e-3, 1e-10, u_out=out)
    u, times, odts, orej, oits = O.run_adaptive(P, u0, T, dmin, dmax, 1e-3, 1e-10)
    assert len(dts) == len(odts) and rej == orej
    assert np.allclose(dts, odts, rtol=1e-12, atol=0)
    assert np.allclose(t, times, rtol=1e-12, atol=0)
    assert np.linalg.norm(out - u) <= 1e-12 * np.linalg.norm(u)
    un, _, st = S.get_state()
    assert st == len(dts) and np.array_equal(un, out)
