"""GPU parity of adaptive time stepping (pagd_run_adaptive, Algorithm 3) and of
R(v) = M Lap mu (pagd_rhs) against the oracle: same accepted steps and final
state in FP64; the FCH 256^2 workload in FP32-mixed against the oracle's
adaptive run (1e-6 on u)."""
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
    return t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("model,scheme,n,L,args,mean,T,dmin,dmax", [
    ("fch", "bdf2", (64, 64), (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0), -0.3, 0.05, 1e-4, 1e-2),
    ("pfc", "mp", (64, 32), (32 * math.pi, 16 * math.pi), (0.25, 0.0, 0.0, 0.0), 0.1, 3.0, 1e-2, 0.5),
    ("fch", "lbdf2", (64, 64), (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0), -0.3, 0.05, 1e-4, 1e-2),
])
def test_adaptive_fp64_matches_oracle(torch, model, scheme, n, L, args, mean, T, dmin, dmax):
    S = pagd.Solver(model, n, L, *args, scheme=scheme)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args,
                  scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2}[scheme])
    u0 = I.noisy_field(n, mean, 0.05, 4)
    v = I.noisy_field(n, mean, 0.3, 5)
    ref_r = O.rhs(P, v)
    assert np.abs(S.rhs(dev(torch, v)).cpu().numpy() - ref_r).max() <= 1e-12 * np.abs(ref_r).max()
    S.set_state(dev(torch, u0))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    t, dts, its, rej = S.run_adaptive(T, dmin, dmax, 1e-3, 1e-10, u_out=out)
    u, times, odts, orej, oits = O.run_adaptive(P, u0, T, dmin, dmax, 1e-3, 1e-10)
    assert len(dts) == len(odts) and rej == orej
    assert np.allclose(dts, odts, rtol=1e-9, atol=0)
    assert np.linalg.norm(out.cpu().numpy() - u) <= 1e-9 * np.linalg.norm(u)


def test_adaptive_fch256_mixed_against_oracle(torch):
    w = I.FCH256
    S = pagd.solver_for(w)
    u0 = w.u0(1)
    S.set_state(dev(torch, u0))
    out = torch.empty(w.n, dtype=torch.float64, device="cuda")
    T = 0.01
    t, dts, its, rej = S.run_adaptive(T, 1e-4, 5e-3, 1e-3, w.tol, u_out=out)
    P = O.Problem(O.FCH, w.n, w.L, w.eps, w.eta1, w.eta2, w.tau, scheme=O.BDF2)
    u, times, odts, orej, _ = O.run_adaptive(P, u0, T, 1e-4, 5e-3, 1e-3, w.tol)
    assert len(dts) == len(odts)
    assert np.allclose(dts, odts, rtol=1e-4)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - u) <= 1e-6 * np.linalg.norm(u)
    assert abs(got.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
