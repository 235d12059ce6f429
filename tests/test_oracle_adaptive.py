"""Pins of the oracle's adaptive time stepping (Sec. 3.1.2, Algorithm 3):
R(v) = M Lap mu(v) on single small modes against the linear symbol, the AM3
estimate's fourth-order local error on exact exponential data (any wrong
coefficient drops the order), the midAB2 extrapolation exact on quadratics in
time, and the adaptive driver's invariants.  No CUDA."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I


def _mode(P, r):
    axes = [np.arange(n) * (L / n) for n, L in zip(P.n, P.L)]
    X = np.meshgrid(*axes, indexing="ij")
    k = [2 * math.pi * ri / Li for ri, Li in zip(r, P.L)]
    return np.cos(sum(ki * xi for ki, xi in zip(k, X))), sum(ki * ki for ki in k)


def _sigma(P, kap):
    if P.model == O.PFC:
        m = 1 - P.eps - 2 * kap + kap * kap
    else:
        e = P.eps
        m = e ** 4 * kap * kap - e * e * (2 + P.eta1) * kap + (1 + P.eta2)
    return -P.M * kap * m


PROBLEMS = [O.Problem(O.PFC, (16, 16), (8 * math.pi,) * 2, eps=0.25),
            O.Problem(O.FCH, (16, 16), (2 * math.pi,) * 2, eps=0.18, eta1=0.0324, eta2=0.0324)]


@pytest.mark.parametrize("P", PROBLEMS)
def test_rhs_single_mode_is_the_linear_symbol(P):
    phi, kap = _mode(P, (1, 2))
    d = 1e-6  # nonlinear terms O(d^2) relative, rounding O(1e-16 / d)
    R = O.rhs(P, d * phi)
    assert np.abs(R - _sigma(P, kap) * d * phi).max() <= 1e-7 * abs(_sigma(P, kap)) * d
    assert abs(R.mean()) <= 1e-20


@pytest.mark.parametrize("rho", [1.0, 0.7, 1.6])
def test_am3_estimate_has_fourth_order_local_error(rho):
    P = PROBLEMS[0]
    phi, kap = _mode(P, (1, 1))
    sig = _sigma(P, kap)
    a0 = 1e-7
    errs = []
    for dt in (0.4, 0.2, 0.1):
        a = lambda t: a0 * math.exp(sig * t)
        un, unm1, ut = a(0.0) * phi, a(-dt / rho) * phi, a(dt) * phi
        _, uh = O.am3_err(P, un, ut, O.rhs(P, ut), O.rhs(P, un), O.rhs(P, unm1), dt, dt / rho)
        errs.append(np.abs(uh - ut).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, errs


def test_midab2_exact_on_quadratics_in_time():
    P = PROBLEMS[1]
    a, b, c = (I.noisy_field(P.n, 0.0, 1.0, s) for s in (1, 2, 3))
    q = lambda t: a + b * t + c * t * t
    dt, dtn, dtnm1 = 0.03, 0.05, 0.02
    err, uh = O.midab2_err(P, q(0.0), q(-dtn), q(-dtn - dtnm1), q(dt), dt, dtn, dtnm1)
    assert np.abs(uh - q(dt)).max() <= 1e-13 and err <= 1e-13


@pytest.mark.parametrize("scheme", [O.BDF2, O.MP, O.LBDF2])
def test_adaptive_driver_invariants(scheme):
    P = O.Problem(O.FCH, (16, 16), (2 * math.pi,) * 2, eps=0.18, eta1=0.0324, eta2=0.0324, scheme=scheme)
    u0 = I.noisy_field(P.n, -0.3, 0.05, 4)
    T, dmin, dmax = 0.05, 1e-4, 1e-2
    u, times, dts, rej, its = O.run_adaptive(P, u0, T, dmin, dmax, 1e-3, 1e-10)
    assert times[-1] >= T and np.all(np.diff(times) > 0)
    assert np.all(dts >= dmin * (1 - 1e-12)) and np.all(dts <= dmax * (1 + 1e-12))
    assert dts.max() > 4 * dmin  # the controller grows the step
    assert abs(u.mean() - u0.mean()) <= 1e-13
    # against a fine fixed-step run to the same final time
    nf = int(round(times[-1] / 5e-5))
    ref, _ = O.run(O.Problem(O.FCH, P.n, P.L, eps=0.18, eta1=0.0324, eta2=0.0324,
                             scheme=O.BDF2 if scheme != O.LBDF2 else O.LBDF2), u0, times[-1] / nf, nf, 1e-10)
    assert np.linalg.norm(u - ref) <= 1e-2 * np.linalg.norm(ref)
