"""Exact pin of the momentum sweep of Algorithm 2 (and of Algorithm 1) in the
FP64 oracle.

On a single Fourier mode phi = cos(k.x) of tiny amplitude around u = 0 the
gradient G'_N (Eq. obj:G') is linear in the mode amplitude up to O(V^3), the
averaged Newton symbol (Sec. 3.4.1) is a number, and every PAGD iterate stays
a multiple of phi.  Writing x_i = X_i phi, Algorithm 2 becomes the scalar
recurrence

    Y_i     = X_i + lambda_i (X_i - X_{i-1}),  X_{-1} = X_0,
    D_i     = -(A Y_i + B) / Lcal,
    X_{i+1} = Y_i + s D_i,
    lambda_i = (1 - eta_j sqrt s) / (1 + eta_j sqrt s),  j = i mod n_eta,

with A, B the linear coefficients of G' in the mode and Lcal the symbol at its
wavenumber; ||d_i||_inf on the grid is |D_i| (max |cos| = 1 at x = 0).  The
recurrence below is written from those formulas alone and checked against
every entry of the oracle's ||d_i||_inf history, so a shifted friction list, a
wrong sign of lambda, a wrong sweep index, a missing momentum term or a wrong
preconditioner constant each fail it.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as O

# Mode amplitude and tolerance per model.  PFC: mu(V phi) has no cancellation,
# so V = 1e-8 leaves the O(V^2) nonlinearity and the rounding far below 1e-8.
# FCH: the oracle's F'(z) (product rule of Sec. 2.2's F) cancels to O(z) near
# 0, an absolute floor of about 1e-16 per point; V = 3e-6 balances that floor
# against the O(V^3) shift of the fixed point by the nonlinear terms, both a
# few 1e-6 of the smallest direction compared.
AMP = {O.PFC: (1e-8, 1e-8, 1e-6), O.FCH: (3e-6, 5e-6, 1e-4)}  # V, rtol, kept range


def _grid(P):
    axes = [np.arange(n) * (L / n) for n, L in zip(P.n, P.L)]
    return np.meshgrid(*axes, indexing="ij")


def _mode(P, r):
    X = _grid(P)
    k = [2 * math.pi * ri / Li for ri, Li in zip(r, P.L)]
    kap = sum(ki * ki for ki in k)
    return np.cos(sum(ki * xi for ki, xi in zip(k, X))), kap


def _linear_mu(P, kap):
    """mu(V phi) = m(kappa) V phi + O(V^3) around u = 0 (tau = 0).
    PFC (eqn:PFCsystem): u^3 + (1 - eps) u + 2 Lap u + Lap^2 u.
    FCH (eqn:FCHsystem with omega = eps^2 Lap u - F'(u), F'(z) = z^3 - z):
    eps^4 kappa^2 - eps^2 (2 + eta1) kappa + 1 + eta2."""
    if P.model == O.PFC:
        return 1 - P.eps - 2 * kap + kap * kap
    e2 = P.eps ** 2
    return e2 * e2 * kap * kap - e2 * (2 + P.eta1) * kap + 1 + P.eta2


def _symbol(P, a, kap, Vb0):
    """Averaged Newton symbol (Sec. 3.4.1) at the argument Vb0 phi of the
    initial guess: grid averages <phi^2> = 1/2, <phi^4> = 3/8."""
    th = 0.5 if (P.scheme == O.MP and P.theta_mode == 0) else 1.0
    z2, z4 = 0.5 * Vb0 ** 2, 0.375 * Vb0 ** 4
    if P.model == O.PFC:
        b0 = th * abs(3 * z2 + 1 - P.eps)
        b2, b4 = -2 * th, th
    else:
        e2 = P.eps ** 2
        # F''^2 - eta2 F'' + F''' F' = (1 + eta2) - (12 + 3 eta2) z^2 + 15 z^4
        b0 = th * abs((1 + P.eta2) - (12 + 3 * P.eta2) * z2 + 15 * z4)
        # eps^2 (F'' - eta1) = eps^2 (3 z^2 - 1 - eta1)
        b2 = th * abs(e2 * (3 * z2 - 1 - P.eta1))
        b4 = th * e2 * e2
    return (a / P.M) / kap + b0 + b2 * kap + b4 * kap * kap


def _recurrence(P, step, Un, Unm1, dt, kap, lams, niter):
    """|D_i| of Algorithm 2 (lams[i] = lambda_i; zeros give Algorithm 1)."""
    a, b, c = O.coeffs(P.scheme, step, dt, dt)
    m = _linear_mu(P, kap)
    rho = 0.0 if step == 0 else 1.0
    X0 = Un + rho * (Un - Unm1)
    if P.scheme == O.MP:
        # G'(V) = (a V + b U^n) / (M kappa) + m (V + U^n) / 2
        A, B = a / (P.M * kap) + m / 2, b * Un / (P.M * kap) + m * Un / 2
        Vb0 = (X0 + Un) / 2
    else:
        A, B = a / (P.M * kap) + m, (b * Un + c * Unm1) / (P.M * kap)
        Vb0 = X0
    Lc = _symbol(P, a, kap, Vb0)
    X, Xp = X0, X0
    out = []
    for i in range(niter):
        Y = X + lams[i] * (X - Xp)
        D = -(A * Y + B) / Lc
        Xp, X = X, Y + P.s * D
        out.append(abs(D))
    return np.array(out)


def _lams(P, niter, shift=0, sign=1.0):
    if not P.accel:
        return [0.0] * niter
    sq = math.sqrt(P.s)
    return [sign * (1 - P.eta[(i + shift) % len(P.eta)] * sq) / (1 + P.eta[(i + shift) % len(P.eta)] * sq)
            for i in range(niter)]


CASES = {
    # PFC around 0: the symbol matches G'' exactly for BDF2 and for MP with the
    # 1/2 of the second variation, so the PGD contraction is 1 - s
    "pfc_bdf2": (O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=O.BDF2), (1, 3), 0.5),
    "pfc_mp": (O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=O.MP), (2, 1), 0.5),
    # the literal MP symbol (theta_mode = 1) is twice the energy part of G''
    "pfc_mp_literal": (O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=O.MP,
                                 theta_mode=1), (2, 1), 0.5),
    # FCH: the symbol's eps^2 kappa term has the opposite sign of G''s, so the
    # contraction depends on kappa
    "fch_bdf2": (O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.0324, eta2=0.0324,
                           scheme=O.BDF2), (2, 3), 0.1),
    "fch_mp": (O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.05, eta2=0.07,
                         scheme=O.MP), (3, 1), 0.1),
    # a non-default step size and friction list (Table 1 knobs)
    "fch_bdf2_knobs": (O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.0324,
                                 eta2=0.0324, scheme=O.BDF2, s=0.6, eta=(0.3, 0.9, 1.7)), (2, 3), 0.1),
}

NITER = 14  # more than two sweeps of the default five-value friction list


def _oracle_hist(P, step, phi, Un, Unm1, dt):
    Pq = dataclasses.replace(P, max_iter=NITER)
    r = O.pagd_step(Pq, step, Un * phi, Unm1 * phi, dt, dt, tol=0.0)
    assert r.status == O.ENOCONV and r.iters == NITER
    return r.hist


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("accel", [1, 0])
@pytest.mark.parametrize("step", [0, 1])
def test_pagd_history_follows_the_scalar_recurrence(case, accel, step):
    P, r, dt = CASES[case]
    P = dataclasses.replace(P, accel=accel)
    phi, kap = _mode(P, r)
    V, rtol, rng = AMP[P.model]
    Un, Unm1 = V, 0.6 * V  # step 1: BDF2 history term and the extrapolated guess
    if step == 0:
        Unm1 = Un
    hist = _oracle_hist(P, step, phi, Un, Unm1, dt)
    ref = _recurrence(P, step, Un, Unm1, dt, kap, _lams(P, NITER), NITER)
    # compare while the direction is well above the rounding floor
    keep = ref >= rng * ref[0]
    assert keep.sum() >= 6
    np.testing.assert_allclose(hist[keep], ref[keep], rtol=rtol, atol=0)


@pytest.mark.parametrize("case", ["pfc_mp_literal", "fch_bdf2", "fch_mp", "fch_bdf2_knobs"])
def test_pin_rejects_plausible_slips(case):
    """The pin is sharp: the recurrence with the friction list shifted by one,
    with lambda of the wrong sign, or without momentum (PGD) misses the
    oracle's history by far more than the tolerance above."""
    P, r, dt = CASES[case]
    phi, kap = _mode(P, r)
    V, _, rng = AMP[P.model]
    Un, Unm1 = V, 0.6 * V
    hist = _oracle_hist(P, 1, phi, Un, Unm1, dt)
    ref = _recurrence(P, 1, Un, Unm1, dt, kap, _lams(P, NITER), NITER)
    keep = ref >= rng * ref[0]
    for lams in (_lams(P, NITER, shift=1), _lams(P, NITER, sign=-1.0), [0.0] * NITER):
        bad = _recurrence(P, 1, Un, Unm1, dt, kap, lams, NITER)
        err = np.max(np.abs(bad[keep] - hist[keep]) / hist[keep])
        assert err > 1e-4, err
