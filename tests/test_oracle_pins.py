"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (closed forms, brute force, invariants, finite differences,
library routines).  None of these tests touches the CUDA library.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
sign, a transposed index, a wrong normalisation) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def grid(P):
    axes = [np.arange(n) * (L / n) for n, L in zip(P.n, P.L)]
    return np.meshgrid(*axes, indexing="ij")


def kvec(P, r):
    return [2 * math.pi * ri / Li for ri, Li in zip(r, P.L)]


def ipN(P, u, v):
    return float(np.sum(u * v)) * float(np.prod([L / n for n, L in zip(P.n, P.L)]))


def smooth_field(P, mean, amps, seed):
    """mean + a few low Fourier modes with seeded coefficients."""
    X = grid(P)
    rng = np.random.default_rng(seed)
    u = np.full(P.shape, mean, dtype=np.float64)
    for a in amps:
        r = rng.integers(-2, 3, size=P.dim)
        ph = rng.uniform(0, 2 * math.pi)
        k = kvec(P, r)
        u += a * np.cos(sum(ki * xi for ki, xi in zip(k, X)) + ph)
    return u


# ---------------------------------------------------------------------- FFT

@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (4, 4, 4), (8, 4), (2, 16)])
def test_fft_matches_brute_force_dft(shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for sign in (-1, +1):
        a = O.fft(x, sign)
        b = O.dft_brute(x, sign)
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("shape", [(64, 32), (16, 8, 32), (256,)])
def test_fft_matches_numpy(shape):
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.allclose(O.fft(x, -1), np.fft.fftn(x), rtol=0, atol=1e-11)
    assert np.allclose(O.fft(x, +1), np.fft.ifftn(x) * x.size, rtol=0, atol=1e-11)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.fft(np.zeros((6, 8), complex))


# ------------------------------------------------------- spectral operators

@pytest.mark.parametrize("r", [(1, 0), (2, 3), (-3, 1), (4, 4)])
def test_fractional_laplacian_single_modes(r):
    """(-Lap_N)^alpha of cos(k.x) is kappa^alpha cos(k.x) (Eq. def:frac-Lap)."""
    P = O.Problem(O.PFC, (8, 16), (2.0, 3.0), eps=0.1)
    X = grid(P)
    k = kvec(P, r)
    kap = sum(ki * ki for ki in k)
    w = np.cos(sum(ki * xi for ki, xi in zip(k, X)) + 0.3)
    for alpha in (-1, 1, 2):
        out = O.frac_lap(P, w, alpha)
        assert np.abs(out - kap ** alpha * w).max() <= 1e-12 * max(1.0, kap ** alpha)
    # zero mode: inverse Laplacian annihilates constants
    assert np.abs(O.frac_lap(P, np.ones(P.shape), -1)).max() <= 1e-15


def test_negative_norm_single_mode():
    """||A cos(k.x)||_{-1,N}^2 = |Omega| A^2 / (2 kappa) (Eq. def:neg-norm)."""
    P = O.Problem(O.FCH, (16, 16), (2 * math.pi, 4.0), eps=0.1, eta1=0.1, eta2=0.1)
    X = grid(P)
    k = kvec(P, (2, 1))
    kap = sum(ki * ki for ki in k)
    w = 0.7 * np.cos(k[0] * X[0] + k[1] * X[1])
    got = ipN(P, O.frac_lap(P, w, -1), w)
    assert abs(got - 2 * math.pi * 4.0 * 0.49 / (2 * kap)) <= 1e-13


def test_mass_of_constant_and_mode():
    P = O.Problem(O.PFC, (8, 16), (3.0, 5.0), eps=0.1)
    X = grid(P)
    assert abs(O.mass(P, np.full(P.shape, 0.25)) - 0.25 * 15.0) <= 1e-14
    k = kvec(P, (1, 2))
    assert abs(O.mass(P, np.cos(k[0] * X[0] + k[1] * X[1]))) <= 1e-13


# ------------------------------------------------------------ energies

def test_pfc_energy_closed_form():
    """E_PFC of c + A cos(k x) by hand (Eq. obj:PFC-egy); exact on the grid."""
    eps, c, A = 0.025, 0.07, 0.3
    L = 8 * math.pi
    P = O.Problem(O.PFC, (16, 16), (L, L), eps=eps)
    X = grid(P)
    k = 2 * math.pi * 3 / L
    u = c + A * np.cos(k * X[1])
    avg = (0.25 * (c ** 4 + 3 * c * c * A * A + 3 * A ** 4 / 8)
           + 0.5 * (1 - eps) * (c * c + A * A / 2)
           - A * A * k * k / 2 + 0.5 * A * A * k ** 4 / 2)
    assert abs(O.energy(P, u) - avg * L * L) <= 1e-12 * L * L


def _F_poly(z, tau):
    """Expanded double well: F = z^4/4 + tau z^3/3 - z^2/2 - tau z + (1/2 - 4 tau/3)/2."""
    return 0.25 * z ** 4 + tau * z ** 3 / 3 - 0.5 * z ** 2 - tau * z + 0.5 * (0.5 - 4 * tau / 3)


def _F1_poly(z, tau):
    return (z * z - 1) * (z + tau)


def _F2_poly(z, tau):
    return 3 * z * z + 2 * tau * z - 1


def _F3_poly(z, tau):
    return 6 * z + 2 * tau


@pytest.mark.parametrize("tau", [0.0, 0.125])
def test_fch_energy_closed_form(tau):
    """E_FCH of c + A cos(k x) (Eq. obj:FCHegy), integrated with analytic
    derivatives on a fine periodic quadrature (exact for trig polynomials)."""
    eps, eta1, eta2 = 0.1, 0.145, 0.2
    L = 4 * math.pi
    P = O.Problem(O.FCH, (16, 16), (L, L), eps=eps, eta1=eta1, eta2=eta2, tau=tau)
    c, A, r = -0.3, 0.4, 2
    k = 2 * math.pi * r / L
    X = grid(P)
    u = c + A * np.cos(k * X[0])
    t = np.arange(256) * (L / 256)
    ut = c + A * np.cos(k * t)
    lap = -k * k * A * np.cos(k * t)
    grad2 = (k * A * np.sin(k * t)) ** 2
    f = 0.5 * (eps * eps * lap - _F1_poly(ut, tau)) ** 2 - (0.5 * eps * eps * eta1 * grad2
                                                             + eta2 * _F_poly(ut, tau))
    exact = f.mean() * L * L
    assert abs(O.energy(P, u) - exact) <= 1e-12 * max(1.0, abs(exact))


@pytest.mark.parametrize("model", [O.PFC, O.FCH])
def test_mu_is_variational_derivative_of_energy(model):
    """(mu(u), w)_N = d/dt E_N(u + t w) (Sec. 2): five-point central difference."""
    if model == O.PFC:
        P = O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.3)
        u = smooth_field(P, 0.1, [0.3, 0.2, 0.1], 3)
    else:
        P = O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.0324,
                      eta2=0.0324, tau=0.125)
        u = smooth_field(P, -0.2, [0.4, 0.2, 0.1], 3)
    w = smooth_field(P, 0.05, [0.3, 0.3], 4)
    t = 1e-3
    E = lambda s: O.energy(P, u + s * w)
    fd = (-E(2 * t) + 8 * E(t) - 8 * E(-t) + E(-2 * t)) / (12 * t)
    an = ipN(P, O.mu(P, u), w)
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


# ------------------------------------------------ objective and gradient

@pytest.mark.parametrize("model,scheme", [(O.PFC, O.BDF2), (O.PFC, O.MP), (O.FCH, O.BDF2),
                                          (O.FCH, O.MP)])
def test_gradient_is_derivative_of_objective(model, scheme):
    """(G'_N(v), w)_N = d/dt G_N(v + t w) for mean-zero w (Proposition, Eqs.
    obj:FCH-mini-objv and obj:G')."""
    if model == O.PFC:
        P = O.Problem(O.PFC, (16, 8), (8 * math.pi, 4 * math.pi), eps=0.2, scheme=scheme)
        un = smooth_field(P, 0.1, [0.2, 0.1], 5)
        unm1 = smooth_field(P, 0.1, [0.2, 0.1], 6)
        v = smooth_field(P, 0.1, [0.25, 0.1], 7)
    else:
        P = O.Problem(O.FCH, (16, 8), (2 * math.pi, math.pi), eps=0.18, eta1=0.05, eta2=0.07,
                      tau=0.1, scheme=scheme)
        un = smooth_field(P, -0.3, [0.2, 0.1], 5)
        unm1 = smooth_field(P, -0.3, [0.2, 0.1], 6)
        v = smooth_field(P, -0.3, [0.25, 0.1], 7)
    abc = O.coeffs(scheme, 1, 0.1, 0.07)
    w = smooth_field(P, 0.0, [0.3, 0.2], 8)
    w -= w.mean()
    t = 1e-3
    G = lambda s: O.objective(P, abc, un, unm1, v + s * w)
    fd = (-G(2 * t) + 8 * G(t) - 8 * G(-t) + G(-2 * t)) / (12 * t)
    an = ipN(P, O.gradient(P, abc, un, unm1, v), w)
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


def test_gradient_has_zero_mean():
    P = O.Problem(O.FCH, (8, 8), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.1, eta2=0.1)
    un = I.noisy_field(P.shape, -0.3, 0.05, 1)
    g = O.gradient(P, O.coeffs(O.BDF2, 1, 0.01, 0.01), un, un, un + 0.01)
    assert abs(g.mean()) <= 1e-15


# ------------------------------------------------------------ schemes

def test_bdf2_coefficients_closed_forms():
    """Fixed step: (3/2, -2, 1/2)/dt; first step backward Euler (obj:BDF2)."""
    dt = 0.1
    assert np.allclose(O.coeffs(O.BDF2, 3, dt, dt), [1.5 / dt, -2 / dt, 0.5 / dt], rtol=1e-15)
    assert np.allclose(O.coeffs(O.BDF2, 0, dt, 123.0), [1 / dt, -1 / dt, 0.0], rtol=1e-15)
    assert np.allclose(O.coeffs(O.MP, 7, dt, 0.3), [1 / dt, -1 / dt, 0.0], rtol=1e-15)


@pytest.mark.parametrize("dt,dtp", [(0.1, 0.1), (0.2, 0.05), (0.03, 0.11)])
def test_variable_bdf2_is_exact_on_quadratics(dt, dtp):
    """Variable-step BDF2 differentiates quadratics exactly at t_{n+1}."""
    a, b, c = O.coeffs(O.BDF2, 1, dt, dtp)
    t1, t0, tm = dt + dtp, dtp, 0.0
    for f, df in [(lambda t: 1.0, 0.0), (lambda t: t, 1.0), (lambda t: t * t, 2 * t1)]:
        assert abs(a * f(t1) + b * f(t0) + c * f(tm) - df) <= 1e-12 / min(dt, dtp)


def test_golden_table1_settings():
    vals = {}
    with open(os.path.join(GOLD, "table1_solver_settings.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            vals[key] = [float(x) for x in rest]
    eta = [math.sqrt(x) for x in vals["eta_sq"]]
    assert np.allclose(eta, O.PAPER_ETA, rtol=1e-15)
    assert np.allclose(eta, I.PAPER_ETA, rtol=1e-15)
    # equally spaced on [0.1, 2]
    assert np.allclose(np.diff(vals["eta_sq"]), 0.475)
    assert vals["max_iter"] == [1000.0]
    # extrapolation coefficients lambda = (1 - eta sqrt s)/(1 + eta sqrt s) at s = 0.9
    lam = [(1 - e * math.sqrt(0.9)) / (1 + e * math.sqrt(0.9)) for e in eta]
    assert lam[0] > 0.5 and lam[-1] < 0 and all(np.diff(lam) < 0)


# -------------------------------------------------------- preconditioner

@pytest.mark.parametrize("scheme", [O.BDF2, O.MP])
def test_betas_on_constant_fields(scheme):
    """Averaged-Newton constants for a constant argument (Sec. 3.4.1)."""
    th = 0.5 if scheme == O.MP else 1.0
    P = O.Problem(O.PFC, (8, 8), (1.0, 1.0), eps=0.3, scheme=scheme, M=2.0)
    c = 0.2
    b = O.betas(P, 10.0, np.full(P.shape, c))
    assert np.allclose(b, [5.0, th * abs(3 * c * c + 1 - 0.3), -2 * th, th], rtol=1e-14)
    for tau in (0.0, 0.125):
        P = O.Problem(O.FCH, (8, 8), (1.0, 1.0), eps=0.1, eta1=0.145, eta2=0.2, tau=tau,
                      scheme=scheme)
        c = -0.3
        f1, f2, f3 = _F1_poly(c, tau), _F2_poly(c, tau), _F3_poly(c, tau)
        b = O.betas(P, 1000.0, np.full(P.shape, c))
        exp = [1000.0, th * abs(f2 * f2 - 0.2 * f2 + f3 * f1), th * abs(0.01 * (f2 - 0.145)),
               th * 1e-4]
        assert np.allclose(b, exp, rtol=1e-13)


# ------------------------------------------------------ linear evolution

def _lin_symbol(P, kap):
    if P.model == O.PFC:
        return 1 - P.eps - 2 * kap + kap * kap
    e = P.eps
    return e ** 4 * kap * kap - e * e * (2 + P.eta1) * kap + (1 + P.eta2)


def _split_L(P, kap):
    if P.model == O.PFC:
        return (1 - kap) ** 2
    k0 = 1 - 2 * P.tau ** 2 + P.eta2
    return P.eps ** 4 * kap * kap + kap + k0


@pytest.mark.parametrize("model", [O.PFC, O.FCH])
@pytest.mark.parametrize("scheme", [O.BDF2, O.MP, O.LBDF2, O.LMP])
def test_single_mode_linear_evolution(model, scheme):
    """Tiny single Fourier mode around 0: each scheme reduces to its exact
    scalar recurrence with the linear symbol sigma = -M kappa m(kappa)
    (PFC m = 1 - eps - 2 kappa + kappa^2; FCH m = eps^4 kappa^2
    - eps^2 (2 + eta1) kappa + 1 + eta2).  Nonlinear terms are O(delta^2)."""
    if model == O.PFC:
        P = O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=scheme)
        r, dt = (1, 4), 0.5
    else:
        P = O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.0324,
                      eta2=0.0324, scheme=scheme)
        r, dt = (1, 2), 0.01
    X = grid(P)
    k = kvec(P, r)
    kap = k[0] ** 2 + k[1] ** 2
    phi = np.cos(k[0] * X[0] + k[1] * X[1])
    delta = 1e-6
    m = _lin_symbol(P, kap)
    Lh = _split_L(P, kap)
    u = [delta * phi, delta * phi]  # u^{-1} := u^0
    amps = [delta, delta]
    for n in range(4):
        if scheme in (O.BDF2, O.MP):
            res = O.pagd_step(P, n, u[-1], u[-2], dt, dt, tol=1e-20 * 1e3)
            assert res.status == O.OK
            unew = res.u
        else:
            unew = O.imex_step(P, n, u[-1], u[-2], dt, dt)
        a, b, c = O.coeffs(scheme, n, dt, dt)
        An, Am = amps[-1], amps[-2]
        rho = 0.0 if n == 0 else 1.0
        if scheme == O.BDF2:
            Anew = -(b * An + c * Am) / (a + kap * m)
        elif scheme == O.MP:
            Anew = -(b + kap * m / 2) * An / (a + kap * m / 2)
        elif scheme == O.LBDF2:
            ub = An + rho * (An - Am)
            Anew = (-(b * An + c * Am) - kap * (m - Lh) * ub) / (a + kap * Lh)
        else:
            ub = ((2 + rho) * An - rho * Am) / 2
            Anew = (-(b * An + c * Am) - kap * (Lh * An / 2 + (m - Lh) * ub)) / (a + kap * Lh / 2)
        got = ipN(P, unew, phi) / ipN(P, phi, phi)
        assert abs(got - Anew) <= 1e-9 * abs(Anew)
        # nothing leaks into other modes beyond the nonlinear O(delta^3)
        assert np.abs(unew - got * phi).max() <= 1e-15
        u.append(unew)
        amps.append(got)


def test_imex_split_sums_to_mu():
    """L(u) + N(u) = mu(u) (Sec. 3.1.1 IMEX split): one backward-Euler IMEX step
    from u^{n-1} = u^n = w with a tiny dt gives (u^1 - w)/dt -> M Lap mu(w)."""
    for model in (O.PFC, O.FCH):
        if model == O.PFC:
            P = O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=O.LBDF2)
            w = smooth_field(P, 0.1, [0.3, 0.2], 9)
        else:
            P = O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.05,
                          eta2=0.07, tau=0.125, scheme=O.LBDF2)
            w = smooth_field(P, -0.2, [0.3, 0.2], 9)
        dt = 1e-9
        u1 = O.imex_step(P, 0, w, w, dt, dt)
        rate = (u1 - w) / dt
        target = -O.frac_lap(P, O.mu(P, w), 1) * P.M
        assert np.abs(rate - target).max() <= 1e-5 * np.abs(target).max()


# ---------------------------------------------- solver-level invariants

def _fch_small(scheme=O.BDF2, **kw):
    return O.Problem(O.FCH, (16, 16), (2 * math.pi, 2 * math.pi), eps=0.18, eta1=0.0324,
                     eta2=0.0324, scheme=scheme, **kw)


def _pfc_small(scheme=O.MP, **kw):
    return O.Problem(O.PFC, (16, 16), (8 * math.pi, 8 * math.pi), eps=0.25, scheme=scheme, **kw)


@pytest.mark.parametrize("mk", ["pfc", "fch"])
@pytest.mark.parametrize("scheme", [O.BDF2, O.MP])
def test_converged_step_solves_the_scheme(mk, scheme):
    """The accepted iterate satisfies eqn:FCH-fulldis-implicit (Proposition)."""
    if mk == "pfc":
        P = _pfc_small(scheme)
        u0 = smooth_field(P, 0.1, [0.3, 0.2, 0.1], 11)
        dt = 0.5
    else:
        P = _fch_small(scheme)
        u0 = smooth_field(P, -0.2, [0.3, 0.2, 0.1], 11)
        dt = 0.01
    u1 = O.pagd_step(P, 0, u0, u0, dt, dt, 1e-12).u
    r = O.pagd_step(P, 1, u1, u0, dt, dt, 1e-12)
    assert r.status == O.OK and r.iters >= 2
    res = O.scheme_residual(P, 1, u1, u0, dt, dt, r.u)
    scale = np.abs(O.coeffs(scheme, 1, dt, dt)[0] * r.u).max()
    assert np.abs(res).max() <= 1e-8 * scale


@pytest.mark.parametrize("mk", ["pfc", "fch"])
def test_solver_knobs_do_not_change_the_fixed_point(mk):
    """PGD, PAGD, the literal MP preconditioner and other friction lists all
    converge to the same discrete solution (Algorithms 1 and 2)."""
    base = _pfc_small(O.MP) if mk == "pfc" else _fch_small(O.MP)
    u0 = smooth_field(base, 0.1 if mk == "pfc" else -0.2, [0.3, 0.2], 12)
    dt = 0.5 if mk == "pfc" else 0.01
    ref = O.pagd_step(base, 0, u0, u0, dt, dt, 1e-13)
    assert ref.status == O.OK
    import dataclasses
    variants = [dataclasses.replace(base, accel=0), dataclasses.replace(base, theta_mode=1),
                dataclasses.replace(base, eta=(0.5, 1.0)), dataclasses.replace(base, s=0.5)]
    for V in variants:
        r = O.pagd_step(V, 0, u0, u0, dt, dt, 1e-13)
        assert r.status == O.OK
        assert np.abs(r.u - ref.u).max() <= 1e-10


def test_pagd_needs_fewer_iterations_than_pgd():
    """Table 2's qualitative finding on a hard FCH step (large dt, many iterations)."""
    P = _fch_small(O.BDF2)
    u0 = I.noisy_field(P.shape, -0.3, 0.05, 13)
    a = O.pagd_step(P, 0, u0, u0, 0.05, 0.05, 1e-10)
    import dataclasses
    b = O.pagd_step(dataclasses.replace(P, accel=0), 0, u0, u0, 0.05, 0.05, 1e-10)
    assert a.status == O.OK and b.status == O.OK
    assert a.iters < b.iters


@pytest.mark.parametrize("mk", ["pfc", "fch"])
def test_mass_is_conserved(mk):
    P = _pfc_small(O.MP) if mk == "pfc" else _fch_small(O.BDF2)
    u0 = I.noisy_field(P.shape, 0.1 if mk == "pfc" else -0.3, 0.05, 14)
    dt = 0.5 if mk == "pfc" else 0.01
    m0 = O.mass(P, u0)
    u, _ = O.run(P, u0, dt, 8, 1e-10)
    assert abs(O.mass(P, u) - m0) <= 1e-12 * abs(m0)


@pytest.mark.parametrize("mk", ["pfc", "fch"])
def test_energy_decreases(mk):
    """Energy dissipation (Sec. 2) carried by small-step backward Euler / BDF2."""
    P = _pfc_small(O.BDF2) if mk == "pfc" else _fch_small(O.BDF2)
    u0 = I.noisy_field(P.shape, 0.1 if mk == "pfc" else -0.3, 0.05, 15)
    dt = 0.1 if mk == "pfc" else 0.001
    es = [O.energy(P, u0)]
    O.run(P, u0, dt, 6, 1e-12, callback=lambda n, u: es.append(O.energy(P, u)))
    assert all(np.diff(es) < 0)


@pytest.mark.parametrize("mk", ["pfc", "fch"])
@pytest.mark.parametrize("scheme", [O.BDF2, O.MP, O.LBDF2, O.LMP])
def test_second_order_in_time(mk, scheme):
    """Self-convergence at fixed T: errors at dt and dt/2 against dt/8 shrink
    about 4x (all four schemes are second order, Sec. 3.1.1).  The FCH IMEX
    split treats stiff Laplacian terms explicitly, so its asymptotic range
    starts at smaller steps."""
    if mk == "pfc":
        P, mean, T = _pfc_small(scheme), 0.1, 2.0
    else:
        P, mean = _fch_small(scheme), -0.2
        T = 0.08 if scheme in (O.BDF2, O.MP) else 0.002
    u0 = smooth_field(P, mean, [0.3, 0.2], 16)
    sols = {}
    for m in (2, 4, 16):
        nst = 4 * m
        sols[m], _ = O.run(P, u0, T / nst, nst, 1e-13)
    e1 = np.abs(sols[2] - sols[16]).max()
    e2 = np.abs(sols[4] - sols[16]).max()
    ratio = e1 / e2
    assert 3.2 < ratio < 5.5, ratio


def test_nonconvergence_reports_status():
    P = _fch_small(O.BDF2, max_iter=3)
    u0 = I.noisy_field(P.shape, -0.3, 0.05, 17)
    r = O.pagd_step(P, 0, u0, u0, 0.01, 0.01, 1e-14)
    assert r.status == O.ENOCONV and r.iters == 3


def test_learned_guess_mass_projection():
    """A supplied initial iterate takes the mass of u^n before use."""
    P = _fch_small(O.BDF2)
    u0 = I.noisy_field(P.shape, -0.3, 0.05, 18)
    ref = O.pagd_step(P, 0, u0, u0, 0.01, 0.01, 1e-12)
    g = ref.u + 0.37  # wrong mass
    r = O.pagd_step(P, 0, u0, u0, 0.01, 0.01, 1e-12, guess=g)
    assert r.status == O.OK and r.iters <= 2
    assert np.abs(r.u - ref.u).max() <= 1e-10


def test_thread_count_does_not_change_results():
    """The oracle's line transforms may run on several host threads (the
    CPU baseline); every line is transformed as with one thread, so the
    transforms and a whole PAGD step are bit-identical."""
    n = (64, 32)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    P = O.Problem(O.FCH, n, (2 * math.pi, math.pi), 0.18, 0.05, 0.07, 0.1, scheme=O.BDF2)
    u = -0.3 + 0.05 * rng.uniform(-1, 1, n)
    out = {}
    try:
        for th in (1, 4):
            O.set_threads(th)
            r = O.pagd_step(P, 0, u, u.copy(), 0.01, 0.01, 1e-10)
            out[th] = (O.fft(x), r.u, r.iters)
    finally:
        O.set_threads(1)
    assert np.array_equal(out[1][0], out[4][0])
    assert np.array_equal(out[1][1], out[4][1]) and out[1][2] == out[4][2]
