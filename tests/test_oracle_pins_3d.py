"""Pins of the FP64 oracle in three dimensions (the paper's Secs. 2-3 are
written for any dimension; kappa = |k|^2 sums over the three axes and the
trapezoidal weights are h0 h1 h2).  Closed forms, finite differences and the
exact single-mode recurrences, on grids whose axes differ so that an axis mix-up
fails.  No CUDA."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def grid(P):
    axes = [np.arange(n) * (L / n) for n, L in zip(P.n, P.L)]
    return np.meshgrid(*axes, indexing="ij")


def kvec(P, r):
    return [2 * math.pi * ri / Li for ri, Li in zip(r, P.L)]


def ipN(P, u, v):
    return float(np.sum(u * v)) * float(np.prod([L / n for n, L in zip(P.n, P.L)]))


def smooth_field(P, mean, amps, seed):
    X = grid(P)
    rng = np.random.default_rng(seed)
    u = np.full(P.shape, mean, dtype=np.float64)
    for a in amps:
        r = rng.integers(-2, 3, size=P.dim)
        ph = rng.uniform(0, 2 * math.pi)
        k = kvec(P, r)
        u += a * np.cos(sum(ki * xi for ki, xi in zip(k, X)) + ph)
    return u


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_pfc_energy_closed_form_3d(axis):
    """E_PFC of c + A cos(k x_axis) on a box (Eq. obj:PFC-egy): the grid mean of
    the energy density times the volume, exact on the grid."""
    eps, c, A = 0.3, -0.25, 0.2
    L = (8 * math.pi, 4 * math.pi, 16 * math.pi)
    P = O.Problem(O.PFC, (16, 8, 32), L, eps=eps)
    X = grid(P)
    k = 2 * math.pi * 1 / L[axis]  # u^4 holds mode 4: below every axis's Nyquist
    u = c + A * np.cos(k * X[axis])
    avg = (0.25 * (c ** 4 + 3 * c * c * A * A + 3 * A ** 4 / 8)
           + 0.5 * (1 - eps) * (c * c + A * A / 2)
           - A * A * k * k / 2 + 0.5 * A * A * k ** 4 / 2)
    vol = L[0] * L[1] * L[2]
    assert abs(O.energy(P, u) - avg * vol) <= 1e-12 * vol


@pytest.mark.parametrize("model", [O.PFC, O.FCH])
def test_mu_is_variational_derivative_of_energy_3d(model):
    if model == O.PFC:
        P = O.Problem(O.PFC, (8, 16, 8), (8 * math.pi, 16 * math.pi, 8 * math.pi), eps=0.3)
        u = smooth_field(P, -0.25, [0.3, 0.2, 0.1], 3)
    else:
        P = O.Problem(O.FCH, (8, 8, 16), (2 * math.pi, 2 * math.pi, 4 * math.pi), eps=0.18,
                      eta1=0.0324, eta2=0.0324, tau=0.125)
        u = smooth_field(P, -0.2, [0.4, 0.2, 0.1], 3)
    w = smooth_field(P, 0.05, [0.3, 0.3], 4)
    t = 1e-3
    E = lambda s: O.energy(P, u + s * w)
    fd = (-E(2 * t) + 8 * E(t) - 8 * E(-t) + E(-2 * t)) / (12 * t)
    an = ipN(P, O.mu(P, u), w)
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


@pytest.mark.parametrize("scheme", [O.BDF2, O.MP])
def test_gradient_is_derivative_of_objective_3d(scheme):
    P = O.Problem(O.PFC, (8, 16, 8), (8 * math.pi, 16 * math.pi, 4 * math.pi), eps=0.3, scheme=scheme)
    un = smooth_field(P, -0.25, [0.2, 0.1], 5)
    unm1 = smooth_field(P, -0.25, [0.2, 0.1], 6)
    v = smooth_field(P, -0.25, [0.25, 0.1], 7)
    abc = O.coeffs(scheme, 1, 0.5, 0.4)
    w = smooth_field(P, 0.0, [0.3, 0.2], 8)
    w -= w.mean()
    t = 1e-3
    G = lambda s: O.objective(P, abc, un, unm1, v + s * w)
    fd = (-G(2 * t) + 8 * G(t) - 8 * G(-t) + G(-2 * t)) / (12 * t)
    an = ipN(P, O.gradient(P, abc, un, unm1, v), w)
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


@pytest.mark.parametrize("scheme", [O.BDF2, O.MP])
def test_single_mode_linear_evolution_3d(scheme):
    """A tiny 3D mode around 0 follows the scheme's scalar recurrence with
    sigma = -kappa (1 - eps - 2 kappa + kappa^2), kappa = k0^2 + k1^2 + k2^2."""
    P = O.Problem(O.PFC, (8, 16, 8), (8 * math.pi, 16 * math.pi, 8 * math.pi), eps=0.3, scheme=scheme)
    r, dt = (1, 3, 2), 0.5
    X = grid(P)
    k = kvec(P, r)
    kap = sum(ki * ki for ki in k)
    phi = np.cos(sum(ki * xi for ki, xi in zip(k, X)))
    delta = 1e-6
    m = 1 - P.eps - 2 * kap + kap * kap
    u = [delta * phi, delta * phi]
    amps = [delta, delta]
    for n in range(3):
        res = O.pagd_step(P, n, u[-1], u[-2], dt, dt, tol=1e-17)
        assert res.status == O.OK
        a, b, c = O.coeffs(scheme, n, dt, dt)
        An, Am = amps[-1], amps[-2]
        if scheme == O.BDF2:
            Anew = -(b * An + c * Am) / (a + kap * m)
        else:
            Anew = -(b + kap * m / 2) * An / (a + kap * m / 2)
        got = ipN(P, res.u, phi) / ipN(P, phi, phi)
        assert abs(got - Anew) <= 1e-9 * abs(Anew)
        assert np.abs(res.u - got * phi).max() <= 1e-15
        u.append(res.u)
        amps.append(got)


def test_mass_conserved_3d():
    P = O.Problem(O.PFC, (8, 8, 16), (8 * math.pi, 8 * math.pi, 16 * math.pi), eps=0.3, scheme=O.BDF2)
    u0 = smooth_field(P, -0.25, [0.1, 0.05], 9)
    ref, its = O.run(P, u0, 0.5, 3, 1e-12)
    assert abs(O.mass(P, ref) - O.mass(P, u0)) <= 1e-12 * abs(O.mass(P, u0))
