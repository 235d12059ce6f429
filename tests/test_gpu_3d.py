"""GPU parity on three-dimensional grids: DFT, energy and PAGD steps against
the FP64 oracle element by element on grids the oracle finishes in seconds
(up to 64^3), and the full PFC 256^3 workload (two seeds in one batch) on
properties that hold at any size: every step converges, mass is kept to 1e-12,
the energy decreases, and the oracle's own first PAGD direction at the accepted
state (Algorithm 2 started there) is within the tolerance."""
import dataclasses
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n", [(8, 8, 8), (64, 32, 128), (128, 128, 128)])
def test_3d_dft_energy_mass(torch, lib, n):
    L = (3.0, 5.0, 4.0)
    u = I.noisy_field(n, 0.1, 0.5, 3)
    S = pagd.Solver("pfc", n, L, 0.1, lib=lib)
    spec = host(S.fft_r2c(dev(torch, u)))
    ref = O.fft(u.astype(complex))[..., : n[-1] // 2 + 1]
    assert np.abs(spec[..., 0] + 1j * spec[..., 1] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(host(S.fft_c2r(dev(torch, spec))) - u).max() <= 1e-14
    for model, args in (("pfc", (0.1,)), ("fch", (0.1, 0.1, 0.2, 0.125))):
        S = pagd.Solver(model, n, L, *args, lib=lib)
        P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args)
        assert abs(S.energy(dev(torch, u)) - O.energy(P, u)) <= 1e-12 * abs(O.energy(P, u))
        assert abs(S.mass(dev(torch, u)) - O.mass(P, u)) <= 1e-13 * abs(O.mass(P, u))


CASES3 = [
    ("pfc", (16, 32, 16), (16 * math.pi, 32 * math.pi, 16 * math.pi), 0.3, 0, 0, 0, "bdf2", 0.5, -0.25),
    ("pfc", (32, 32, 32), (32 * math.pi,) * 3, 0.3, 0, 0, 0, "mp", 0.5, -0.25),
    ("fch", (16, 16, 32), (2 * math.pi, 2 * math.pi, 4 * math.pi), 0.18, 0.05, 0.07, 0.1, "bdf2", 0.01,
     -0.3),
    ("pfc", (64, 64, 64), (64 * math.pi / 4,) * 3, 0.3, 0, 0, 0, "bdf2", 0.5, -0.25),
]


@pytest.mark.parametrize("case", CASES3)
@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("fp32_mixed", 1e-8, 1e-6)])
def test_3d_steps_match_oracle(torch, lib, case, precision, tol, bound):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=precision, lib=lib)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    u0 = I.noisy_field(n, mean, 0.1, 7)
    S.set_state(dev(torch, u0))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    its, res = S.run(dt, 2, tol, out)
    ref, oits = O.run(P, u0, dt, 2, tol)
    got = host(out)
    assert np.linalg.norm(got - ref) <= bound * np.linalg.norm(ref)
    assert np.all(res <= tol)
    assert abs(got.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
    if precision == "fp64":
        assert list(its) == list(oits)


@pytest.mark.parametrize("scheme", ["lbdf2", "lmp"])
def test_3d_imex_matches_oracle(torch, lib, scheme):
    model, n, L, eps, e1, e2, tau, _, dt, mean = CASES3[2]
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, lib=lib)
    P = O.Problem(O.FCH, n, L, eps, e1, e2, tau, scheme={"lbdf2": O.LBDF2, "lmp": O.LMP}[scheme])
    u0 = I.noisy_field(n, mean, 0.1, 9)
    S.set_state(dev(torch, u0))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    S.run(dt, 3, 0.0, out)
    ref, _ = O.run(P, u0, dt, 3, 0.0)
    assert np.linalg.norm(host(out) - ref) <= 1e-12 * np.linalg.norm(ref)


def _oracle_direction_norm(w, step, un, unm1, u):
    """||d_0||_inf of the oracle's Algorithm 2 started at u (one direction)."""
    P = O.Problem(O.PFC, w.n, w.L, w.eps, scheme=O.BDF2 if w.scheme == "bdf2" else O.MP, max_iter=1)
    r = O.pagd_step(P, step, un, unm1, w.dt, w.dt, 0.0, guess=u)
    return float(r.hist[0])


@pytest.fixture(scope="module")
def batch3d(torch, lib):
    w = I.PFC3D256
    solvers, u0s = [], []
    for seed in w.seeds:
        S = pagd.solver_for(w, lib=lib)
        u0 = w.u0(seed)
        S.set_state(dev(torch, u0))
        solvers.append(S)
        u0s.append(u0)
    return w, solvers, u0s, pagd.Batch(solvers)


def test_pfc3d_256_first_step_is_a_fixed_point_of_the_oracle(torch, batch3d):
    w, solvers, u0s, Bt = batch3d
    E0 = solvers[0].energy(dev(torch, u0s[0]))
    its, res, status = Bt.run(w.dt, 1, w.tol)
    assert np.all(status == 0) and np.all(res <= w.tol)
    u1 = host(solvers[0].get_state()[0])
    dn = _oracle_direction_norm(w, 0, u0s[0], u0s[0], u1)
    assert dn <= 2 * w.tol, dn
    assert solvers[0].energy(dev(torch, u1)) < E0


def test_pfc3d_256_full_run_properties(torch, batch3d):
    """Steps 2..200: every step converges, mass is kept, the energy decreases;
    the last step is checked by the oracle's direction at the accepted state."""
    w, solvers, u0s, Bt = batch3d
    E1 = [S.energy(S.get_state()[0]) for S in solvers]
    its, res, status = Bt.run(w.dt, w.steps - 2, w.tol)
    assert np.all(status == 0)
    assert np.all(res <= w.tol) and its.max() < 1000
    un, unm1, _ = solvers[1].get_state()
    un, unm1 = host(un), host(unm1)
    its, res, status = Bt.run(w.dt, 1, w.tol)
    assert np.all(status == 0) and np.all(res <= w.tol)
    for S, u0, e1 in zip(solvers, u0s, E1):
        u, _, st = S.get_state()
        assert st == w.steps
        assert S.energy(u) < e1
        u = host(u)
        assert np.all(np.isfinite(u))
        assert abs(u.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
    dn = _oracle_direction_norm(w, w.steps - 1, un, unm1, host(solvers[1].get_state()[0]))
    assert dn <= 2 * w.tol, dn


def test_3d_batched_launch_matches_member_after_member(torch, lib, monkeypatch):
    """Two 3D members fill the device on their own, so pagd_batch_run runs
    them member after member through the single-instance kernel; forced into
    one batched launch (PAGD_BATCH_SEQ=0) they take the same steps."""
    import dataclasses
    w = dataclasses.replace(I.PFC3D256, n=(64,) * 3, L=tuple(l / 4 for l in I.PFC3D256.L))
    outs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_BATCH_SEQ", mode)
        sols = []
        for seed in w.seeds:
            S = pagd.solver_for(w, lib=lib)
            S.set_state(dev(torch, w.u0(seed)))
            sols.append(S)
        B = pagd.Batch(sols)
        its, res, status = B.run(w.dt, 6, w.tol)
        assert np.all(status == 0) and np.all(res <= w.tol)
        assert B.launch_info()["sequential"] == (mode == "1")
        outs[mode] = [host(S.get_state()[0]) for S in sols]
    for a, b in zip(outs["0"], outs["1"]):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)
