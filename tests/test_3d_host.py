"""Three-dimensional grids on the CPU emulation harness: the row passes
transform the last axis, a middle pass the middle axis (writing the spectrum
transposed so the column passes see contiguous lines of the first axis), and
every program (DFT, energy, PAGD steps, IMEX) agrees with the FP64 oracle.
No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd


@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


@pytest.mark.parametrize("n", [(8, 8, 8), (16, 8, 32), (8, 32, 16)])
def test_emulated_3d_dft_energy_mass(emu, n):
    L = (3.0, 5.0, 4.0)
    u = I.noisy_field(n, 0.1, 0.5, 3)
    S = pagd.Solver("pfc", n, L, 0.1, lib=emu)
    spec = S.fft_r2c(u)
    ref = O.fft(u.astype(complex))[..., : n[-1] // 2 + 1]
    assert np.abs(spec[..., 0] + 1j * spec[..., 1] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(S.fft_c2r(spec) - u).max() <= 1e-14
    for model, args in (("pfc", (0.1,)), ("fch", (0.1, 0.1, 0.2, 0.125))):
        S = pagd.Solver(model, n, L, *args, lib=emu)
        P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args)
        assert abs(S.energy(u) - O.energy(P, u)) <= 1e-12 * abs(O.energy(P, u))
        assert abs(S.mass(u) - O.mass(P, u)) <= 1e-13 * abs(O.mass(P, u))


CASES3 = [
    ("pfc", (8, 8, 8), (8 * math.pi,) * 3, 0.3, 0, 0, 0, "bdf2", 0.5, -0.25),
    ("pfc", (16, 8, 16), (16 * math.pi, 8 * math.pi, 16 * math.pi), 0.3, 0, 0, 0, "mp", 0.5, -0.25),
    ("fch", (8, 16, 8), (2 * math.pi, 4 * math.pi, 2 * math.pi), 0.18, 0.05, 0.07, 0.1, "bdf2", 0.01, -0.3),
]


@pytest.mark.parametrize("case", CASES3)
@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-12), ("fp32_mixed", 1e-8, 1e-6)])
def test_emulated_3d_steps_match_oracle(emu, case, precision, tol, bound):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=precision, lib=emu)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    u0 = I.noisy_field(n, mean, 0.1, 7)
    S.set_state(u0)
    out = S.empty_field()
    its, res = S.run(dt, 3, tol, out)
    ref, oits = O.run(P, u0, dt, 3, tol)
    assert np.linalg.norm(out - ref) <= bound * np.linalg.norm(ref)
    assert all(res <= tol)
    assert abs(out.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
    if precision == "fp64":
        assert list(its) == list(oits)


@pytest.mark.parametrize("case", CASES3)
@pytest.mark.parametrize("scheme", ["lbdf2", "lmp"])
def test_emulated_3d_imex_matches_oracle(emu, case, scheme):
    model, n, L, eps, e1, e2, tau, _, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, lib=emu)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"lbdf2": O.LBDF2, "lmp": O.LMP}[scheme])
    u0 = I.noisy_field(n, mean, 0.1, 9)
    S.set_state(u0)
    out = S.empty_field()
    S.run(dt, 3, 0.0, out)
    ref, _ = O.run(P, u0, dt, 3, 0.0)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_emulated_3d_batch_with_2d_members(emu, monkeypatch):
    """A batch mixing 3D and 2D members: the middle passes of the 3D members
    share global phases with the 2D members' row and column passes."""
    monkeypatch.setenv("PAGD_EMU_SMS", "3")
    cases = [CASES3[0], ("pfc", (16, 16), (8 * math.pi,) * 2, 0.25, 0, 0, 0, "bdf2", 0.5, 0.1),
             CASES3[1]]
    solvers, u0s = [], []
    for i, (model, n, L, eps, e1, e2, tau, scheme, dt, mean) in enumerate(cases):
        S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision="fp32_mixed", lib=emu)
        u0 = I.noisy_field(n, mean, 0.1, 20 + i)
        S.set_state(u0)
        solvers.append(S)
        u0s.append(u0)
    its, res, status = pagd.Batch(solvers).run(0.5, 3, 1e-8)
    assert list(status) == [0, 0, 0]
    for (model, n, L, eps, e1, e2, tau, scheme, dt, mean), S, u0 in zip(cases, solvers, u0s):
        P = O.Problem(O.PFC, n, L, eps, scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
        ref, _ = O.run(P, u0, 0.5, 3, 1e-8)
        un = S.get_state()[0]
        assert np.linalg.norm(un - ref) <= 1e-6 * np.linalg.norm(ref)


def test_emulated_3d_cubic_fixed_length_middle_pass(emu):
    """A cubic 64^3 grid runs the middle passes through the fixed-length
    stages (both lines of a unit in lockstep): DFT round trip and two FP64
    steps against the oracle."""
    n, L = (64, 64, 64), (16 * math.pi,) * 3
    u = I.noisy_field(n, -0.25, 0.1, 5)
    S = pagd.Solver("pfc", n, L, 0.3, lib=emu)
    spec = S.fft_r2c(u)
    ref = O.fft(u.astype(complex))[..., : n[-1] // 2 + 1]
    assert np.abs(spec[..., 0] + 1j * spec[..., 1] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(S.fft_c2r(spec) - u).max() <= 1e-14
    P = O.Problem(O.PFC, n, L, 0.3, 0, 0, 0, scheme=O.BDF2)
    S.set_state(u)
    out = S.empty_field()
    its, res = S.run(0.5, 2, 1e-10, out)
    uref, oits = O.run(P, u, 0.5, 2, 1e-10)
    assert np.linalg.norm(out - uref) <= 1e-12 * np.linalg.norm(uref)
    assert list(its) == list(oits)


def test_emulated_fp64_batch_with_cubic_member(emu, monkeypatch):
    """An FP64 batch of a cubic 64^3 member beside a 64^2 member: both match
    the oracle with the oracle's iteration counts."""
    monkeypatch.setenv("PAGD_EMU_SMS", "3")
    cases = [("pfc", (64, 64, 64), (16 * math.pi,) * 3, 0.3, "bdf2", -0.25),
             ("pfc", (64, 64), (32 * math.pi,) * 2, 0.25, "bdf2", 0.1)]
    solvers, u0s = [], []
    for i, (model, n, L, eps, scheme, mean) in enumerate(cases):
        S = pagd.Solver(model, n, L, eps, scheme=scheme, precision="fp64", lib=emu)
        u0 = I.noisy_field(n, mean, 0.1, 30 + i)
        S.set_state(u0)
        solvers.append(S)
        u0s.append(u0)
    its, res, status = pagd.Batch(solvers).run(0.5, 2, 1e-10)
    assert list(status) == [0, 0]
    for (model, n, L, eps, scheme, mean), S, u0, it in zip(cases, solvers, u0s, its):
        P = O.Problem(O.PFC, n, L, eps, scheme=O.BDF2)
        ref, oits = O.run(P, u0, 0.5, 2, 1e-10)
        assert np.linalg.norm(S.get_state()[0] - ref) <= 1e-12 * np.linalg.norm(ref)
        assert list(it) == list(oits)
