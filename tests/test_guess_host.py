"""pagd_step_with_guess on the CPU emulation harness against the FP64 oracle.
The caller's initial iterate is moved to the mass of u^n, the first PAGD
direction (Algorithm 2) is evaluated at it and at the extrapolated guess
(Sec. 3.4.2), and the step continues from the smaller one: with a guess close
to the solution the guess is kept and the result is the oracle's step from
that guess; with a poor guess the step falls back to the extrapolation and is
the oracle's plain step.  The two probe evaluations count in the cost."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

CASES = [
    ("fch", (16, 16), (2 * math.pi,) * 2, 0.18, 0.0324, 0.0324, 0, "bdf2", 0.01, -0.3),
    ("pfc", (16, 32), (8 * math.pi, 16 * math.pi), 0.25, 0, 0, 0, "mp", 0.5, 0.1),
]


@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-12), ("fp32_mixed", 1e-8, 1e-6)])
def test_step_with_guess_matches_oracle(emu, case, precision, tol, bound):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    u0 = I.noisy_field(n, mean, 0.05, 5)
    tight = O.pagd_step(P, 0, u0, u0, dt, dt, 1e-13).u
    good = tight + 1e-6 * I.noisy_field(n, 0.0, 1.0, 9) + 0.3  # off in mass on purpose
    bad = I.noisy_field(n, mean, 0.5, 11)
    for g, expect_used in ((good, True), (bad, False)):
        S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=precision, lib=emu)
        S.set_state(u0)
        out = S.empty_field()
        its, res, used = S.step_with_guess(out, g, dt, tol)
        assert used == expect_used
        ref = O.pagd_step(P, 0, u0, u0, dt, dt, tol, guess=g if used else None)
        assert ref.status == O.OK
        assert np.linalg.norm(out - ref.u) <= bound * np.linalg.norm(ref.u)
        assert res <= tol
        assert abs(out.sum() - u0.sum()) <= 1e-13 * abs(u0.sum())
        if precision == "fp64":
            # the probe at the guess (and, if the guess is kept, the probe at
            # the extrapolation) come on top of the oracle's count
            assert its == ref.iters + (2 if used else 1)
        assert S.get_state()[2] == 1


def test_step_with_guess_rejects_imex(emu):
    S = pagd.Solver("pfc", (16, 16), (8 * math.pi,) * 2, 0.25, scheme="lbdf2", lib=emu)
    u0 = I.noisy_field((16, 16), 0.1, 0.05, 5)
    S.set_state(u0)
    with pytest.raises(pagd.PagdError) as e:
        S.step_with_guess(S.empty_field(), u0, 0.1, 1e-8)
    assert e.value.status == 1


@pytest.mark.parametrize("case", CASES)
def test_step_with_guess_against_the_record(emu, case):
    """After a plain step the solver holds the record R (||d_0||_inf of that
    step from the extrapolation).  A guess with ||d_0||_inf <= R is kept at no
    extra cost: the evaluations equal the oracle's from that guess.  A poor
    guess costs its one probe and the step starts over from the extrapolation."""
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    tol = 1e-10
    u0 = I.noisy_field(n, mean, 0.05, 5)
    u1 = O.pagd_step(P, 0, u0, u0, dt, dt, tol).u
    tight = O.pagd_step(P, 1, u1, u0, dt, dt, 1e-13).u
    good = tight + 1e-7 * I.noisy_field(n, 0.0, 1.0, 9) + 0.3
    bad = I.noisy_field(n, mean, 0.5, 11)
    for g, expect_used in ((good, True), (bad, False)):
        S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision="fp64", lib=emu)
        S.set_state(u0)
        S.step(S.empty_field(), dt, tol)  # the plain step that sets the record
        out = S.empty_field()
        its, res, used = S.step_with_guess(out, g, dt, tol)
        assert used == expect_used
        ref = O.pagd_step(P, 1, u1, u0, dt, dt, tol, guess=g if used else None)
        assert np.linalg.norm(out - ref.u) <= 1e-12 * np.linalg.norm(ref.u)
        assert its == ref.iters + (0 if used else 1), (its, ref.iters)
        assert res <= tol


def test_batch_step_with_guess_matches_single_members(emu):
    """pagd_batch_step_with_guess: every member of one launch takes the step
    pagd_step_with_guess takes alone (a member without a guess takes the plain
    step), including the judging against each member's record."""
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = CASES[0]
    P = O.Problem(O.FCH, n, L, eps, e1, e2, tau, scheme=O.BDF2)
    tol = 1e-10
    u0s = [I.noisy_field(n, mean, 0.05, 70 + k) for k in range(3)]
    guesses = []
    for k, u0 in enumerate(u0s):
        u1 = O.pagd_step(P, 0, u0, u0, dt, dt, tol).u
        tight = O.pagd_step(P, 1, u1, u0, dt, dt, 1e-13).u
        guesses.append([tight + 1e-7 * I.noisy_field(n, 0.0, 1.0, 9), I.noisy_field(n, mean, 0.5, 11), None][k])

    def fresh():
        out = []
        for u0 in u0s:
            S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision="fp64", lib=emu)
            S.set_state(u0)
            S.step(S.empty_field(), dt, tol)  # the record
            out.append(S)
        return out

    alone = fresh()
    ref = []
    for S, g in zip(alone, guesses):
        o = S.empty_field()
        if g is None:
            its, res = S.step(o, dt, tol)
            used = False
        else:
            its, res, used = S.step_with_guess(o, g, dt, tol)
        ref.append((o, its, used))
    sols = fresh()
    B = pagd.Batch(sols)
    its, res, status, used = B.step_with_guess(guesses, dt, tol)
    assert np.all(status == 0) and np.all(res <= tol)
    for S, (o, it, u), k, uu in zip(sols, ref, its, used):
        un = S.get_state()[0]
        assert np.linalg.norm(un - o) <= 1e-12 * np.linalg.norm(o)
        assert k == it and bool(uu) == bool(u)
    assert list(used) == [True, False, False]
