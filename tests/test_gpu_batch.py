"""GPU parity of batched launches (pagd_batch_*): members of uneven grids and
parameters advanced by one persistent launch end where the FP64 oracle ends
(1e-9 relative L2 for FP64 members, 1e-6 for FP32-mixed), take the oracle's
iteration counts in FP64, and keep their mass to 1e-12 relative.  The full
96-member PFC batch (32 each at 128^2, 256^2, 512^2) is checked on sampled
members against the oracle and on properties over its 500 steps."""
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


def _oracle(w, u0, nsteps, tol):
    P = O.Problem(O.PFC if w.model == "pfc" else O.FCH, w.n, w.L, w.eps, w.eta1, w.eta2, w.tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[w.scheme])
    return O.run(P, u0, w.dt, nsteps, tol)


def _members(torch, lib, ws, precision=None):
    solvers, u0s = [], []
    for w in ws:
        S = pagd.solver_for(w, lib=lib, **({"precision": precision} if precision else {}))
        u0 = w.u0(w.seeds[0])
        S.set_state(dev(torch, u0))
        solvers.append(S)
        u0s.append(u0)
    return solvers, u0s


DT = 0.003  # one dt for the whole batch; the FCH member needs a small one


def _mixed_group():
    W = I.Workload
    return [
        W("a", "pfc", (64, 64), (16 * math.pi,) * 2, eps=0.2, scheme="mp", dt=DT, mean=0.1, seeds=(11,)),
        W("b", "pfc", (128, 128), (32 * math.pi,) * 2, eps=0.05, scheme="mp", dt=DT, mean=0.12, seeds=(12,)),
        W("c", "pfc", (256, 256), (64 * math.pi,) * 2, eps=0.25, scheme="mp", dt=DT, mean=0.08, seeds=(13,)),
        W("d", "pfc", (32, 128), (8 * math.pi, 32 * math.pi), eps=0.1, scheme="bdf2", dt=DT, mean=0.15,
          seeds=(14,)),
        W("e", "fch", (128, 128), (4 * math.pi,) * 2, eps=0.1, eta1=0.1, eta2=0.1, scheme="bdf2", dt=DT,
          mean=-0.3, seeds=(15,)),
    ]


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-10, 1e-9), ("fp32_mixed", 1e-8, 1e-6)])
def test_batch_of_uneven_members_matches_oracle(torch, lib, precision, tol, bound):
    group = _mixed_group()
    solvers, u0s = _members(torch, lib, group, precision)
    its, res, status = pagd.Batch(solvers).run(DT, 3, tol)
    assert list(status) == [0] * len(group)
    for i, (w, S, u0) in enumerate(zip(group, solvers, u0s)):
        ref, oits = _oracle(w, u0, 3, tol)
        un, _, st = S.get_state()
        un = host(un)
        assert st == 3
        assert np.linalg.norm(un - ref) <= bound * np.linalg.norm(ref), w.name
        assert abs(un.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
        assert np.all(res[i] <= tol)
        if precision == "fp64":
            assert list(its[i]) == list(oits), w.name


def test_batch_equals_single_instance_runs(torch, lib):
    group = _mixed_group()[:4]
    solvers, u0s = _members(torch, lib, group, "fp64")
    its_b, _, _ = pagd.Batch(solvers).run(DT, 4, 1e-10)
    for i, (w, S, u0) in enumerate(zip(group, solvers, u0s)):
        alone = pagd.solver_for(w, lib=lib, precision="fp64")
        alone.set_state(dev(torch, u0))
        its, _ = alone.run(DT, 4, 1e-10)
        a, b = host(alone.get_state()[0]), host(S.get_state()[0])
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
        assert list(its) == list(its_b[i])


@pytest.fixture(scope="module")
def batch96(torch, lib):
    bw = I.PFC_BATCH96
    solvers, u0s = _members(torch, lib, bw.members)
    return bw, solvers, u0s, pagd.Batch(solvers)


def test_batch96_sampled_members_match_oracle(torch, batch96):
    """Two steps of the full batch; one member per grid size against the oracle."""
    bw, solvers, u0s, Bt = batch96
    its, res, status = Bt.run(bw.dt, 2, bw.tol)
    assert np.all(status == 0)
    assert np.all(res <= bw.tol) and np.all(its > 0)
    for i in (0, 32 + 7, 64 + 31):
        w = bw.members[i]
        ref, _ = _oracle(w, u0s[i], 2, bw.tol)
        un = host(solvers[i].get_state()[0])
        assert np.linalg.norm(un - ref) <= 1e-6 * np.linalg.norm(ref), w.name


def test_batch96_full_run_properties(torch, batch96):
    """The remaining 498 steps: every member converges at every step, stays
    finite and keeps its mass."""
    bw, solvers, u0s, Bt = batch96
    its, res, status = Bt.run(bw.dt, bw.steps - 2, bw.tol)
    assert np.all(status == 0)
    assert np.all(res <= bw.tol)
    assert its.max() < 1000
    for S, u0 in zip(solvers, u0s):
        un, _, st = S.get_state()
        un = host(un)
        assert st == bw.steps
        assert np.all(np.isfinite(un))
        assert abs(un.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())


def test_launch_shapes_agree_and_autotuner_keeps_the_fastest(torch, lib):
    """The autotuner's knob (warps per CTA x CTAs per SM) retiles the global
    phases; every shape gives the same steps up to the summation order, and
    tune_batch keeps the shape it timed fastest and restores the states."""
    from paper_2204_07247_gb300 import autotune
    ms = [m for m in I.PFC_BATCH96.members[::16]]
    sols, u0s = [], []
    for m in ms:
        S = pagd.solver_for(m, lib=lib)
        u0s.append(dev(torch, m.u0(m.seeds[0])))
        S.set_state(u0s[-1])
        sols.append(S)
    B = pagd.Batch(sols)
    rep = autotune.tune_batch(torch, B, u0s, 0.1, 1e-8, steps=1)
    assert len(rep["candidates"]) >= 2
    best = min(rep["candidates"], key=lambda r: r["ms_per_step"])
    assert rep["chosen"]["warps_per_cta"] == best["warps_per_cta"]
    assert all(S.get_state()[2] == 0 for S in sols)  # states restored
    B.run(0.1, 3, 1e-8)
    ref = [host(S.get_state()[0]) for S in sols]
    assert not B.set_shape(1, 8)  # eight 512^2 slices do not fit one SM
    for w, c in ((2, 1), (1, 2)):
        assert B.set_shape(w, c)
        for S, u0 in zip(sols, u0s):
            S.set_state(u0)
        _, res, status = B.run(0.1, 3, 1e-8)
        assert np.all(status == 0) and np.all(res <= 1e-8)
        for S, r in zip(sols, ref):
            assert np.linalg.norm(host(S.get_state()[0]) - r) <= 1e-6 * np.linalg.norm(r)


def test_batch_step_with_guess_matches_single_members(torch, lib):
    """pagd_batch_step_with_guess: each member of one launch takes the step it
    takes alone through pagd_step_with_guess (a good guess kept, a poor one
    abandoned for the extrapolation, no guess: the plain step)."""
    w = I.FCH256
    P = O.Problem(O.FCH, w.n, w.L, w.eps, w.eta1, w.eta2, w.tau, scheme=O.BDF2)
    u0s = [w.u0(80 + k) for k in range(3)]
    guesses = []
    for k, u0 in enumerate(u0s):
        u1 = O.pagd_step(P, 0, u0, u0, w.dt, w.dt, 1e-12).u
        tight = O.pagd_step(P, 1, u1, u0, w.dt, w.dt, 1e-12).u
        guesses.append([dev(torch, tight + 1e-8 * I.noisy_field(w.n, 0.0, 1.0, 9)),
                        dev(torch, I.noisy_field(w.n, w.mean, 0.3, 11)), None][k])

    def fresh():
        out = []
        for u0 in u0s:
            S = pagd.solver_for(w, lib=lib)
            S.set_state(dev(torch, u0))
            S.step(S.empty_field(), w.dt, w.tol)  # the record
            out.append(S)
        return out

    ref = []
    for S, g in zip(fresh(), guesses):
        o = S.empty_field()
        if g is None:
            S.step(o, w.dt, w.tol)
            used = False
        else:
            _, _, used = S.step_with_guess(o, g, w.dt, w.tol)
        ref.append((host(o), used))
    sols = fresh()
    B = pagd.Batch(sols)
    its, res, status, used = B.step_with_guess(guesses, w.dt, w.tol)
    assert np.all(status == 0) and np.all(res <= w.tol)
    assert list(used) == [True, False, False]
    for S, (o, u) in zip(sols, ref):
        un = host(S.get_state()[0])
        assert np.linalg.norm(un - o) <= 1e-6 * np.linalg.norm(o)
