"""Batched launches (pagd_batch_*) on the CPU emulation harness: one
persistent launch advances members of different grids, models, schemes and
parameters, each through its own PAGD iterations (Algorithm 2 per step), and
every member ends where the FP64 oracle does.  The schedule (cost-weighted
contiguous unit ranges per warp) is exercised on several emulated grid sizes so
that members split across CTAs in different ways.  No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

# (model, n, L, eps, eta1, eta2, tau, scheme, dt, mean)
MEMBERS = [
    ("pfc", (16, 16), (8 * math.pi,) * 2, 0.25, 0, 0, 0, "mp", 0.5, 0.1),
    ("fch", (32, 16), (2 * math.pi, math.pi), 0.18, 0.05, 0.07, 0.1, "mp", 0.01, -0.3),
    ("pfc", (16, 32), (8 * math.pi, 16 * math.pi), 0.25, 0, 0, 0, "bdf2", 0.5, 0.1),
    ("fch", (16, 16), (2 * math.pi,) * 2, 0.18, 0.0324, 0.0324, 0, "bdf2", 0.01, -0.3),
    # a square 128 grid runs the fixed-length passes inside the batched kernel
    ("pfc", (128, 128), (32 * math.pi,) * 2, 0.1, 0, 0, 0, "mp", 0.1, 0.07),
]


@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


def _solver(emu, m, precision="fp64", **kw):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = m
    return pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=precision, lib=emu, **kw)


def _oracle(m, u0, nsteps, tol):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = m
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, e1, e2, tau,
                  scheme={"bdf2": O.BDF2, "mp": O.MP}[scheme])
    return O.run(P, u0, dt, nsteps, tol)


def _u0(m, seed):
    return I.noisy_field(m[1], m[9], 0.05, seed)


@pytest.mark.parametrize("sms", ["1", "3", "8"])
def test_batch_fp64_members_match_oracle(emu, monkeypatch, sms):
    """All members share one dt per batch, so this batch uses the members
    that share dt = 0.5 / 0.01 in two batches."""
    monkeypatch.setenv("PAGD_EMU_SMS", sms)
    for group in ([MEMBERS[0], MEMBERS[2]], [MEMBERS[1], MEMBERS[3]]):
        solvers = [_solver(emu, m) for m in group]
        u0s = [_u0(m, 30 + i) for i, m in enumerate(group)]
        for S, u0 in zip(solvers, u0s):
            S.set_state(u0)
        Bt = pagd.Batch(solvers)
        its, res, status = Bt.run(group[0][8], 3, 1e-10)
        assert list(status) == [0] * len(group)
        for i, (m, S, u0) in enumerate(zip(group, solvers, u0s)):
            ref, oits = _oracle(m, u0, 3, 1e-10)
            un, _, st = S.get_state()
            assert st == 3
            assert np.linalg.norm(un - ref) <= 1e-12 * np.linalg.norm(ref)
            assert list(its[i]) == list(oits)
            assert all(res[i] <= 1e-10)


def test_batch_mixed_sizes_and_precision(emu, monkeypatch):
    """FP32-mixed batch of a 128^2 fixed-length member and two small runtime-
    length members: within 1e-6 of the FP64 oracle, mass kept to 1e-12."""
    monkeypatch.setenv("PAGD_EMU_SMS", "5")
    group = [MEMBERS[4], ("pfc", (32, 32), (16 * math.pi,) * 2, 0.2, 0, 0, 0, "mp", 0.1, 0.1),
             ("pfc", (16, 64), (8 * math.pi, 32 * math.pi), 0.05, 0, 0, 0, "mp", 0.1, 0.15)]
    solvers = [_solver(emu, m, "fp32_mixed") for m in group]
    u0s = [_u0(m, 40 + i) for i, m in enumerate(group)]
    for S, u0 in zip(solvers, u0s):
        S.set_state(u0)
    its, res, status = pagd.Batch(solvers).run(0.1, 3, 1e-8)
    assert list(status) == [0, 0, 0]
    for i, (m, S, u0) in enumerate(zip(group, solvers, u0s)):
        ref, _ = _oracle(m, u0, 3, 1e-8)
        un, _, _ = S.get_state()
        assert np.linalg.norm(un - ref) <= 1e-6 * np.linalg.norm(ref)
        assert abs(un.mean() - u0.mean()) <= 1e-12 * abs(u0.mean())
        assert all(res[i] <= 1e-8)


def test_batch_equals_separate_runs(emu, monkeypatch):
    """A member advanced in a batch ends where the same solver run alone ends
    (same arithmetic; only the order of the grid sums differs)."""
    monkeypatch.setenv("PAGD_EMU_SMS", "4")
    m = MEMBERS[3]
    u0 = _u0(m, 50)
    alone = _solver(emu, m, "fp32_mixed")
    alone.set_state(u0)
    ref_its, _ = alone.run(m[8], 4, 1e-8)
    ref = alone.get_state()[0]
    a, b = _solver(emu, m, "fp32_mixed"), _solver(emu, MEMBERS[1], "fp32_mixed")
    a.set_state(u0)
    b.set_state(_u0(MEMBERS[1], 51))
    its, _, _ = pagd.Batch([a, b]).run(m[8], 4, 1e-8)
    assert np.linalg.norm(a.get_state()[0] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert list(its[0]) == list(ref_its)


def test_batch_member_failure_is_isolated(emu):
    """A member that hits its iteration cap stops with PAGD_ENOCONV and keeps
    its state; the other members finish their steps."""
    good, bad = MEMBERS[3], MEMBERS[3]
    sg = _solver(emu, good)
    sb = _solver(emu, bad, max_iter=3)
    u0g, u0b = _u0(good, 60), _u0(bad, 61)
    sg.set_state(u0g)
    sb.set_state(u0b)
    Bt = pagd.Batch([sb, sg])
    with pytest.raises(pagd.PagdError) as e:
        Bt.run(0.01, 2, 1e-12)
    assert e.value.status == 4
    its, res, status = Bt.run(0.01, 2, 1e-10, check=False)
    # the failed member failed again at its first step; the good one advanced 2 more
    assert status[0] == 4 and status[1] == 0
    un, um, st = sb.get_state()
    assert st == 0 and np.array_equal(un, u0b)
    assert sg.get_state()[2] == 4 and all(its[1] > 0) and all(res[1] <= 1e-10)


def test_batch_rejects_bad_membership(emu):
    a = _solver(emu, MEMBERS[0])
    b = _solver(emu, MEMBERS[0], "fp32_mixed")
    with pytest.raises(pagd.PagdError) as e:
        pagd.Batch([a, b])  # one precision per batch
    assert e.value.status == 1
    with pytest.raises(pagd.PagdError) as e:
        pagd.Batch([a, a])
    assert e.value.status == 1
    Bt = pagd.Batch([a])
    with pytest.raises(pagd.PagdError) as e:
        Bt.run(0.1, 1, 1e-8)  # no state set
    assert e.value.status == 7


def test_launch_shape_changes_the_schedule_not_the_results():
    """pagd_batch_set_shape (the autotuner's knob) retiles the global phases
    over other warp and CTA counts; the members' steps agree with the default
    shape up to the summation order of the reductions."""
    lib = pagd.load_emulation()
    ws = [("pfc", (16, 16), (8 * math.pi,) * 2, (0.25,), "mp"), ("fch", (32, 16), (2 * math.pi, math.pi),
          (0.18, 0.05, 0.07, 0.1), "bdf2"), ("pfc", (32, 32), (16 * math.pi,) * 2, (0.25,), "bdf2")]
    outs = []
    for shape in (None, (1, 2), (2, 4)):
        sols = []
        for k, (model, n, L, args, scheme) in enumerate(ws):
            S = pagd.Solver(model, n, L, *args, scheme=scheme, precision="fp32_mixed", lib=lib)
            S.set_state(I.noisy_field(n, 0.1 if model == "pfc" else -0.3, 0.05, 60 + k))
            sols.append(S)
        B = pagd.Batch(sols)
        if shape:
            assert B.set_shape(*shape)
            info = B.launch_info()
            assert info["warps_per_cta"] == shape[0]
        B.run(0.05 if ws[0][0] == "pfc" else 1e-3, 3, 1e-8)
        outs.append([S.get_state()[0].copy() for S in sols])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)
    assert not pagd.Batch(sols).set_shape(9, 1)
