"""GPU: the PFC FP32 iteration passes with inputs staged in shared memory by
asynchronous copies (row_pass_staged / col_pass_staged) against the
register-staged passes (PAGD_STAGED=0) on the same seeded inputs: single
instances at 128^2, 256^2 and 512^2, a batch of uneven members, and a 3D grid.
The arithmetic is the same up to how the compiler contracts FP32 multiply-adds
in each context (bit-identical in the emulation, tests/test_staged_host.py), so
the evaluation counts agree to one per step and the states to far below the
step tolerance: both are certified accepted iterates of the same steps, whose
FP32 corrections differ at FP32 rounding.  The full-run tests check both
against the oracle's reference trajectories at full length."""
import dataclasses

import numpy as np
import pytest

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


# FP32 rounding of the corrections (|delta| ~ 1e-3 |u|) over tens of steps
REL = 1e-8


def _counts_agree(a, b):
    return len(a) == len(b) and all(abs(int(x) - int(y)) <= 1 for x, y in zip(np.ravel(a), np.ravel(b)))


def _member(N, i):
    w = I.PFC_BATCH96.members[{128: 0, 256: 32, 512: 64}[N] + i]
    return w


@pytest.mark.parametrize("N", [128, 256, 512])
def test_staged_single_instance_matches_register_staged(torch, lib, monkeypatch, N):
    w = _member(N, 1)
    runs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_STAGED", mode)
        S = pagd.solver_for(w, lib=lib)
        assert S.launch_info()["staged"] == (mode == "1")
        S.set_state(dev(torch, w.u0(w.seeds[0])))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        its, res = S.run(w.dt, 20, w.tol, out)
        assert np.all(res <= w.tol)
        runs[mode] = (list(its), host(out))
    assert _counts_agree(runs["1"][0], runs["0"][0])
    a, b = runs["1"][1], runs["0"][1]
    assert np.linalg.norm(a - b) <= REL * np.linalg.norm(b)


def test_staged_batch_matches_register_staged(torch, lib, monkeypatch):
    members = [_member(N, i) for N in (128, 256, 512) for i in range(3)]
    runs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_STAGED", mode)
        sols = []
        for w in members:
            S = pagd.solver_for(w, lib=lib)
            S.set_state(dev(torch, w.u0(w.seeds[0])))
            sols.append(S)
        B = pagd.Batch(sols)
        assert B.launch_info()["staged_members"] == (len(members) if mode == "1" else 0)
        its, res, status = B.run(0.1, 10, 1e-8)
        assert np.all(status == 0) and np.all(res <= 1e-8)
        runs[mode] = (its, [host(S.get_state()[0]) for S in sols])
    assert _counts_agree(runs["1"][0], runs["0"][0])
    for a, b in zip(runs["1"][1], runs["0"][1]):
        assert np.linalg.norm(a - b) <= REL * np.linalg.norm(b)


def test_staged_3d_matches_register_staged(torch, lib, monkeypatch):
    w = dataclasses.replace(I.PFC3D256, n=(64,) * 3, L=tuple(l / 4 for l in I.PFC3D256.L))
    runs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_STAGED", mode)
        S = pagd.solver_for(w, lib=lib)
        assert S.launch_info()["staged"] == (mode == "1")
        S.set_state(dev(torch, w.u0(w.seeds[0])))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        its, res = S.run(w.dt, 8, w.tol, out)
        assert np.all(res <= w.tol)
        runs[mode] = (list(its), host(out))
    assert _counts_agree(runs["1"][0], runs["0"][0])
    a, b = runs["1"][1], runs["0"][1]
    assert np.linalg.norm(a - b) <= REL * np.linalg.norm(b)


def test_cooperative_fp32_passes_match_warp_owned(torch, lib, monkeypatch):
    """FCH 256^2 with the opt-in CTA-cooperative FP32 iteration passes
    (PAGD_COOP32=1) against the warp-owned passes (0) on the same input, and
    both against the oracle's reference trajectory at step 25."""
    import json
    import os
    w = I.FCH256
    runs = {}
    monkeypatch.setenv("PAGD_STAGED", "0")  # the cooperative passes replace the register-staged ones
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_COOP32", mode)
        S = pagd.solver_for(w, lib=lib)
        S.set_state(dev(torch, w.u0(1)))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        its, res = S.run(w.dt, 25, w.tol, out)
        assert np.all(res <= w.tol)
        runs[mode] = (list(its), host(out))
    assert _counts_agree(runs["1"][0], runs["0"][0])
    a, b = runs["1"][1], runs["0"][1]
    assert np.linalg.norm(a - b) <= REL * np.linalg.norm(b)
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_fch2d_256_bdf2_fp32mixed.json")))
    st = ref["states"]["25"]
    for u in (a, b):
        est = I.sketch_rel_l2(I.sketch(u, ref["sketch"]["count"], ref["sketch"]["seed"]), st["sketch"], st["sumsq"])
        # within the oracle's own tolerance floor at this step (twice, for the sketch's spread)
        assert est <= 2 * ref["tol_floor"]["rel_l2"]["25"], est


@pytest.mark.parametrize("name", ["fch2d_256_bdf2_fp32mixed", "fch2d_512_bdf2_fp32mixed"])
def test_staged_fch_matches_register_staged(torch, lib, monkeypatch, name):
    """FCH's staged passes (two fields, one staging slot) against its
    register-staged passes on the same input, 20 steps."""
    w = I.WORKLOADS[name]
    runs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_STAGED", mode)
        S = pagd.solver_for(w, lib=lib)
        assert S.launch_info()["staged"] == (mode == "1")
        S.set_state(dev(torch, w.u0(1)))
        out = torch.empty(w.n, dtype=torch.float64, device="cuda")
        its, res = S.run(w.dt, 20, w.tol, out)
        assert np.all(res <= w.tol)
        runs[mode] = (list(its), host(out))
    assert _counts_agree(runs["1"][0], runs["0"][0])
    a, b = runs["1"][1], runs["0"][1]
    assert np.linalg.norm(a - b) <= REL * np.linalg.norm(b)
