"""The PFC FP32 iteration passes with their inputs staged in shared memory by
asynchronous copies (row_pass_staged / col_pass_staged) against the
register-staged passes they replace (PAGD_STAGED=0): the same arithmetic, so
the same states bit for bit and the same evaluation counts, in the emulation
harness (one thread per CTA).  Also which plans select them.  No GPU."""
import math

import numpy as np
import pytest

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd


@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


def _run(emu, monkeypatch, staged, n, scheme, dt, steps, seed):
    monkeypatch.setenv("PAGD_STAGED", "1" if staged else "0")
    S = pagd.Solver("pfc", n, (n[0] * math.pi / 4,) * 2, 0.25, scheme=scheme, precision="fp32_mixed", lib=emu)
    assert S.launch_info()["staged"] == staged
    u0 = I.noisy_field(n, 0.1, 0.05, seed)
    S.set_state(u0)
    out = S.empty_field()
    its, res = S.run(dt, steps, 1e-8, out)
    return out, list(its), res


@pytest.mark.parametrize("n,scheme", [((64, 64), "bdf2"), ((64, 64), "mp"), ((128, 128), "mp")])
def test_staged_passes_match_register_staged_bitwise(emu, monkeypatch, n, scheme):
    a, ia, ra = _run(emu, monkeypatch, True, n, scheme, 0.1, 3, 21)
    b, ib, rb = _run(emu, monkeypatch, False, n, scheme, 0.1, 3, 21)
    assert ia == ib
    assert np.array_equal(a, b)
    assert np.array_equal(ra, rb)
    assert all(ra <= 1e-8)


def test_staging_selection(emu, monkeypatch):
    monkeypatch.delenv("PAGD_STAGED", raising=False)
    # PFC FP32-mixed on a square power-of-two grid: staged
    S = pagd.Solver("pfc", (64, 64), (16 * math.pi,) * 2, 0.25, precision="fp32_mixed", lib=emu)
    assert S.launch_info()["staged"]
    # FCH FP32-mixed too (one staging slot)
    S = pagd.Solver("fch", (64, 64), (16 * math.pi,) * 2, 0.1, 0.1, 0.1, 0.0, precision="fp32_mixed", lib=emu)
    assert S.launch_info()["staged"]
    # FP64 iterations and runtime line lengths keep the register-staged passes
    for kw in (dict(model="pfc", n=(64, 64), precision="fp64"),
               dict(model="fch", n=(64, 64), precision="fp64"),
               dict(model="pfc", n=(16, 32), precision="fp32_mixed")):
        args = (0.25,) if kw["model"] == "pfc" else (0.1, 0.1, 0.1, 0.0)
        S = pagd.Solver(kw["model"], kw["n"], (16 * math.pi,) * 2, *args, precision=kw["precision"], lib=emu)
        assert not S.launch_info()["staged"], kw


def test_staged_batch_matches_register_staged_bitwise(emu, monkeypatch):
    def run(staged):
        monkeypatch.setenv("PAGD_STAGED", "1" if staged else "0")
        sols = []
        for i, N in enumerate((64, 128, 64)):
            S = pagd.Solver("pfc", (N, N), (N * math.pi / 4,) * 2, 0.1 + 0.05 * i, scheme="mp",
                            precision="fp32_mixed", lib=emu)
            S.set_state(I.noisy_field((N, N), 0.1, 0.05, 30 + i))
            sols.append(S)
        B = pagd.Batch(sols)
        assert B.launch_info()["staged_members"] == (3 if staged else 0)
        its, res, status = B.run(0.1, 2, 1e-8)
        return [S.get_state()[0].copy() for S in sols], its, status

    a, ia, sa = run(True)
    b, ib, sb = run(False)
    assert np.array_equal(ia, ib) and np.array_equal(sa, sb)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_pass_probe_keeps_the_state(emu):
    """The pass probe (one iteration pass repeated in one launch) rejects what
    it cannot run and leaves u^n, u^{n-1} and the step count alone: the run
    after it takes the same steps as a run without it."""
    n = (64, 64)

    def solver():
        S = pagd.Solver("pfc", n, (16 * math.pi,) * 2, 0.25, scheme="bdf2", precision="fp32_mixed", lib=emu)
        S.set_state(I.noisy_field(n, 0.1, 0.05, 41))
        return S

    S = solver()
    with pytest.raises(pagd.PagdError) as e:
        S.pass_probe("RI", 4)  # no completed step yet
    assert e.value.status == 7
    S.run(0.1, 2, 1e-8)
    with pytest.raises(pagd.PagdError) as e:
        S.pass_probe("MF", 4)  # 2D has no middle pass
    assert e.value.status == 1
    for p in ("RI", "CI"):
        S.pass_probe(p, 3)
    u1, _, step = S.get_state()
    assert step == 2
    out_a = S.empty_field()
    its_a, _ = S.run(0.1, 2, 1e-8, out_a)
    R = solver()
    R.run(0.1, 2, 1e-8)
    out_b = R.empty_field()
    its_b, _ = R.run(0.1, 2, 1e-8, out_b)
    assert list(its_a) == list(its_b)
    assert np.array_equal(out_a, out_b)


def test_staged_3d_cubic_matches_register_staged_bitwise(emu, monkeypatch):
    """A cubic 64^3 FP32-mixed grid: the staged row, column and middle passes
    (mid_pass_staged) give the register-staged passes' states bit for bit; a
    non-cubic 3D grid stages its row and column passes only."""
    n, L = (64, 64, 64), (16 * math.pi,) * 3
    u0 = I.noisy_field(n, -0.25, 0.05, 6)
    outs = {}
    for staged in (True, False):
        monkeypatch.setenv("PAGD_STAGED", "1" if staged else "0")
        S = pagd.Solver("pfc", n, L, 0.3, scheme="bdf2", precision="fp32_mixed", lib=emu)
        assert S.launch_info()["staged"] == staged
        S.set_state(u0)
        out = S.empty_field()
        its, res = S.run(0.5, 2, 1e-8, out)
        assert all(res <= 1e-8)
        outs[staged] = (list(its), out)
        if staged:
            for p in ("RI", "CI", "MF", "MI"):
                S.pass_probe(p, 2)
    assert outs[True][0] == outs[False][0]
    assert np.array_equal(outs[True][1], outs[False][1])
    monkeypatch.delenv("PAGD_STAGED")
    S = pagd.Solver("pfc", (64, 32, 64), (16 * math.pi, 8 * math.pi, 16 * math.pi), 0.3,
                    precision="fp32_mixed", lib=emu)
    assert S.launch_info()["staged"]


@pytest.mark.parametrize("model", ["fch", "pfc"])
def test_cooperative_fp32_passes_match_warp_owned_bitwise(emu, monkeypatch, model):
    """The FP32 iteration passes with CTA-cooperative units (opt-in,
    PAGD_COOP32=1) give the warp-owned passes' states bit for bit in the
    emulation."""
    n = (64, 64)
    if model == "fch":
        args, L, dt, mean = (0.1, 0.1, 0.1, 0.0), (4 * math.pi,) * 2, 0.001, -0.3
    else:
        args, L, dt, mean = (0.25,), (16 * math.pi,) * 2, 0.1, 0.1
    outs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PAGD_COOP32", mode)
        monkeypatch.setenv("PAGD_STAGED", "0")
        S = pagd.Solver(model, n, L, *args, scheme="bdf2", precision="fp32_mixed", lib=emu)
        S.set_state(I.noisy_field(n, mean, 0.05, 51))
        out = S.empty_field()
        its, res = S.run(dt, 3, 1e-8, out)
        assert all(res <= 1e-8)
        outs[mode] = (list(its), out)
    assert outs["1"][0] == outs["0"][0]
    assert np.array_equal(outs["1"][1], outs["0"][1])


@pytest.mark.parametrize("n,scheme", [((64, 64), "bdf2"), ((128, 128), "mp"), ((64, 64, 64), "bdf2")])
def test_staged_fch_matches_register_staged_bitwise(emu, monkeypatch, n, scheme):
    """FCH stages its two-field passes with one slot (and, on a cubic 3D grid,
    its middle passes): the same states bit for bit as the register-staged
    passes."""
    L = (4 * math.pi,) * len(n)
    outs = {}
    for staged in (True, False):
        monkeypatch.setenv("PAGD_STAGED", "1" if staged else "0")
        S = pagd.Solver("fch", n, L, 0.1, 0.05, 0.07, 0.1, scheme=scheme, precision="fp32_mixed", lib=emu)
        assert S.launch_info()["staged"] == staged
        S.set_state(I.noisy_field(n, -0.3, 0.05, 61))
        out = S.empty_field()
        its, res = S.run(0.001, 3, 1e-8, out)
        assert all(res <= 1e-8)
        outs[staged] = (list(its), out)
    assert outs[True][0] == outs[False][0]
    assert np.array_equal(outs[True][1], outs[False][1])
