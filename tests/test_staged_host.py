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
    # FP64 iterations, FCH, and runtime line lengths keep the register-staged passes
    for kw in (dict(model="pfc", n=(64, 64), precision="fp64"),
               dict(model="fch", n=(64, 64), precision="fp32_mixed"),
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
