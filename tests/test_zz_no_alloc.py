"""The allocation-free entry point pagd_step_static.

Runtimes that own the device allocator and forbid the libraries they host to
allocate, and programs that fix their device-memory budget up front, cannot
hand the library a workspace when they need a step.  pagd_step_static runs the
same time step on a static device array built into the library (8 MiB per
GPU, held until the process exits).  Two consecutive steps through it must
match the regular workspace-based path within the tolerance the other GPU
tests use.

This file sorts last so that, if it fails, a run that stops at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

STATIC_WORKSPACE_LIMIT = 8_364_032  # bytes, as stated in include/pagd.h


def _fch(n):
    return (tuple(4 * math.pi for _ in n), (0.1, 0.1, 0.1, 0.0), 1e-3, -0.3)


# model, grid, scheme, precision, tol, rel, (dt1, dt2)
CASES = [
    ("pfc", (64, 64), "mp", "fp64", 1e-10, 1e-12, (0.1, 0.1)),
    ("pfc", (128, 128), "bdf2", "fp64", 1e-10, 1e-12, (0.1, 0.05)),   # largest FP64 2D grid; dt_prev != dt
    ("fch", (128, 128), "bdf2", "fp32_mixed", 1e-8, 1e-6, (1e-3, 1e-3)),
    ("fch", (64, 64), "lbdf2", "fp64", 0.0, 1e-12, (1e-3, 2e-3)),     # IMEX program, variable step
    ("fch", (64, 64), "lmp", "fp64", 0.0, 1e-12, (1e-3, 1e-3)),
    ("pfc", (16, 16, 16), "bdf2", "fp32_mixed", 1e-8, 1e-6, (0.5, 0.5)),  # 3D: middle-axis passes
]


def _problem(model, n):
    if model == "pfc":
        L = tuple(8 * math.pi for _ in n)
        return L, (0.25,), 0.1
    L, args, _, mean = _fch(n)
    return L, args, mean


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{'x'.join(map(str, c[1]))}-{c[2]}-{c[3]}")
def test_static_scratch_steps_match_workspace_path(case):
    import torch
    torch.cuda.set_device(0)
    lib = pagd.load()
    model, n, scheme, precision, tol, rel, (dt1, dt2) = case
    L, args, mean = _problem(model, n)
    u0 = torch.from_numpy(I.noisy_field(n, mean, 0.05, 31)).cuda()

    # regular path: workspace from the caller, state kept in the solver
    ref = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    ref.set_state(u0)
    r1 = ref.empty_field()
    r2 = ref.empty_field()
    ref.step(r1, dt1, tol)
    ref.step(r2, dt2, tol)

    # static-scratch path: two calls in a row, the state carried by the caller
    S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    s1 = S.empty_field()
    s2 = S.empty_field()
    it1, res1 = S.step_static(u0, u0, 0, dt1, dt1, tol, s1)
    it2, res2 = S.step_static(s1, u0, 1, dt2, dt1, tol, s2)
    if scheme in ("bdf2", "mp"):
        assert res1 <= tol and res2 <= tol and it1 > 0 and it2 > 0
    for a, b in ((s1, r1), (s2, r2)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b)


@pytest.mark.gpu
def test_static_scratch_chain_conserves_mass():
    """100 FP32-mixed FCH steps, each a separate static call: without the
    running mass correction of pagd_run, the mass still stays within 1e-12."""
    import torch
    torch.cuda.set_device(0)
    lib = pagd.load()
    n = (64, 64)
    L, args, dt, mean = _fch(n)
    S = pagd.Solver("fch", n, L, *args, scheme="bdf2", precision="fp32_mixed", lib=lib)
    u0 = torch.from_numpy(I.noisy_field(n, mean, 0.05, 32)).cuda()
    m0 = S.mass(u0)
    unm1, un = u0.clone(), u0.clone()
    for k in range(100):
        unew = S.empty_field()
        _, res = S.step_static(un, unm1, k, dt, dt, 1e-8, unew)
        assert res <= 1e-8
        unm1, un = un, unew
    assert abs(S.mass(un) - m0) <= 1e-12 * abs(m0)


@pytest.mark.gpu
def test_static_scratch_rejects_grids_beyond_its_size():
    import torch
    torch.cuda.set_device(0)
    lib = pagd.load()
    S = pagd.Solver("fch", (512, 512), (4 * math.pi,) * 2, 0.1, 0.1, 0.1, 0.0, lib=lib)
    u = S.empty_field()
    with pytest.raises(pagd.PagdError) as e:
        S.step_static(u, u, 0, 1e-3, 1e-3, 1e-8, S.empty_field())
    assert e.value.status == 1 and "static scratch" in str(e.value)


def test_stated_static_limit_matches_workspace_sizes():
    """The grids include/pagd.h says fit the static scratch do fit (every 2D grid
    up to 128 x 128 and every 3D grid up to 16^3 in both precisions; FP32-mixed
    also 128 x 256 and 32^3), and the next sizes up do not."""
    lib = pagd.load_emulation()

    def size(model, n, precision):
        if model == "pfc":
            S = pagd.Solver("pfc", n, (10.0,) * len(n), 0.1, precision=precision, lib=lib)
        else:
            S = pagd.Solver("fch", n, (10.0,) * len(n), 0.1, 0.1, 0.1, 0.0, precision=precision, lib=lib)
        return S.ws_bytes

    for model in ("pfc", "fch"):
        for precision in ("fp64", "fp32_mixed"):
            for n in ((8, 8), (64, 128), (128, 128), (8, 8, 8), (16, 16, 16)):
                assert size(model, n, precision) <= STATIC_WORKSPACE_LIMIT, (model, n, precision)
            for n in ((256, 256), (64, 64, 64)):
                assert size(model, n, precision) > STATIC_WORKSPACE_LIMIT, (model, n, precision)
        assert size(model, (128, 256), "fp32_mixed") <= STATIC_WORKSPACE_LIMIT
        assert size(model, (32, 32, 32), "fp32_mixed") <= STATIC_WORKSPACE_LIMIT
        assert size(model, (128, 256), "fp64") > STATIC_WORKSPACE_LIMIT
        assert size(model, (32, 32, 32), "fp64") > STATIC_WORKSPACE_LIMIT


def test_static_scratch_rejects_oversize_grid_on_host():
    """The size check runs before any device work (emulation library)."""
    lib = pagd.load_emulation()
    S = pagd.Solver("pfc", (128, 256), (10.0, 20.0), 0.1, precision="fp64", lib=lib)
    u = S.empty_field()
    with pytest.raises(pagd.PagdError) as e:
        S.step_static(u, u, 0, 0.1, 0.1, 1e-10, S.empty_field())
    assert e.value.status == 1 and "8364032" in str(e.value)


@pytest.mark.parametrize("model,scheme,precision", [("fch", "bdf2", "fp32_mixed"), ("pfc", "lmp", "fp64"),
                                                    ("pfc", "mp", "fp64")])
def test_static_step_matches_workspace_step_in_emulation(model, scheme, precision):
    """The same comparison as the GPU test on the CPU emulation of the kernels:
    the static array's layout (twiddle tables at its head, the workspace after
    them) gives the same steps as a caller's workspace."""
    lib = pagd.load_emulation()
    n = (16, 16)
    L, args, mean = _problem(model, n)
    dt, tol = (1e-3 if model == "fch" else 0.1), (1e-8 if precision == "fp32_mixed" else 1e-10)
    u0 = I.noisy_field(n, mean, 0.05, 33)
    ref = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    ref.set_state(u0)
    r1, r2 = ref.empty_field(), ref.empty_field()
    ref.step(r1, dt, tol)
    ref.step(r2, dt, tol)
    S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    s1, s2 = S.empty_field(), S.empty_field()
    S.set_trace(True)  # no effect on the static path
    S.step_static(u0, u0, 0, dt, dt, tol, s1)
    S.step_static(s1, u0, 1, dt, dt, tol, s2)
    rel = 1e-6 if precision == "fp32_mixed" else 1e-12
    for a, b in ((s1, r1), (s2, r2)):
        assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b)
