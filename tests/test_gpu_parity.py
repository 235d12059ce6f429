"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 configurations 1e-9 relative L2 on u
(the PAGD stopping rule at tol 1e-10 bounds the iterate error well below it);
FP32-mixed configurations 1e-6 relative L2; mass 1e-12 relative in both."""
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


def oproblem(model, n, L, eps, eta1=0.0, eta2=0.0, tau=0.0, scheme="bdf2", **kw):
    return O.Problem(O.PFC if model == "pfc" else O.FCH, tuple(n), tuple(L), eps, eta1, eta2, tau,
                     scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2, "lmp": O.LMP}[scheme],
                     **kw)


# ------------------------------------------------------------------- DFT

@pytest.mark.parametrize("n", [(8, 8), (16, 32), (64, 64), (32, 256), (256, 256), (512, 512),
                               (512, 16)])
def test_dft_matches_oracle(torch, lib, n):
    S = pagd.Solver("pfc", n, (3.0, 5.0), 0.1, lib=lib)
    u = I.noisy_field(n, 0.1, 0.5, 3)
    spec = host(S.fft_r2c(dev(torch, u)))
    ref = O.fft(u.astype(complex))[:, : n[1] // 2 + 1]
    got = spec[..., 0] + 1j * spec[..., 1]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    back = host(S.fft_c2r(dev(torch, spec)))
    assert np.abs(back - u).max() <= 1e-14


@pytest.mark.parametrize("model", ["pfc", "fch"])
def test_energy_and_mass_match_oracle(torch, lib, model):
    n, L = (256, 128), (4 * math.pi, 2 * math.pi)
    args = (0.025,) if model == "pfc" else (0.1, 0.1, 0.2, 0.125)
    S = pagd.Solver(model, n, L, *args, lib=lib)
    P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args)
    u = I.noisy_field(n, -0.2, 0.3, 4)
    assert abs(S.energy(dev(torch, u)) - O.energy(P, u)) <= 1e-11 * abs(O.energy(P, u))
    assert abs(S.mass(dev(torch, u)) - O.mass(P, u)) <= 1e-12 * max(1.0, abs(O.mass(P, u)))


# ------------------------------------------------------ small all-schemes

SMALL = [
    ("pfc", (16, 16), (8 * math.pi,) * 2, (0.25,), 0.5, 0.1),
    ("pfc", (32, 64), (16 * math.pi, 32 * math.pi), (0.25,), 0.5, 0.1),
    ("fch", (16, 16), (2 * math.pi,) * 2, (0.18, 0.0324, 0.0324, 0.0), 0.01, -0.3),
    ("fch", (64, 32), (2 * math.pi, math.pi), (0.18, 0.05, 0.07, 0.1), 0.01, -0.3),
]


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("scheme", ["bdf2", "mp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_implicit_steps_match_oracle(torch, lib, case, scheme, precision):
    model, n, L, args, dt, mean = case
    tol = 1e-10 if precision == "fp64" else 1e-8
    S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    P = oproblem(model, n, L, *args, scheme=scheme)
    u0 = I.noisy_field(n, mean, 0.05, 11)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    its, res = S.run(dt, 5, tol, out)
    ref, oits = O.run(P, u0, dt, 5, tol)
    u = host(out)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    if precision == "fp64":
        assert err <= 1e-12
        assert all(abs(a - b) <= 1 for a, b in zip(its, oits))
    else:
        assert err <= 1e-6
    assert all(res <= tol)
    assert abs(u.mean() - u0.mean()) <= 1e-12 * abs(u0.mean())


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("scheme", ["lbdf2", "lmp"])
def test_imex_steps_match_oracle(torch, lib, case, scheme):
    model, n, L, args, dt, mean = case
    S = pagd.Solver(model, n, L, *args, scheme=scheme, lib=lib)
    P = oproblem(model, n, L, *args, scheme=scheme)
    u0 = I.noisy_field(n, mean, 0.05, 12)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    S.run(dt, 6, 0.0, out)
    ref, _ = O.run(P, u0, dt, 6, 0.0)
    assert np.linalg.norm(host(out) - ref) <= 1e-12 * np.linalg.norm(ref)


# ----------------------------------------------------- workload sizes

def test_pfc64_mp_fp64_full_run(torch, lib):
    """PFC 2D 64x64 on [0, 32 pi]^2, MP, dt = 0.1, 100 steps, FP64, tol 1e-10:
    the whole trajectory against the oracle."""
    w = I.PFC64
    S = pagd.solver_for(w, lib=lib)
    P = oproblem("pfc", w.n, w.L, w.eps, scheme=w.scheme)
    u0 = w.u0(1)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    its, res = S.run(w.dt, w.steps, w.tol, out)
    ref, oits = O.run(P, u0, w.dt, w.steps, w.tol)
    u = host(out)
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)
    assert all(abs(a - b) <= 1 for a, b in zip(its, oits))
    assert abs(O.mass(P, u) - O.mass(P, u0)) <= 1e-12 * abs(O.mass(P, u0))


def test_fch256_mixed_first_steps(torch, lib):
    """FCH 2D 256x256 on [0, 4 pi]^2, BDF2, FP32-mixed, dt = 1e-3, tol 1e-8:
    the first steps against the oracle (2 s of CPU per oracle step)."""
    w = I.FCH256
    S = pagd.solver_for(w, lib=lib)
    P = oproblem("fch", w.n, w.L, w.eps, w.eta1, w.eta2, w.tau, scheme=w.scheme)
    u0 = w.u0(1)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    its, res = S.run(w.dt, 3, w.tol, out)
    ref, oits = O.run(P, u0, w.dt, 3, w.tol)
    u = host(out)
    assert np.linalg.norm(u - ref) <= 1e-6 * np.linalg.norm(ref)
    assert all(res <= w.tol)
    assert abs(O.mass(P, u) - O.mass(P, u0)) <= 1e-12 * abs(O.mass(P, u0))


def test_fch256_fp64_first_steps(torch, lib):
    w = I.FCH256
    S = pagd.solver_for(w, lib=lib, precision="fp64")
    P = oproblem("fch", w.n, w.L, w.eps, w.eta1, w.eta2, w.tau, scheme=w.scheme)
    u0 = w.u0(2)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    its, res = S.run(w.dt, 2, 1e-10, out)
    ref, oits = O.run(P, u0, w.dt, 2, 1e-10)
    assert np.linalg.norm(host(out) - ref) <= 1e-9 * np.linalg.norm(ref)
    assert all(abs(a - b) <= 1 for a, b in zip(its, oits))


def test_fch256_full_run_properties(torch, lib):
    """All 1000 steps of the FCH 256^2 workload: every step converges to the
    tolerance, mass is conserved, and the energy decreases."""
    w = I.FCH256
    S = pagd.solver_for(w, lib=lib)
    P = oproblem("fch", w.n, w.L, w.eps, w.eta1, w.eta2, w.tau, scheme=w.scheme)
    u0 = w.u0(3)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    energies = [S.energy(dev(torch, u0))]
    total = []
    for chunk in range(10):
        its, res = S.run(w.dt, w.steps // 10, w.tol, out)
        total.extend(its)
        assert all(res <= w.tol)
        energies.append(S.energy(out))
    u = host(out)
    assert abs(O.mass(P, u) - O.mass(P, u0)) <= 1e-12 * abs(O.mass(P, u0))
    assert all(np.diff(energies) < 0)
    assert np.isfinite(u).all() and np.abs(u).max() < 2.0
    # the energy of the device field agrees with the oracle's at the end
    assert abs(S.energy(out) - O.energy(P, u)) <= 1e-10 * abs(O.energy(P, u))


def test_max_grid_512(torch, lib):
    """512 x 512 (the largest supported axis) PFC, one MP step, FP64."""
    n, L = (512, 512), (128 * math.pi, 128 * math.pi)
    S = pagd.Solver("pfc", n, L, 0.25, scheme="mp", lib=lib)
    P = oproblem("pfc", n, L, 0.25, scheme="mp")
    u0 = I.noisy_field(n, 0.1, 0.05, 13)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    its, _ = S.run(0.1, 1, 1e-10, out)
    r = O.pagd_step(P, 0, u0, u0, 0.1, 0.1, 1e-10)
    assert np.linalg.norm(host(out) - r.u) <= 1e-12 * np.linalg.norm(r.u)
    assert abs(its[0] - r.iters) <= 1


# ------------------------------------------------------------ edge cases

def test_min_grid_8x8(torch, lib):
    n, L = (8, 8), (2 * math.pi,) * 2
    S = pagd.Solver("fch", n, L, 0.18, 0.0324, 0.0324, 0.0, lib=lib)
    P = oproblem("fch", n, L, 0.18, 0.0324, 0.0324, 0.0)
    u0 = I.noisy_field(n, -0.3, 0.05, 14)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    S.run(0.01, 3, 1e-10, out)
    ref, _ = O.run(P, u0, 0.01, 3, 1e-10)
    assert np.linalg.norm(host(out) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_noconvergence_leaves_state(torch, lib):
    n = (32, 32)
    S = pagd.Solver("fch", n, (2 * math.pi,) * 2, 0.18, 0.0324, 0.0324, 0.0, max_iter=3, lib=lib)
    u0 = I.noisy_field(n, -0.3, 0.05, 15)
    S.set_state(dev(torch, u0))
    out = torch.full(n, 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(pagd.PagdError) as e:
        S.run(0.01, 2, 1e-12, out)
    assert e.value.status == 4
    un, um, st = S.get_state()
    assert st == 0 and np.array_equal(host(un), u0) and np.array_equal(host(um), u0)
    assert bool((out == 7.0).all())


def test_nan_input_reports_enan(torch, lib):
    n = (32, 32)
    u0 = I.noisy_field(n, 0.1, 0.05, 16)
    u0[5, 6] = np.nan
    S = pagd.Solver("pfc", n, (8 * math.pi,) * 2, 0.25, lib=lib)
    S.set_state(dev(torch, u0))
    with pytest.raises(pagd.PagdError) as e:
        S.run(0.1, 1, 1e-10)
    assert e.value.status == 6


def test_nonpositive_preconditioner_reports_eprecond(torch, lib):
    n = (16, 16)
    S = pagd.Solver("pfc", n, (8 * math.pi,) * 2, 1.5, lib=lib)
    S.set_state(torch.zeros(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(pagd.PagdError) as e:
        S.run(100.0, 1, 1e-10)
    assert e.value.status == 5


def test_host_buffer_entry_point_matches_device_path(torch, lib):
    w = I.PFC64
    u0 = w.u0(4)
    S = pagd.solver_for(w, lib=lib)
    u_host, its_h, _ = S.run_host(u0, w.dt, 10, w.tol)
    S2 = pagd.solver_for(w, lib=lib)
    S2.set_state(dev(torch, u0))
    out = S2.empty_field()
    its_d, _ = S2.run(w.dt, 10, w.tol, out)
    # FP64 sums use atomics, so runs agree to rounding, not bit for bit
    assert np.abs(u_host - host(out)).max() <= 1e-13
    assert all(abs(a - b) <= 1 for a, b in zip(its_h, its_d))


def test_step_by_step_equals_run(torch, lib):
    """pagd_step repeated equals one pagd_run (state carried in the solver)."""
    w = I.PFC64
    u0 = w.u0(5)
    S = pagd.solver_for(w, lib=lib)
    S.set_state(dev(torch, u0))
    out = S.empty_field()
    for _ in range(4):
        S.step(out, w.dt, w.tol)
    S2 = pagd.solver_for(w, lib=lib)
    S2.set_state(dev(torch, u0))
    out2 = S2.empty_field()
    S2.run(w.dt, 4, w.tol, out2)
    assert np.abs(host(out) - host(out2)).max() <= 1e-13


def test_phase_trace_structure(torch, lib):
    """The phase trace of an FCH 128^2 FP32-mixed run: times increase, every
    step starts with a base evaluation (B C D E, then R1), the step's first
    evaluation is incremental once a reference exists and the last before
    acceptance is exact, and the R1 / RI records equal the reported evaluation
    counts."""
    w = I.FCH256
    S = pagd.solver_for(w, lib=lib, n=(128, 128))
    S.set_state(dev(torch, I.noisy_field((128, 128), -0.3, 0.05, 5)))
    S.run(w.dt, 2, w.tol)
    S.set_trace(True)
    its, res = S.run(w.dt, 6, w.tol)
    names, t = S.get_trace()
    S.set_trace(False)
    assert names[0] == "START" and np.all(np.diff(t) >= 0)
    body = names[1:]
    assert body.count("R1") + body.count("RI") == int(np.sum(its))
    assert body[:4] == ["B/inc", "C/inc", "D/inc", "E/inc"]
    base = [i for i, n in enumerate(body) if n.startswith("B")]
    for i in base:
        tag = body[i][1:]
        assert body[i:i + 5] == ["B" + tag, "C" + tag, "D" + tag, "E" + tag, "R1"]
    # the evaluation before each acceptance (the next step's B or the final
    # ACCEPT) is exact
    accepts = [i for i, n in enumerate(body) if n == "ACCEPT"]
    assert len(accepts) == 1
    exact = [i for i in base if body[i] == "B"]
    assert len(exact) >= 6
