"""Host-side tests of the C ABI: the CUDA library builds and exports every
symbol that include/pagd.h declares, argument validation happens on the host,
and the kernels' index arithmetic and control flow (compiled as host C++ in the
emulation harness, one thread per CTA) agree with the FP64 oracle.  No GPU."""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_07247_gb300 import build as B
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pagd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pagd_status|const char\s*\*|void)\s+(\w+)\s*\(", src,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def cuda_lib():
    try:
        return pagd.load()
    except Exception as e:  # pragma: no cover - nvcc missing
        pytest.fail(f"libpagd.so did not build: {e}")


def test_header_declares_the_binding_names():
    assert set(declared_functions()) == set(pagd.EXPORTS)


def test_cuda_library_exports_every_declared_symbol(cuda_lib):
    for name in declared_functions():
        assert hasattr(cuda_lib, name), name


@pytest.mark.parametrize("bad", [dict(n=(12, 16)), dict(n=(4, 4)), dict(n=(1024, 16)),
                                 dict(L=(0.0, 1.0)), dict(M=0.0), dict(scheme=7),
                                 dict(precision=3), dict(s=0.0), dict(max_iter=0),
                                 dict(eta=(0.5, -1.0))])
def test_init_rejects_bad_arguments(cuda_lib, bad):
    kw = dict(model="pfc", n=(16, 16), L=(1.0, 1.0), eps=0.1)
    kw.update(bad)
    with pytest.raises(pagd.PagdError) as e:
        pagd.Solver(lib=cuda_lib, **kw) if False else _init_only(cuda_lib, **kw)
    assert e.value.status == 1


def _init_only(lib, model, n, L, eps, M=1.0, scheme=0, precision=0, s=0.9, max_iter=1000, eta=None):
    import ctypes
    o = pagd.Opts()
    lib.pagd_default_opts(ctypes.byref(o))
    o.s, o.max_iter = s, max_iter
    if eta is not None:
        o.n_eta = len(eta)
        for j, e in enumerate(eta):
            o.eta[j] = e
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 3)(*(list(n) + [1]))
    LL = (ctypes.c_double * 3)(*(list(L) + [1.0]))
    st = lib.pfc_init(ctypes.byref(h), 2, nn, LL, eps, M, scheme, precision, ctypes.byref(o), None)
    if st != 0:
        raise pagd.PagdError(st, "init")
    lib.pagd_destroy(h)


def test_calls_out_of_order_are_rejected(cuda_lib):
    import ctypes
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 3)(16, 16, 1)
    LL = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert cuda_lib.pfc_init(ctypes.byref(h), 2, nn, LL, 0.1, 1.0, 0, 0, None, None) == 0
    it = ctypes.c_int()
    r = ctypes.c_double()
    # no workspace, no state: ESTATE, nothing launched
    assert cuda_lib.pagd_run(h, None, 0.1, 1, 1e-8, None, None) == 7
    assert cuda_lib.pagd_set_workspace(h, ctypes.c_void_p(8), 1 << 30) == 1  # misaligned
    cuda_lib.pagd_destroy(h)


# ------------------------------------------------------------- emulation

@pytest.fixture(scope="module")
def emu():
    return pagd.load_emulation()


def _oracle_problem(model, n, L, eps, eta1, eta2, tau, scheme):
    return O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, eps, eta1, eta2, tau,
                     scheme={"bdf2": O.BDF2, "mp": O.MP, "lbdf2": O.LBDF2, "lmp": O.LMP}[scheme])


@pytest.mark.parametrize("n", [(8, 8), (16, 32), (64, 16), (64, 64), (128, 128)])
def test_emulated_dft_matches_oracle(emu, n):
    S = pagd.Solver("pfc", n, (3.0, 5.0), 0.1, lib=emu)
    u = I.noisy_field(n, 0.1, 0.5, 3)
    spec = S.fft_r2c(u)
    full = O.fft(u.astype(complex))
    ref = full[:, : n[1] // 2 + 1]
    assert np.abs(spec[..., 0] + 1j * spec[..., 1] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(S.fft_c2r(spec) - u).max() <= 1e-15


CASES = [
    ("pfc", (16, 16), (8 * math.pi,) * 2, 0.25, 0, 0, 0, "mp", 0.5, 0.1),
    # square 64 / 128 grids run the fixed-length passes
    ("pfc", (64, 64), (32 * math.pi,) * 2, 0.25, 0, 0, 0, "bdf2", 0.5, 0.1),
    ("fch", (64, 64), (4 * math.pi,) * 2, 0.1, 0.1, 0.1, 0.0, "bdf2", 0.001, -0.3),
    ("fch", (128, 128), (4 * math.pi,) * 2, 0.1, 0.05, 0.07, 0.1, "mp", 0.001, -0.3),
    ("pfc", (16, 32), (8 * math.pi, 16 * math.pi), 0.25, 0, 0, 0, "bdf2", 0.5, 0.1),
    ("fch", (16, 16), (2 * math.pi,) * 2, 0.18, 0.0324, 0.0324, 0, "bdf2", 0.01, -0.3),
    ("fch", (32, 16), (2 * math.pi, math.pi), 0.18, 0.05, 0.07, 0.1, "mp", 0.01, -0.3),
]


@pytest.mark.parametrize("case", CASES)
def test_emulated_fp64_steps_match_oracle(emu, case):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, lib=emu)
    P = _oracle_problem(model, n, L, eps, e1, e2, tau, scheme)
    u0 = I.noisy_field(n, mean, 0.05, 7)
    S.set_state(u0)
    out = S.empty_field()
    its, res = S.run(dt, 4, 1e-10, out)
    ref, oits = O.run(P, u0, dt, 4, 1e-10)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    assert list(its) == list(oits)
    assert all(res <= 1e-10)


@pytest.mark.parametrize("case", CASES)
def test_emulated_mixed_precision_within_tolerance(emu, case):
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision="fp32_mixed", lib=emu)
    P = _oracle_problem(model, n, L, eps, e1, e2, tau, scheme)
    u0 = I.noisy_field(n, mean, 0.05, 8)
    S.set_state(u0)
    out = S.empty_field()
    its, res = S.run(dt, 4, 1e-8, out)
    ref, _ = O.run(P, u0, dt, 4, 1e-8)
    assert np.linalg.norm(out - ref) <= 1e-6 * np.linalg.norm(ref)
    assert all(res <= 1e-8)
    assert abs(out.mean() - u0.mean()) <= 1e-12 * abs(u0.mean())


@pytest.mark.parametrize("model,scheme", [("pfc", "lbdf2"), ("pfc", "lmp"), ("fch", "lbdf2"),
                                          ("fch", "lmp")])
def test_emulated_imex_matches_oracle(emu, model, scheme):
    if model == "pfc":
        n, L, eps, e1, e2, tau, dt, mean = (16, 16), (8 * math.pi,) * 2, 0.25, 0, 0, 0, 0.5, 0.1
    else:
        n, L, eps, e1, e2, tau, dt, mean = (16, 16), (2 * math.pi,) * 2, 0.18, 0.05, 0.07, 0.1, 0.01, -0.3
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, lib=emu)
    P = _oracle_problem(model, n, L, eps, e1, e2, tau, scheme)
    u0 = I.noisy_field(n, mean, 0.05, 9)
    S.set_state(u0)
    out = S.empty_field()
    S.run(dt, 5, 0.0, out)
    ref, _ = O.run(P, u0, dt, 5, 0.0)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_emulated_energy_and_mass(emu):
    n, L = (16, 32), (3.0, 5.0)
    u = I.noisy_field(n, 0.1, 0.5, 3)
    for model, args in (("pfc", (0.1,)), ("fch", (0.1, 0.1, 0.2, 0.125))):
        S = pagd.Solver(model, n, L, *args, lib=emu)
        P = O.Problem(O.PFC if model == "pfc" else O.FCH, n, L, *args)
        assert abs(S.energy(u) - O.energy(P, u)) <= 1e-12 * abs(O.energy(P, u))
        assert abs(S.mass(u) - O.mass(P, u)) <= 1e-14


def test_emulated_failure_keeps_state(emu):
    """ENOCONV at the iteration cap leaves u^n, u^{n-1} and the step count as
    they were; NaN input gives ENAN."""
    n = (16, 16)
    S = pagd.Solver("fch", n, (2 * math.pi,) * 2, 0.18, 0.0324, 0.0324, 0.0, max_iter=3, lib=emu)
    u0 = I.noisy_field(n, -0.3, 0.05, 10)
    S.set_state(u0)
    out = np.full(n, 7.0)
    with pytest.raises(pagd.PagdError) as e:
        S.run(0.01, 2, 1e-12, out)
    assert e.value.status == 4
    un, um, st = S.get_state()
    assert st == 0 and np.array_equal(un, u0) and np.array_equal(um, u0)
    assert np.all(out == 7.0)
    bad = u0.copy()
    bad[3, 4] = np.nan
    S2 = pagd.Solver("pfc", n, (8 * math.pi,) * 2, 0.25, lib=emu)
    S2.set_state(bad)
    with pytest.raises(pagd.PagdError) as e:
        S2.run(0.1, 1, 1e-10)
    assert e.value.status == 6


def test_emulated_precond_failure(emu):
    """eps > 1 makes 1 - eps < 0; with a huge dt the PFC averaged-Newton symbol
    beta_{-2}/kappa + beta_0 - 2 kappa + kappa^2 dips below zero near kappa = 1."""
    n = (16, 16)
    S = pagd.Solver("pfc", n, (2 * math.pi * 4,) * 2, 1.5, scheme="bdf2", lib=emu)
    S.set_state(np.zeros(n))
    with pytest.raises(pagd.PagdError) as e:
        S.run(100.0, 1, 1e-10)
    assert e.value.status == 5


@pytest.mark.parametrize("case", CASES)
def test_emulated_mixed_precision_costs_few_extra_evaluations(emu, case):
    """FP32 rounding must stay relative to the correction: if it leaked in at
    O(1) (e.g. two fields of very different size packed into one transform) the
    FP32 norm would stall far above tol and force many FP64 rebases."""
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    u0 = I.noisy_field(n, mean, 0.05, 21)
    counts = {}
    for prec in ("fp64", "fp32_mixed"):
        S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=prec, lib=emu)
        S.set_state(u0)
        its, _ = S.run(dt, 3, 1e-8, S.empty_field())
        counts[prec] = its
    assert all(m <= f + 6 for m, f in zip(counts["fp32_mixed"], counts["fp64"])), counts


def test_emulated_mass_error_does_not_accumulate(emu):
    """Removing the mean of an FP32 correction from FP64 points rounds every
    point the same way; the acceptance feeds the exact mass change back, so the
    drift stays at rounding level instead of growing with the step count."""
    n = (64, 64)
    S = pagd.Solver("fch", n, (4 * math.pi,) * 2, 0.1, 0.1, 0.1, 0.0, scheme="bdf2",
                    precision="fp32_mixed", lib=emu)
    u0 = I.noisy_field(n, -0.3, 0.05, 3)
    S.set_state(u0)
    out = S.empty_field()
    m0 = math.fsum(u0.ravel())
    drift = []
    for _ in range(8):
        S.run(1e-3, 25, 1e-8, out)
        drift.append(abs(math.fsum(out.ravel()) - m0) / abs(m0))
    assert max(drift) <= 2e-15, drift


@pytest.mark.parametrize("case", [c for c in CASES if c[1][0] == c[1][1] and c[1][0] >= 64])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_emulated_cooperative_passes_match_oracle(emu, case, precision, monkeypatch):
    """The CTA-cooperative variants of the passes with FP64 lines (chosen for
    grids with fewer units than warps) follow the same arithmetic: the steps
    still match the oracle, and the FP64 steps take the same iteration counts."""
    monkeypatch.setenv("PAGD_COOP", "1")
    model, n, L, eps, e1, e2, tau, scheme, dt, mean = case
    S = pagd.Solver(model, n, L, eps, e1, e2, tau, scheme=scheme, precision=precision, lib=emu)
    P = _oracle_problem(model, n, L, eps, e1, e2, tau, scheme)
    u0 = I.noisy_field(n, mean, 0.05, 11)
    S.set_state(u0)
    out = S.empty_field()
    tol = 1e-10 if precision == "fp64" else 1e-8
    its, res = S.run(dt, 3, tol, out)
    ref, oits = O.run(P, u0, dt, 3, tol)
    bound = 1e-12 if precision == "fp64" else 1e-6
    assert np.linalg.norm(out - ref) <= bound * np.linalg.norm(ref)
    assert all(res <= tol)
    if precision == "fp64":
        assert list(its) == list(oits)
    spec = S.fft_r2c(u0)
    ref_spec = O.fft(u0.astype(complex))[:, : n[1] // 2 + 1]
    assert np.abs(spec[..., 0] + 1j * spec[..., 1] - ref_spec).max() <= 1e-13 * np.abs(ref_spec).max()


def test_phase_names_follow_the_kernel_enum():
    src = open(os.path.join(ROOT, "paper_2204_07247_gb300", "csrc", "solver.cuh")).read()
    body = src[src.index("enum Phase {"):]
    body = body[: body.index("};")]
    names = re.findall(r"PH_(\w+)", body)
    assert len(names) == len(pagd.PHASES)
    assert [n for n in names[:-1]] == list(pagd.PHASES[:-1]) and names[-1] == "DONE"
