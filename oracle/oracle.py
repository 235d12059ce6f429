"""ctypes front end of the FP64 CPU oracle (``pagd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke`` and the
CPU-baseline leg of ``bench.py`` may use this module; the product package never
imports it.  It shares no code with the CUDA library.

The C source is compiled with the host ``gcc`` into ``oracle/_build`` on first
use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pagd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpagd_oracle.so")

PFC, FCH = 0, 1
BDF2, MP, LBDF2, LMP = 0, 1, 2, 3
OK, EINVAL, ENOCONV, EPRECOND, ENAN = 0, 1, 4, 5, 6

# Sweeping friction list of Table 1: square roots of five equally spaced
# numbers in [0.1, 2].
PAPER_ETA = tuple(math.sqrt(0.1 + 0.475 * j) for j in range(5))


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:  # OpenMP only parallelises the line transforms; without it they run serially
            subprocess.check_call(cmd[:4] + ["-fopenmp"] + cmd[4:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double * 3), ("eps", ctypes.c_double), ("eta1", ctypes.c_double),
        ("eta2", ctypes.c_double), ("tau", ctypes.c_double), ("M", ctypes.c_double),
        ("scheme", ctypes.c_int), ("s", ctypes.c_double), ("n_eta", ctypes.c_int),
        ("eta", ctypes.c_double * 16), ("max_iter", ctypes.c_int),
        ("theta_mode", ctypes.c_int), ("accel", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        if _lib.orc_sizeof_params() != ctypes.sizeof(_Params):
            raise RuntimeError("oracle parameter struct layout mismatch")
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_Params)
        I = ctypes.POINTER(ctypes.c_int)
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_fft.argtypes = [ctypes.c_int, I, D, ctypes.c_int]
        _lib.orc_dft_brute.argtypes = [ctypes.c_int, I, D, D, ctypes.c_int]
        _lib.orc_frac_lap.argtypes = [P, D, D, ctypes.c_int]
        _lib.orc_mass.argtypes = [P, D]
        _lib.orc_mass.restype = ctypes.c_double
        _lib.orc_mu.argtypes = [P, D, D]
        _lib.orc_energy.argtypes = [P, D, D]
        _lib.orc_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, D]
        _lib.orc_objective.argtypes = [P, D, D, D, D, D]
        _lib.orc_gradient.argtypes = [P, D, D, D, D, D]
        _lib.orc_betas.argtypes = [P, ctypes.c_double, D, D]
        _lib.orc_pagd_step.argtypes = [P, ctypes.c_int, D, D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, D, D, I, D, D]
        _lib.orc_imex_step.argtypes = [P, ctypes.c_int, D, D, ctypes.c_double, ctypes.c_double, D]
        _lib.orc_scheme_residual.argtypes = [P, ctypes.c_int, D, D, ctypes.c_double,
                                             ctypes.c_double, D, D]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Problem:
    """Model, grid, scheme and solver settings (Table 1 style)."""
    model: int
    n: tuple
    L: tuple
    eps: float
    eta1: float = 0.0
    eta2: float = 0.0
    tau: float = 0.0
    M: float = 1.0
    scheme: int = BDF2
    s: float = 0.9
    eta: tuple = PAPER_ETA
    max_iter: int = 1000
    theta_mode: int = 0
    accel: int = 1

    @property
    def dim(self):
        return len(self.n)

    @property
    def shape(self):
        return tuple(self.n)

    def cparams(self) -> _Params:
        p = _Params()
        p.model, p.dim = self.model, len(self.n)
        for d in range(len(self.n)):
            p.n[d] = self.n[d]
            p.L[d] = self.L[d]
        p.eps, p.eta1, p.eta2, p.tau, p.M = self.eps, self.eta1, self.eta2, self.tau, self.M
        p.scheme, p.s = self.scheme, self.s
        p.n_eta = len(self.eta)
        for j, e in enumerate(self.eta):
            p.eta[j] = e
        p.max_iter, p.theta_mode, p.accel = self.max_iter, self.theta_mode, self.accel
        return p


def set_threads(n: int) -> None:
    """Threads for the oracle's line transforms (default 1).  Results do not
    depend on the count (each line is transformed as with one thread)."""
    lib().orc_set_threads(int(n))


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised complex DFT of a 1-3 dimensional array (own radix-2 FFT)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n = np.array(a.shape, dtype=np.int32)
    buf = a.view(np.float64)
    st = lib().orc_fft(a.ndim, _ip(n), _dp(buf), sign)
    if st != OK:
        raise ValueError("oracle fft: sizes must be powers of two")
    return a


def dft_brute(x: np.ndarray, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(a)
    n = np.array(a.shape, dtype=np.int32)
    lib().orc_dft_brute(a.ndim, _ip(n), _dp(a.view(np.float64)), _dp(out.view(np.float64)), sign)
    return out


def _r(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def frac_lap(P: Problem, w, alpha: int) -> np.ndarray:
    w = _r(w)
    out = np.empty_like(w)
    p = P.cparams()
    lib().orc_frac_lap(ctypes.byref(p), _dp(w), _dp(out), alpha)
    return out


def mass(P: Problem, u) -> float:
    u = _r(u)
    p = P.cparams()
    return lib().orc_mass(ctypes.byref(p), _dp(u))


def mu(P: Problem, u) -> np.ndarray:
    u = _r(u)
    out = np.empty_like(u)
    p = P.cparams()
    lib().orc_mu(ctypes.byref(p), _dp(u), _dp(out))
    return out


def energy(P: Problem, u) -> float:
    u = _r(u)
    e = np.zeros(1)
    p = P.cparams()
    lib().orc_energy(ctypes.byref(p), _dp(u), _dp(e))
    return float(e[0])


def coeffs(scheme: int, step: int, dt: float, dt_prev: float) -> np.ndarray:
    abc = np.zeros(3)
    lib().orc_coeffs(scheme, step, dt, dt_prev, _dp(abc))
    return abc


def objective(P: Problem, abc, un, unm1, v) -> float:
    abc, un, unm1, v = _r(abc), _r(un), _r(unm1), _r(v)
    g = np.zeros(1)
    p = P.cparams()
    lib().orc_objective(ctypes.byref(p), _dp(abc), _dp(un), _dp(unm1), _dp(v), _dp(g))
    return float(g[0])


def gradient(P: Problem, abc, un, unm1, v) -> np.ndarray:
    abc, un, unm1, v = _r(abc), _r(un), _r(unm1), _r(v)
    out = np.empty_like(v)
    p = P.cparams()
    lib().orc_gradient(ctypes.byref(p), _dp(abc), _dp(un), _dp(unm1), _dp(v), _dp(out))
    return out


def betas(P: Problem, a: float, vb0) -> np.ndarray:
    vb0 = _r(vb0)
    out = np.zeros(4)
    p = P.cparams()
    lib().orc_betas(ctypes.byref(p), a, _dp(vb0), _dp(out))
    return out


@dataclass
class StepResult:
    u: np.ndarray
    status: int
    iters: int
    hist: np.ndarray
    beta: np.ndarray = field(default_factory=lambda: np.zeros(4))


def pagd_step(P: Problem, step: int, un, unm1, dt: float, dt_prev: float, tol: float,
              guess=None) -> StepResult:
    """One fully implicit step solved by PAGD (or PGD when P.accel == 0)."""
    un, unm1 = _r(un), _r(unm1)
    out = np.empty_like(un)
    hist = np.zeros(max(P.max_iter, 1))
    beta = np.zeros(4)
    it = ctypes.c_int(0)
    p = P.cparams()
    g = None if guess is None else _r(guess)
    st = lib().orc_pagd_step(ctypes.byref(p), step, _dp(un), _dp(unm1), dt, dt_prev, tol,
                             None if g is None else _dp(g), _dp(out), ctypes.byref(it),
                             _dp(hist), _dp(beta))
    return StepResult(out, st, it.value, hist[: it.value].copy(), beta)


def imex_step(P: Problem, step: int, un, unm1, dt: float, dt_prev: float) -> np.ndarray:
    un, unm1 = _r(un), _r(unm1)
    out = np.empty_like(un)
    p = P.cparams()
    st = lib().orc_imex_step(ctypes.byref(p), step, _dp(un), _dp(unm1), dt, dt_prev, _dp(out))
    if st != OK:
        raise ValueError(f"oracle imex step failed: {st}")
    return out


def scheme_residual(P: Problem, step: int, un, unm1, dt: float, dt_prev: float, u) -> np.ndarray:
    un, unm1, u = _r(un), _r(unm1), _r(u)
    out = np.empty_like(u)
    p = P.cparams()
    lib().orc_scheme_residual(ctypes.byref(p), step, _dp(un), _dp(unm1), dt, dt_prev, _dp(u),
                              _dp(out))
    return out


def run(P: Problem, u0, dt: float, nsteps: int, tol: float, callback=None):
    """March nsteps fixed steps from u0 (u^{-1} := u^0).  Implicit schemes use
    PAGD/PGD; LBDF2/LMP use the linear IMEX solve.  Returns (u, per-step iters)."""
    un = _r(u0).copy()
    unm1 = un.copy()
    iters = []
    for n in range(nsteps):
        if P.scheme in (BDF2, MP):
            r = pagd_step(P, n, un, unm1, dt, dt, tol)
            if r.status != OK:
                raise RuntimeError(f"oracle step {n} failed with status {r.status}")
            unew = r.u
            iters.append(r.iters)
        else:
            unew = imex_step(P, n, un, unm1, dt, dt)
            iters.append(0)
        unm1, un = un, unew
        if callback is not None:
            callback(n, un)
    return un, iters


def rhs(P: Problem, v) -> np.ndarray:
    """R(v) = M Lap (delta E / delta u)(v)."""
    v = _r(v)
    out = np.empty_like(v)
    p = P.cparams()
    lib().orc_rhs(ctypes.byref(p), _dp(v), _dp(out))
    return out


def am3_err(P: Problem, un, ut, Rt, Rn, Rnm1, dt, dt_prev):
    un, ut, Rt, Rn, Rnm1 = (_r(a) for a in (un, ut, Rt, Rn, Rnm1))
    uh = np.empty_like(un)
    p = P.cparams()
    f = lib().orc_am3_err
    f.restype = ctypes.c_double
    e = f(ctypes.byref(p), _dp(un), _dp(ut), _dp(Rt), _dp(Rn), _dp(Rnm1), ctypes.c_double(dt),
          ctypes.c_double(dt_prev), _dp(uh))
    return e, uh


def midab2_err(P: Problem, un, unm1, unm2, ut, dt, dtn, dtnm1):
    un, unm1, unm2, ut = (_r(a) for a in (un, unm1, unm2, ut))
    uh = np.empty_like(un)
    p = P.cparams()
    f = lib().orc_midab2_err
    f.restype = ctypes.c_double
    e = f(ctypes.byref(p), _dp(un), _dp(unm1), _dp(unm2), _dp(ut), ctypes.c_double(dt), ctypes.c_double(dtn),
          ctypes.c_double(dtnm1), _dp(uh))
    return e, uh


def run_adaptive(P: Problem, u0, T, dt_min, dt_max, step_tol, tol, max_steps=100000):
    """Algorithm 3: tentative step, higher-order estimate (AM3, or midAB2 for
    MP from the third step on), accept if ERR <= step_tol or dt <= dt_min,
    next dt = clamp(0.9 (step_tol / ERR)^(1/3) dt, dt_min, dt_max).
    Returns (u, times, dts, rejections, iterations per accepted step)."""
    un = _r(u0).copy()
    unm1 = un.copy()
    unm2 = None
    t, n, dtt = 0.0, 0, dt_min
    dts, times, its = [], [0.0], []
    dt_prev = dt_min
    rej = 0
    Rn = rhs(P, un)
    Rnm1 = Rn.copy()
    while t < T and n < max_steps:
        if P.scheme in (BDF2, MP):
            r = pagd_step(P, n, un, unm1, dtt, dt_prev, tol)
            if r.status != OK:
                raise RuntimeError(f"oracle step failed with status {r.status}")
            ut, it = r.u, r.iters
        else:
            ut, it = imex_step(P, n, un, unm1, dtt, dt_prev), 0
        Rt = rhs(P, ut)
        if P.scheme == MP and n >= 2:
            err, _ = midab2_err(P, un, unm1, unm2, ut, dtt, dts[-1], dts[-2])
        else:
            err, _ = am3_err(P, un, ut, Rt, Rn, Rnm1, dtt, dt_prev if n > 0 else dtt)
        tmp = dtt
        if err <= step_tol or dtt <= dt_min:
            unm2, unm1, un = unm1, un, ut
            Rnm1, Rn = Rn, Rt
            dt_prev = dtt
            dts.append(dtt)
            t += dtt
            times.append(t)
            its.append(it)
            n += 1
        else:
            rej += 1
        dtt = max(dt_min, min(0.9 * (step_tol / max(err, 1e-300)) ** (1.0 / 3.0) * tmp, dt_max))
    return un, np.array(times), np.array(dts), rej, its

