"""Thin Python binding of the C ABI in ``include/pagd.h`` (ctypes).

Argument marshalling only: every step of the time step runs in the CUDA
kernels of ``libpagd.so``.  PyTorch provides the device memory (the solver
workspace is a torch uint8 tensor) and the stream.  If the CUDA library is
missing or no GPU is present the calls raise; there is no CPU fallback.

The same binding can drive the test-only emulation library
(``load_emulation()``), in which "device" buffers are host numpy arrays.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

PFC, FCH = 0, 1
BDF2, MP, LBDF2, LMP = 0, 1, 2, 3
FP64, FP32_MIXED = 0, 1
STATUS = {0: "PAGD_OK", 1: "PAGD_EINVAL", 2: "PAGD_ENOMEM", 3: "PAGD_ECUDA", 4: "PAGD_ENOCONV",
          5: "PAGD_EPRECOND", 6: "PAGD_ENAN", 7: "PAGD_ESTATE", 8: "PAGD_ETIMEOUT"}
SCHEMES = {"bdf2": BDF2, "mp": MP, "lbdf2": LBDF2, "lmp": LMP}
PRECISIONS = {"fp64": FP64, "fp32_mixed": FP32_MIXED}
EXPORTS = ("pagd_default_opts", "pfc_init", "fch_init", "pagd_workspace_size", "pagd_set_workspace",
           "pagd_set_state", "pagd_step", "pagd_step_with_guess", "pagd_run", "pagd_run_host", "pagd_energy", "pagd_mass",
           "pagd_rhs", "pagd_run_adaptive", "pagd_fft_r2c", "pagd_fft_c2r", "pagd_get_state", "pagd_step_static", "pagd_barrier_probe", "pagd_pass_probe", "pagd_launch_info", "pagd_set_trace",
           "pagd_get_trace", "pagd_last_error", "pagd_destroy", "pagd_batch_create",
           "pagd_batch_workspace_size", "pagd_batch_set_workspace", "pagd_batch_run", "pagd_batch_set_shape",
           "pagd_batch_step_with_guess",
           "pagd_batch_launch_info",
           "pagd_batch_last_error", "pagd_batch_destroy")
# phase identifiers of the persistent kernel's control machine (for traces)
PHASES = ("B", "C", "D", "E", "R1", "CI", "RI", "ACCEPT", "FAIL", "FWD_R", "FWD_C", "INV_C", "INV_R",
          "EN_R", "EN_C", "EN_R2", "MASS", "IM_R0", "IM_C0", "IM_R1", "IM_C1", "IM_R2", "MF", "MI",
          "GS", "RH_R0", "RH_C0", "RH_R1", "RH_C1", "RH_R2", "EST", "NOP", "START")


class PagdError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class Opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double), ("n_eta", ctypes.c_int), ("eta", ctypes.c_double * 16),
                ("max_iter", ctypes.c_int), ("theta_mode", ctypes.c_int), ("accel", ctypes.c_int)]


def _declare(lib):
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    IP = ctypes.POINTER(ctypes.c_int)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "pagd_default_opts": [ctypes.POINTER(Opts)],
        "pfc_init": [ctypes.POINTER(P), i, IP, D, d, d, i, i, ctypes.POINTER(Opts), P],
        "fch_init": [ctypes.POINTER(P), i, IP, D, d, d, d, d, d, i, i, ctypes.POINTER(Opts), P],
        "pagd_workspace_size": [P, ctypes.POINTER(ctypes.c_size_t)],
        "pagd_set_workspace": [P, P, ctypes.c_size_t],
        "pagd_set_state": [P, P],
        "pagd_step": [P, P, d, d, IP, D],
        "pagd_step_with_guess": [P, P, P, d, d, IP, D, IP],
        "pagd_run": [P, P, d, i, d, IP, D],
        "pagd_run_host": [P, P, P, d, i, d, IP, D],
        "pagd_energy": [P, P, D],
        "pagd_mass": [P, P, D],
        "pagd_rhs": [P, P, P],
        "pagd_run_adaptive": [P, d, d, d, d, d, i, P, P, D, D, IP, IP, IP],
        "pagd_fft_r2c": [P, P, P],
        "pagd_fft_c2r": [P, P, P],
        "pagd_get_state": [P, P, P, IP],
        "pagd_step_static": [P, P, P, i, d, d, d, P, IP, D],
        "pagd_barrier_probe": [P, i, D],
        "pagd_pass_probe": [P, i, i, D],
        "pagd_launch_info": [P, IP, IP, IP, IP, ctypes.POINTER(ctypes.c_size_t), IP],
        "pagd_set_trace": [P, i],
        "pagd_get_trace": [P, IP, D, i, IP],
        "pagd_last_error": [P],
        "pagd_destroy": [P],
        "pagd_batch_create": [ctypes.POINTER(P), ctypes.POINTER(P), i],
        "pagd_batch_workspace_size": [P, ctypes.POINTER(ctypes.c_size_t)],
        "pagd_batch_set_workspace": [P, P, ctypes.c_size_t],
        "pagd_batch_run": [P, d, i, d, IP, D, IP],
        "pagd_batch_set_shape": [P, i, i],
        "pagd_batch_step_with_guess": [P, ctypes.POINTER(P), d, d, IP, D, IP, IP],
        "pagd_batch_launch_info": [P, IP, IP, ctypes.POINTER(ctypes.c_size_t), IP, IP],
        "pagd_batch_last_error": [P],
        "pagd_batch_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.pagd_last_error.restype = ctypes.c_char_p
    lib.pagd_destroy.restype = None
    lib.pagd_batch_last_error.restype = ctypes.c_char_p
    lib.pagd_batch_destroy.restype = None
    return lib


_LIBS = {}


def load(path: str | None = None):
    """Load libpagd.so (building it with nvcc if needed).  Raises if the CUDA
    library cannot be built or loaded."""
    key = path or "cuda"
    if key not in _LIBS:
        p = path or _build.build_library()
        _LIBS[key] = _declare(ctypes.CDLL(p))
    return _LIBS[key]


def load_emulation():
    """Test-only: the CPU emulation of the kernels (host memory as 'device')."""
    if "emu" not in _LIBS:
        _LIBS["emu"] = _declare(ctypes.CDLL(_build.build_emulation()))
    return _LIBS["emu"]


def default_opts(lib=None) -> Opts:
    o = Opts()
    (lib or load_emulation_or_cuda()).pagd_default_opts(ctypes.byref(o))
    return o


def load_emulation_or_cuda():
    return _LIBS.get("cuda") or _LIBS.get("emu") or load()


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Solver:
    """One PFC or FCH problem on a periodic grid, advanced by the C ABI.

    On the CUDA library, fields are torch float64 tensors on the current CUDA
    device; on the emulation library they are numpy float64 arrays.
    """

    def __init__(self, model, n, L, eps, eta1=0.0, eta2=0.0, tau=0.0, M=1.0, scheme="bdf2",
                 precision="fp64", s=0.9, eta=None, max_iter=1000, theta_mode=0, accel=1,
                 lib=None, stream=None):
        self.lib = lib if lib is not None else load()
        self.emu = self.lib is _LIBS.get("emu")
        self.model = {"pfc": PFC, "fch": FCH}.get(model, model)
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.scheme = SCHEMES.get(scheme, scheme)
        self.precision = PRECISIONS.get(precision, precision)
        o = Opts()
        self.lib.pagd_default_opts(ctypes.byref(o))
        o.s = s
        if eta is not None:
            o.n_eta = len(eta)
            for j, e in enumerate(eta):
                o.eta[j] = e
        o.max_iter, o.theta_mode, o.accel = max_iter, theta_mode, accel
        self.opts = o
        self._h = ctypes.c_void_p()
        nn = (ctypes.c_int * 3)(*(list(self.n) + [1] * (3 - len(self.n))))
        LL = (ctypes.c_double * 3)(*(list(self.L) + [1.0] * (3 - len(self.L))))
        self.stream = stream
        sp = None
        if stream is not None:
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        if self.model == PFC:
            st = self.lib.pfc_init(ctypes.byref(self._h), len(self.n), nn, LL, eps, M, self.scheme,
                                   self.precision, ctypes.byref(o), sp)
        else:
            st = self.lib.fch_init(ctypes.byref(self._h), len(self.n), nn, LL, eps, eta1, eta2, tau,
                                   M, self.scheme, self.precision, ctypes.byref(o), sp)
        if st != 0:
            raise PagdError(st, "init")
        nb = ctypes.c_size_t()
        self._check(self.lib.pagd_workspace_size(self._h, ctypes.byref(nb)), "workspace_size")
        self.ws_bytes = nb.value
        if self.emu:
            raw = np.zeros(self.ws_bytes + 256, dtype=np.uint8)
            off = (-raw.ctypes.data) % 256
            self._ws_keep = raw
            self.ws = raw[off:off + self.ws_bytes]
            ptr = self.ws.ctypes.data
        else:
            import torch
            self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self.ws.data_ptr()
            ptr = base + ((-base) % 256)
        self._check(self.lib.pagd_set_workspace(self._h, ctypes.c_void_p(ptr), self.ws_bytes),
                    "set_workspace")

    # -------------------------------------------------------------- helpers
    def _check(self, st, what):
        if st != 0:
            msg = self.lib.pagd_last_error(self._h) if self._h else b""
            raise PagdError(st, f"{what}: {msg.decode() if msg else ''}")

    def _ptr(self, x):
        if x is None:
            return None
        if _is_torch(x):
            if self.emu:
                raise TypeError("emulation library takes numpy arrays")
            assert x.is_cuda and x.is_contiguous(), "expected a contiguous CUDA tensor"
            return ctypes.c_void_p(x.data_ptr())
        if self.emu:
            assert x.flags.c_contiguous
            return ctypes.c_void_p(x.ctypes.data)
        raise TypeError("the CUDA library takes torch CUDA tensors")

    def empty_field(self):
        if self.emu:
            return np.zeros(self.n, dtype=np.float64)
        import torch
        return torch.zeros(self.n, dtype=torch.float64, device="cuda")

    def empty_spectrum(self):
        shp = self.n[:-1] + (self.n[-1] // 2 + 1, 2)
        if self.emu:
            return np.zeros(shp, dtype=np.float64)
        import torch
        return torch.zeros(shp, dtype=torch.float64, device="cuda")

    # ------------------------------------------------------------ C ABI
    def set_state(self, u0):
        self._check(self.lib.pagd_set_state(self._h, self._ptr(u0)), "set_state")

    def step(self, u_out, dt, tol):
        it = ctypes.c_int()
        r = ctypes.c_double()
        self._check(self.lib.pagd_step(self._h, self._ptr(u_out), dt, tol, ctypes.byref(it),
                                       ctypes.byref(r)), "step")
        return it.value, r.value

    def step_with_guess(self, u_out, guess, dt, tol):
        """One implicit step from the caller's initial iterate `guess` (kept only
        if its first PAGD direction is smaller than the extrapolation's);
        returns (evaluations, accepted residual, guess used)."""
        it = ctypes.c_int()
        r = ctypes.c_double()
        used = ctypes.c_int()
        self._check(self.lib.pagd_step_with_guess(self._h, self._ptr(u_out), self._ptr(guess), dt, tol,
                                                  ctypes.byref(it), ctypes.byref(r), ctypes.byref(used)),
                    "step_with_guess")
        return it.value, r.value, bool(used.value)

    def run(self, dt, nsteps, tol, u_out=None):
        iters = (ctypes.c_int * max(nsteps, 1))()
        res = (ctypes.c_double * max(nsteps, 1))()
        self._check(self.lib.pagd_run(self._h, self._ptr(u_out), dt, nsteps, tol, iters, res), "run")
        return np.array(iters[:nsteps]), np.array(res[:nsteps])

    def run_host(self, u0, dt, nsteps, tol):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        out = np.empty_like(u0)
        iters = (ctypes.c_int * max(nsteps, 1))()
        res = (ctypes.c_double * max(nsteps, 1))()
        self._check(self.lib.pagd_run_host(self._h, ctypes.c_void_p(u0.ctypes.data),
                                           ctypes.c_void_p(out.ctypes.data), dt, nsteps, tol, iters,
                                           res), "run_host")
        return out, np.array(iters[:nsteps]), np.array(res[:nsteps])

    def energy(self, u):
        e = ctypes.c_double()
        self._check(self.lib.pagd_energy(self._h, self._ptr(u), ctypes.byref(e)), "energy")
        return e.value

    def mass(self, u):
        m = ctypes.c_double()
        self._check(self.lib.pagd_mass(self._h, self._ptr(u), ctypes.byref(m)), "mass")
        return m.value

    def rhs(self, v, out=None):
        """R(v) = M Lap mu(v)."""
        out = self.empty_field() if out is None else out
        self._check(self.lib.pagd_rhs(self._h, self._ptr(v), self._ptr(out)), "rhs")
        return out

    def run_adaptive(self, T, dt_min, dt_max, step_tol, tol, max_steps=10000, u_out=None):
        """Algorithm 3 from the current state to time T; returns (times, dts,
        evaluations per accepted step, rejected count)."""
        scratch = (np.zeros(6 * int(np.prod(self.n))) if self.emu else
                   __import__("torch").empty(6 * int(np.prod(self.n)), dtype=__import__("torch").float64,
                                             device="cuda"))
        t = (ctypes.c_double * (max_steps + 1))()
        dts = (ctypes.c_double * max_steps)()
        its = (ctypes.c_int * max_steps)()
        n, rej = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.pagd_run_adaptive(self._h, T, dt_min, dt_max, step_tol, tol, max_steps,
                                               self._ptr(scratch), self._ptr(u_out), t, dts, its,
                                               ctypes.byref(n), ctypes.byref(rej)), "run_adaptive")
        k = n.value
        return np.array(t[:k + 1]), np.array(dts[:k]), np.array(its[:k]), rej.value

    def fft_r2c(self, u, spec=None):
        spec = self.empty_spectrum() if spec is None else spec
        self._check(self.lib.pagd_fft_r2c(self._h, self._ptr(u), self._ptr(spec)), "fft_r2c")
        return spec

    def fft_c2r(self, spec, u=None):
        u = self.empty_field() if u is None else u
        self._check(self.lib.pagd_fft_c2r(self._h, self._ptr(spec), self._ptr(u)), "fft_c2r")
        return u

    def get_state(self):
        un, um = self.empty_field(), self.empty_field()
        st = ctypes.c_int()
        self._check(self.lib.pagd_get_state(self._h, self._ptr(un), self._ptr(um), ctypes.byref(st)),
                    "get_state")
        return un, um, st.value

    def step_static(self, un, unm1, step_index, dt, dt_prev, tol, u_out):
        """One step on the library's static device scratch (no workspace use):
        u_out = u^{n+1} from un = u^n, unm1 = u^{n-1}.  For callers that cannot
        allocate device memory; see pagd_step_static in include/pagd.h."""
        it = ctypes.c_int()
        r = ctypes.c_double()
        self._check(self.lib.pagd_step_static(self._h, self._ptr(un), self._ptr(unm1), step_index, dt,
                                              dt_prev, tol, self._ptr(u_out), ctypes.byref(it),
                                              ctypes.byref(r)), "step_static")
        return it.value, r.value

    def launch_info(self):
        """{grid (of the last launch), threads, cluster, coop, smem, staged} of
        the solver's persistent kernel."""
        g, t, c, co, sg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sm = ctypes.c_size_t()
        self._check(self.lib.pagd_launch_info(self._h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(c),
                                              ctypes.byref(co), ctypes.byref(sm), ctypes.byref(sg)), "launch_info")
        return {"grid": g.value, "threads": t.value, "cluster": c.value, "coop": co.value, "smem": sm.value,
                "staged": bool(sg.value)}

    def barrier_probe(self, count=2000):
        """Device time per empty phase of the persistent kernel (microseconds):
        the cost of one device-wide barrier with this solver's launch plan."""
        us = ctypes.c_double()
        self._check(self.lib.pagd_barrier_probe(self._h, int(count), ctypes.byref(us)), "barrier_probe")
        return us.value

    PASSES = ("RI", "CI", "MF", "MI")

    def pass_probe(self, which, count=100):
        """Device time per repetition of one iteration pass ("RI", "CI", and
        in 3D "MF", "MI") run on its own in one launch, barrier included
        (microseconds).  Needs a completed step; overwrites the iteration
        buffers, keeps the state."""
        us = ctypes.c_double()
        self._check(self.lib.pagd_pass_probe(self._h, self.PASSES.index(which), int(count), ctypes.byref(us)),
                    "pass_probe")
        return us.value

    def set_trace(self, enable=True):
        self._check(self.lib.pagd_set_trace(self._h, 1 if enable else 0), "set_trace")

    def get_trace(self, cap=8192, raw=False):
        """(phase names, end times in us) of the last launch's phases (suffix
        "/inc": part of an incremental base evaluation); raw: the identifiers
        as recorded (bit masks for a batch's global phases)."""
        ph = (ctypes.c_int * cap)()
        t = (ctypes.c_double * cap)()
        cnt = ctypes.c_int()
        self._check(self.lib.pagd_get_trace(self._h, ph, t, cap, ctypes.byref(cnt)), "get_trace")
        n = min(cnt.value, cap)
        if raw:
            return [ph[i] & 0xFFFFFFFF for i in range(n)], np.array(t[:n])
        return ([PHASES[ph[i] & 0xFFFF] + ("/inc" if ph[i] >> 16 & 1 else "") for i in range(n)],
                np.array(t[:n]))

    def close(self):
        if self._h:
            self.lib.pagd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Solvers advanced together by one persistent launch per chunk
    (pagd_batch_* in include/pagd.h).  The members must share the library,
    precision and stream, and have their states set; they stay usable on
    their own (get_state, energy, ...) and must outlive the batch."""

    def __init__(self, members):
        self.members = list(members)
        self.lib = self.members[0].lib
        self.emu = self.members[0].emu
        self._h = ctypes.c_void_p()
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        st = self.lib.pagd_batch_create(ctypes.byref(self._h), arr, len(self.members))
        if st != 0:
            raise PagdError(st, "batch_create")
        nb = ctypes.c_size_t()
        self._check(self.lib.pagd_batch_workspace_size(self._h, ctypes.byref(nb)), "batch_workspace_size")
        self.ws_bytes = nb.value
        if self.emu:
            self.ws = np.zeros(self.ws_bytes + 256, dtype=np.uint8)
            base = self.ws.ctypes.data
        else:
            import torch
            self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self.ws.data_ptr()
        ptr = base + ((-base) % 256)
        self._check(self.lib.pagd_batch_set_workspace(self._h, ctypes.c_void_p(ptr), self.ws_bytes),
                    "batch_set_workspace")

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.pagd_batch_last_error(self._h) if self._h else b""
            raise PagdError(st, f"{what}: {msg.decode() if msg else ''}")

    def run(self, dt, nsteps, tol, check=True):
        """Advance every member; returns (iters [count, nsteps], resid, status [count])."""
        cnt = len(self.members)
        iters = np.zeros((cnt, max(nsteps, 1)), dtype=np.int32)
        res = np.zeros((cnt, max(nsteps, 1)), dtype=np.float64)
        status = np.zeros(cnt, dtype=np.int32)
        st = self.lib.pagd_batch_run(self._h, dt, nsteps, tol,
                                     iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if check:
            self._check(st, "batch_run")
        return iters[:, :nsteps], res[:, :nsteps], status

    def step_with_guess(self, guesses, dt, tol, check=True):
        """One step of every member from its guess (None: the extrapolation);
        returns (iters [count], resid [count], status [count], used [count])."""
        cnt = len(self.members)
        arr = (ctypes.c_void_p * cnt)(*[None if g is None else self.members[0]._ptr(g).value for g in guesses])
        iters = np.zeros(cnt, dtype=np.int32)
        res = np.zeros(cnt, dtype=np.float64)
        status = np.zeros(cnt, dtype=np.int32)
        used = np.zeros(cnt, dtype=np.int32)
        st = self.lib.pagd_batch_step_with_guess(self._h, arr, dt, tol,
                                                 iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                 res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                 used.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if check:
            self._check(st, "batch_step_with_guess")
        return iters, res, status, used.astype(bool)

    def set_shape(self, warps_per_cta, ctas_per_sm):
        """Launch shape of the batched kernel; False if it does not fit."""
        return self.lib.pagd_batch_set_shape(self._h, int(warps_per_cta), int(ctas_per_sm)) == 0

    def launch_info(self):
        g, w, q, sg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sm = ctypes.c_size_t()
        self._check(self.lib.pagd_batch_launch_info(self._h, ctypes.byref(g), ctypes.byref(w), ctypes.byref(sm),
                                                    ctypes.byref(q), ctypes.byref(sg)), "batch_launch_info")
        return {"grid": g.value, "warps_per_cta": w.value, "smem": sm.value, "sequential": bool(q.value),
                "staged_members": sg.value}

    def close(self):
        if self._h:
            self.lib.pagd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solver_for(workload, lib=None, **over):
    """A Solver for a named workload from ``inputs.WORKLOADS``."""
    w = workload
    kw = dict(model=w.model, n=w.n, L=w.L, eps=w.eps, eta1=w.eta1, eta2=w.eta2, tau=w.tau, M=w.M,
              scheme=w.scheme, precision=w.precision, s=w.s, eta=w.eta, max_iter=w.max_iter, lib=lib)
    kw.update(over)
    return Solver(**kw)
