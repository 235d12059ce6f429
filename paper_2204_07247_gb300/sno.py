"""Binding of the learned initial iterate's network (include/pagd_sno.h) and
its training on solver trajectories.

Argument marshalling only: the network's forward, backward and Adam update run
in the CUDA kernels of libpagd.so.  Parameters, moments and the workspace are
torch CUDA tensors; there is no CPU path.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import inputs as I
from . import pagd

EXPORTS = ("sno_create", "sno_param_count", "sno_workspace_size", "sno_set_workspace", "sno_predict",
           "sno_loss_grad", "sno_adam_step", "sno_round_bf16", "sno_last_error", "sno_destroy")


def _declare(lib):
    if getattr(lib, "_sno_declared", False):
        return lib
    P = ctypes.c_void_p
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "sno_create": [ctypes.POINTER(P), i, i, i, i, i, i, i, P],
        "sno_param_count": [P, ctypes.POINTER(ctypes.c_size_t)],
        "sno_workspace_size": [P, ctypes.POINTER(ctypes.c_size_t)],
        "sno_set_workspace": [P, P, ctypes.c_size_t],
        "sno_predict": [P, P, P, P, d, d, d, i, P],
        "sno_loss_grad": [P, P, P, P, P, d, d, d, i, P, ctypes.POINTER(ctypes.c_double)],
        "sno_adam_step": [P, P, P, P, P, i, d],
        "sno_round_bf16": [P, P, P],
        "sno_last_error": [P],
        "sno_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sno_last_error.restype = ctypes.c_char_p
    lib.sno_destroy.restype = None
    lib._sno_declared = True
    return lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class SNO:
    """The network on an n0 x n1 grid: channels, layers, kept modes (M0, M1),
    and the largest number of samples per call (batch).  bf16: the network
    computes with its weights rounded to BF16 (FP32 accumulation); Adam keeps
    the FP32 master copy and the weights are re-rounded after every update."""

    def __init__(self, n, channels=16, layers=4, modes=(16, 16), batch=4, seed=0, lib=None, stream=None,
                 bf16=False):
        import torch
        self.torch = torch
        self.lib = _declare(lib if lib is not None else pagd.load())
        self.n = tuple(n)
        self.C, self.L, self.M0, self.M1, self.batch = channels, layers, modes[0], modes[1], batch
        self._h = ctypes.c_void_p()
        st = self.lib.sno_create(ctypes.byref(self._h), n[0], n[1], channels, layers, modes[0], modes[1], batch,
                                 stream)
        if st != 0:
            raise pagd.PagdError(st, "sno_create")
        cnt = ctypes.c_size_t()
        self._check(self.lib.sno_param_count(self._h, ctypes.byref(cnt)), "param_count")
        self.nparams = cnt.value
        wb = ctypes.c_size_t()
        self._check(self.lib.sno_workspace_size(self._h, ctypes.byref(wb)), "workspace_size")
        self.ws = torch.empty(wb.value + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        self._check(self.lib.sno_set_workspace(self._h, ctypes.c_void_p(base + ((-base) % 256)), wb.value),
                    "set_workspace")
        self.bf16 = bool(bf16)
        self.master = torch.from_numpy(self.initial_params(seed)).cuda()
        self.params = torch.empty_like(self.master) if self.bf16 else self.master
        self._round()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.t = 0

    def initial_params(self, seed):
        """Seeded uniform initialisation scaled by fan-in (float32, flat layout)."""
        C, L, M = self.C, self.L, self.M0 * self.M1
        u = (2.0 * I.uniform01(seed, self.nparams) - 1.0).astype(np.float32)
        out = np.empty(self.nparams, dtype=np.float32)
        o = 0

        def put(n, scale):
            nonlocal o
            out[o:o + n] = u[o:o + n] * scale
            o += n
        put(2 * C, 1.0 / np.sqrt(2.0))
        put(C, 0.1)
        for _ in range(L):
            put(C * C, 1.0 / np.sqrt(C))
            put(C, 0.1)
            put(2 * C * C * M, 1.0 / (C * np.sqrt(M)))
        put(C, 0.1 / np.sqrt(C))
        put(1, 0.0)
        assert o == self.nparams
        return out

    def _round(self):
        if self.bf16:
            self._check(self.lib.sno_round_bf16(self._h, _p(self.master), _p(self.params)), "round_bf16")

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.sno_last_error(self._h) if self._h else b""
            raise pagd.PagdError(st, f"{what}: {msg.decode() if msg else ''}")

    def predict(self, un, unm1, rho, s_in, s_out, guess=None):
        B = un.shape[0] if un.dim() == 3 else 1
        guess = self.torch.empty_like(un) if guess is None else guess
        self._check(self.lib.sno_predict(self._h, _p(self.params), _p(un), _p(unm1), rho, s_in, s_out, B,
                                         _p(guess)), "predict")
        return guess

    def loss_grad(self, un, unm1, target, rho, s_in, s_out):
        B = un.shape[0] if un.dim() == 3 else 1
        loss = ctypes.c_double()
        self._check(self.lib.sno_loss_grad(self._h, _p(self.params), _p(un), _p(unm1), _p(target), rho, s_in,
                                           s_out, B, _p(self.grad), ctypes.byref(loss)), "loss_grad")
        return loss.value, self.grad

    def adam(self, lr):
        self.t += 1
        self._check(self.lib.sno_adam_step(self._h, _p(self.master), _p(self.grad), _p(self.m), _p(self.v),
                                           self.t, lr), "adam")
        self._round()

    def close(self):
        if self._h:
            self.lib.sno_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
