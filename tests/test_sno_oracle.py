"""Pins of the network oracle (oracle/sno_oracle.py) against facts that do not
come from it: the spectral operator acting on single Fourier modes (identity on
a kept mode, zero on a dropped one), GELU at closed-form points, and the
gradient of the loss by central finite differences (independent of autograd).
Also: the C ABI of the network is declared and exported.  No GPU."""
import math
import os
import re

import numpy as np
import pytest
import torch

from oracle import sno_oracle as S
from paper_2204_07247_gb300 import pagd
from paper_2204_07247_gb300 import sno as SB

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _grid(n0, n1):
    x0 = torch.arange(n0, dtype=torch.float64)[:, None] * (2 * math.pi / n0)
    x1 = torch.arange(n1, dtype=torch.float64)[None, :] * (2 * math.pi / n1)
    return x0, x1


@pytest.mark.parametrize("k", [(1, 2), (-3, 1), (2, 0), (0, 3)])
def test_spectral_operator_identity_on_kept_modes(k):
    n0, n1, M0, M1, C = 16, 16, 8, 4, 2
    x0, x1 = _grid(n0, n1)
    v = torch.stack([torch.cos(k[0] * x0 + k[1] * x1 + 0.3), torch.sin(k[0] * x0 + k[1] * x1)])
    R = torch.zeros((C, C, M0 * M1), dtype=torch.complex128)
    for c in range(C):
        R[c, c, :] = 1.0
    assert torch.allclose(S.spectral(v, R, M0, M1), v, atol=1e-13)


@pytest.mark.parametrize("k", [(5, 1), (1, 4), (-5, 2)])
def test_spectral_operator_drops_other_modes(k):
    n0, n1, M0, M1 = 16, 16, 8, 4  # kept k0 in [-4, 4), k1 in [0, 4)
    x0, x1 = _grid(n0, n1)
    v = torch.cos(k[0] * x0 + k[1] * x1)[None]
    R = torch.ones((1, 1, M0 * M1), dtype=torch.complex128)
    assert torch.abs(S.spectral(v, R, M0, M1)).max() <= 1e-13


def test_spectral_operator_scales_and_rotates():
    """R = r e^{i phi} on a kept mode k1 > 0 maps cos(k.x) to r cos(k.x + phi)."""
    n0, n1, M0, M1 = 16, 32, 8, 6
    x0, x1 = _grid(n0, n1)
    v = torch.cos(2 * x0 + 3 * x1)[None]
    r, phi = 0.7, 0.4
    R = torch.full((1, 1, M0 * M1), complex(r * math.cos(phi), r * math.sin(phi)), dtype=torch.complex128)
    ref = r * torch.cos(2 * x0 + 3 * x1 + phi)
    assert torch.allclose(S.spectral(v, R, M0, M1)[0], ref, atol=1e-13)


def test_gelu_closed_form():
    x = torch.tensor([0.0, 1.0, -2.0], dtype=torch.float64)
    c = math.sqrt(2 / math.pi)
    ref = [0.0, 0.5 * (1 + math.tanh(c * 1.044715)), -1.0 * (1 + math.tanh(c * (-2 - 0.044715 * 8)))]
    assert torch.allclose(S.gelu(x), torch.tensor(ref, dtype=torch.float64), atol=1e-15)


def test_loss_gradient_by_finite_differences():
    C, L, M0, M1 = 3, 2, 4, 3
    n0, n1, B = 8, 16, 2
    g = torch.Generator().manual_seed(0)
    theta = (torch.rand(S.param_count(C, L, M0, M1), generator=g, dtype=torch.float64) - 0.5) * 0.6
    un = torch.rand((B, n0, n1), generator=g, dtype=torch.float64) - 0.3
    unm1 = un + 0.01 * torch.rand((B, n0, n1), generator=g, dtype=torch.float64)
    target = un + 0.02 * torch.rand((B, n0, n1), generator=g, dtype=torch.float64)
    args = (un, unm1, target, 1.0, 10.0, 0.01, C, L, M0, M1)
    _, grad = S.loss_and_grad(theta, *args)
    h = 1e-6
    for i in torch.randint(0, theta.numel(), (12,), generator=g).tolist() + [0, theta.numel() - 1]:
        tp, tm = theta.clone(), theta.clone()
        tp[i] += h
        tm[i] -= h
        fd = (float(S.loss(tp, *args)) - float(S.loss(tm, *args))) / (2 * h)
        assert abs(fd - float(grad[i])) <= 1e-7 * max(1.0, abs(fd)), i


def test_network_abi_declared_and_exported():
    src = open(os.path.join(ROOT, "include", "pagd_sno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:pagd_status|const char\s*\*|void)\s+(\w+)\s*\(", src, flags=re.M))
    assert names == set(SB.EXPORTS)
    lib = pagd.load()
    for n in names:
        assert hasattr(lib, n), n
