"""Plain PyTorch-CPU (float64) definition of the learned initial iterate's
network, the reference for the CUDA forward and backward kernels.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's checks, never
by the product path.  It shares no code with the CUDA library; the DFTs here are
torch.fft on the full grid followed by selecting the kept modes, and the
gradient is torch autograd.

Network (per sample, grid n0 x n1, np = n0 n1):
  a = [u^n, s_in (u^n - u^{n-1})],  v_0 = P a + b_P,
  v_{l+1} = GELU(W_l v_l + b_l + K_l v_l),  out = Q v_L + b_Q,
  (K v)[o] = Re sum over kept modes m of w_m (sum_c R[o][c][m] F[c][m]) e^{i k_m.x} / np,
  F[c][m] = sum_x v[c](x) e^{-i k_m.x},  kept k0 in [-M0/2, M0/2), k1 in [0, M1),
  w_m = 1 for k1 = 0 and 2 otherwise.
GELU in its tanh form.  The flat parameter layout: P [C][2], b_P [C]; per layer
W [C][C], b [C], R [C][C][M0 M1][2]; Q [C], b_Q.
"""
from __future__ import annotations

import math

import torch


def param_count(C, L, M0, M1):
    M = M0 * M1
    return 3 * C + L * (C * C + C + 2 * C * C * M) + C + 1


def unpack(theta, C, L, M0, M1):
    M = M0 * M1
    o = 0

    def take(n, shape):
        nonlocal o
        t = theta[o:o + n].reshape(shape)
        o += n
        return t
    P = take(2 * C, (C, 2))
    bP = take(C, (C,))
    layers = []
    for _ in range(L):
        W = take(C * C, (C, C))
        b = take(C, (C,))
        R = take(2 * C * C * M, (C, C, M, 2))
        layers.append((W, b, torch.complex(R[..., 0], R[..., 1])))
    Q = take(C, (C,))
    bQ = take(1, (1,))
    assert o == theta.numel()
    return P, bP, layers, Q, bQ


def kept_k0(n0, M0):
    return [m if m < M0 // 2 else n0 - M0 + m for m in range(M0)]


def gelu(x):
    return 0.5 * x * (1.0 + torch.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))


def spectral(v, R, M0, M1):
    """K v for v of shape [C, n0, n1] with weights R [C_out, C_in, M0 M1]."""
    C, n0, n1 = v.shape
    full = torch.fft.fft2(v.to(torch.complex128))          # sum_x v e^{-i k.x}
    k0 = kept_k0(n0, M0)
    F = full[:, k0, :M1].reshape(C, M0 * M1)              # [C_in, M]
    G = torch.einsum("ocm,cm->om", R, F)                   # [C_out, M]
    w = torch.ones(M1, dtype=torch.float64)
    w[1:] = 2.0
    Z = torch.zeros((R.shape[0], n0, n1), dtype=torch.complex128)
    Z[:, k0, :M1] = G.reshape(-1, M0, M1) * w
    return torch.fft.ifft2(Z).real                         # Re sum w G e^{+i k.x} / np


def forward(theta, un, unm1, rho, s_in, s_out, C, L, M0, M1):
    """guess (and the network output) for u^n, u^{n-1} of shape [B, n0, n1]."""
    P, bP, layers, Q, bQ = unpack(theta, C, L, M0, M1)
    outs = []
    for b in range(un.shape[0]):
        a = torch.stack([un[b], s_in * (un[b] - unm1[b])])
        v = torch.einsum("cj,jxy->cxy", P, a) + bP[:, None, None]
        for W, bias, R in layers:
            z = torch.einsum("oc,cxy->oxy", W, v) + bias[:, None, None] + spectral(v, R, M0, M1)
            v = gelu(z)
        outs.append(torch.einsum("c,cxy->xy", Q, v) + bQ[0])
    out = torch.stack(outs)
    ext = un + rho * (un - unm1)
    return ext + s_out * out, out


def loss(theta, un, unm1, target, rho, s_in, s_out, C, L, M0, M1):
    _, out = forward(theta, un, unm1, rho, s_in, s_out, C, L, M0, M1)
    t = (target - (un + rho * (un - unm1))) / s_out
    return ((out - t) ** 2).mean()


def loss_and_grad(theta, *args):
    th = theta.detach().clone().requires_grad_(True)
    L_ = loss(th, *args)
    L_.backward()
    return L_.item(), th.grad.detach().clone()
