"""GPU parity of the learned-guess network (include/pagd_sno.h): the CUDA
forward pass, loss and parameter gradient (own backward kernels) against the
PyTorch-CPU float64 oracle (oracle/sno_oracle.py), and one Adam update against
its closed form.  FP32 kernels: 1e-5 relative on the output, 1e-4 on the
gradient."""
import numpy as np
import pytest
import torch

from oracle import sno_oracle as S
from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import sno as SB

pytestmark = pytest.mark.gpu

CONFIGS = [((32, 64), 4, 2, (4, 3), 2), ((64, 32), 6, 3, (8, 5), 3)]


def _inputs(n, B, seed):
    un = np.stack([I.noisy_field(n, -0.3, 0.3, seed + b) for b in range(B)])
    unm1 = un + 0.01 * np.stack([I.noisy_field(n, 0.0, 1.0, seed + 50 + b) for b in range(B)])
    target = un + 0.02 * np.stack([I.noisy_field(n, 0.0, 1.0, seed + 90 + b) for b in range(B)])
    return un, unm1, target


@pytest.mark.parametrize("cfg", CONFIGS)
def test_forward_loss_and_gradient_match_oracle(cfg):
    n, C, L, modes, B = cfg
    net = SB.SNO(n, channels=C, layers=L, modes=modes, batch=B, seed=3)
    # make the bias and projection terms nonzero so every gradient is exercised
    net.params += 0.05 * torch.from_numpy((2 * I.uniform01(7, net.nparams) - 1).astype(np.float32)).cuda()
    un, unm1, target = _inputs(n, B, 11)
    rho, s_in, s_out = 1.0, 20.0, 0.02
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    theta = net.params.double().cpu()
    guess = net.predict(d(un), d(unm1), rho, s_in, s_out).cpu()
    ref, _ = S.forward(theta, torch.from_numpy(un), torch.from_numpy(unm1), rho, s_in, s_out, C, L, *modes)
    assert torch.linalg.norm(guess - ref) <= 1e-5 * torch.linalg.norm(ref)
    loss, grad = net.loss_grad(d(un), d(unm1), d(target), rho, s_in, s_out)
    rl, rg = S.loss_and_grad(theta, torch.from_numpy(un), torch.from_numpy(unm1), torch.from_numpy(target),
                             rho, s_in, s_out, C, L, *modes)
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    g = grad.double().cpu()
    assert torch.linalg.norm(g - rg) <= 1e-4 * torch.linalg.norm(rg)


def test_adam_step_closed_form():
    net = SB.SNO((32, 32), channels=2, layers=1, modes=(2, 2), batch=1, seed=1)
    p0 = net.params.clone()
    net.grad.copy_(torch.linspace(-1, 1, net.nparams, device="cuda"))
    net.adam(1e-2)
    g = net.grad.double()
    m = 0.1 * g
    v = 0.001 * g * g
    ref = p0.double() - 1e-2 * (m / 0.1) / (torch.sqrt(v / 0.001) + 1e-8)
    assert torch.allclose(net.params.double(), ref, atol=1e-6)
