"""The learned initial iterate end to end on a small FCH workload (128^2):
trajectories from the solver, training with the network's own kernels (BF16
weights, FP32 accumulation and FP32 Adam master), then steps through
pagd_step_with_guess.  The test checks that the weights are BF16 numbers, that
training lowers the loss on held-out trajectories, that every learned step
converges and lands where the plain solver lands (within the FP32-mixed bound,
the network only moves the start), and that a kept guess costs no evaluation
beyond its own (the solver judges it against its record of the
extrapolation's first direction instead of probing both); it prints what the
network gains in PAGD evaluations per step."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import learned as LR
from paper_2204_07247_gb300 import pagd
from paper_2204_07247_gb300 import sno as SB

pytestmark = pytest.mark.gpu


def test_learned_guess_trains_and_keeps_the_solution():
    w = dataclasses.replace(I.FCH512, n=(128, 128), name="fch2d_128_bdf2_fp32mixed")
    traj = LR.trajectories(torch, w, [1000, 1001, 1002], 24)
    vtraj = LR.trajectories(torch, w, [2000], 8)
    s_in, s_out = LR.scales(torch, traj)
    net = SB.SNO(w.n, channels=8, layers=2, modes=(8, 8), batch=4, seed=1, bf16=True)
    assert torch.equal(net.params, net.params.to(torch.bfloat16).to(torch.float32))
    val = [(0, 0), (0, 2), (0, 4), (0, 6)]
    before = LR.batch_loss(torch, net, vtraj, val, s_in, s_out)
    LR.train(torch, net, traj, 150, 4, 1e-3, s_in, s_out)
    after = LR.batch_loss(torch, net, vtraj, val, s_in, s_out)
    print(f"held-out loss: {before:.4f} before training, {after:.4f} after")
    assert after < before
    assert torch.equal(net.params, net.params.to(torch.bfloat16).to(torch.float32))
    # learned steps land where the plain solver lands
    S1, S2 = pagd.solver_for(w), pagd.solver_for(w)
    u0 = torch.from_numpy(w.u0(7)).cuda()
    S1.set_state(u0)
    S2.set_state(u0)
    S1.run(w.dt, 3, w.tol)
    S2.run(w.dt, 3, w.tol)
    a = torch.empty(w.n, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    evals_plain, evals_learned, used = [], [], 0
    for _ in range(6):
        its, _ = S1.run(w.dt, 1, w.tol, a)
        evals_plain.append(int(its[0]))
        un, unm1, _ = S2.get_state()
        g = net.predict(un, unm1, 1.0, s_in, s_out)
        it2, res, u = S2.step_with_guess(b, g, w.dt, w.tol)
        evals_learned.append(it2)
        used += int(u)
        assert res <= w.tol
        assert float(torch.linalg.norm(a - b)) <= 1e-6 * float(torch.linalg.norm(a))
    print(f"PAGD evaluations per step: plain {np.mean(evals_plain):.2f}, "
          f"learned {np.mean(evals_learned):.2f} (guess kept in {used} of 6 steps)")
    # the solver held a record from the plain steps, so no step paid a second
    # probe: a kept guess costs its own first evaluation only, a rejected one
    # that one more
    assert np.mean(evals_learned) <= np.mean(evals_plain) + 1.0
