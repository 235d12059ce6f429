"""The allocation-free entry point pagd_step_static.

Callers that cannot allocate device memory when they need a step (graph
recording, a foreign device allocator, a fixed memory budget) use this entry
point: it runs the same time step on a static device array built into the
library.  Two consecutive steps through it must match the regular
workspace-based path within the tolerance the other GPU tests use.

This file sorts last so that, if it fails, a run that stops at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

from paper_2204_07247_gb300 import inputs as I
from paper_2204_07247_gb300 import pagd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,precision,tol,rel", [("pfc", "fp64", 1e-10, 1e-12),
                                                     ("fch", "fp32_mixed", 1e-8, 1e-6)])
def test_static_scratch_steps_match_workspace_path(model, precision, tol, rel):
    import torch
    torch.cuda.set_device(0)
    lib = pagd.load()
    if model == "pfc":
        n, L, args, dt, mean, scheme = (64, 64), (32 * math.pi,) * 2, (0.025,), 0.1, 0.07, "mp"
    else:
        n, L, args, dt, mean, scheme = (128, 128), (4 * math.pi,) * 2, (0.1, 0.1, 0.1, 0.0), 1e-3, -0.3, "bdf2"
    u0 = torch.from_numpy(I.noisy_field(n, mean, 0.05, 31)).cuda()

    # regular path: workspace from the caller, state kept in the solver
    ref = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    ref.set_state(u0)
    r1 = ref.empty_field()
    r2 = ref.empty_field()
    ref.step(r1, dt, tol)
    ref.step(r2, dt, tol)

    # static-scratch path: two calls in a row, the state carried by the caller
    S = pagd.Solver(model, n, L, *args, scheme=scheme, precision=precision, lib=lib)
    s1 = S.empty_field()
    s2 = S.empty_field()
    it1, res1 = S.step_static(u0, u0, 0, dt, dt, tol, s1)
    it2, res2 = S.step_static(s1, u0, 1, dt, dt, tol, s2)
    assert res1 <= tol and res2 <= tol and it1 > 0 and it2 > 0
    for a, b in ((s1, r1), (s2, r2)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b)


def test_static_scratch_rejects_grids_beyond_its_size():
    import torch
    torch.cuda.set_device(0)
    lib = pagd.load()
    S = pagd.Solver("fch", (512, 512), (4 * math.pi,) * 2, 0.1, 0.1, 0.1, 0.0, lib=lib)
    u = S.empty_field()
    with pytest.raises(pagd.PagdError) as e:
        S.step_static(u, u, 0, 1e-3, 1e-3, 1e-8, S.empty_field())
    assert e.value.status == 1 and "static scratch" in str(e.value)
