"""The learned-guess form: trajectories from the solver, training of the
spectral neural operator (sno.SNO, own CUDA forward / backward / Adam
kernels), and its evaluation through pagd_step_with_guess against the plain
extrapolated initial iterate.

A training sample is a triple (u^{n-1}, u^n, u^{n+1}) of consecutive accepted
states of one trajectory; the network learns u^{n+1} minus the extrapolation
u^n + rho (u^n - u^{n-1}) (rho = 1 at a fixed dt).
"""
from __future__ import annotations

import numpy as np

from . import inputs as I
from . import pagd
from . import sno as SB


def trajectories(torch, w, seeds, steps, skip=20):
    """[len(seeds), steps + 2, n0, n1] accepted states (FP64, device), after
    `skip` steps from u0: the first steps from white-noise data are dominated
    by stiff, fast-decaying high modes that a network with few kept modes
    cannot represent and that no later state resembles."""
    out = torch.empty((len(seeds), steps + 2) + tuple(w.n), dtype=torch.float64, device="cuda")
    for i, seed in enumerate(seeds):
        S = pagd.solver_for(w)
        S.set_state(torch.from_numpy(w.u0(seed)).cuda())
        if skip:
            S.run(w.dt, skip, w.tol)
        for k in range(steps + 2):
            if k:
                S.run(w.dt, 1, w.tol, out[i, k])
            else:
                out[i, 0].copy_(S.get_state()[0])
    return out


def scales(torch, traj):
    """Input and output scales from the data: 1 / rms(u^n - u^{n-1}) and
    rms(u^{n+1} - extrapolation)."""
    d1 = traj[:, 1:] - traj[:, :-1]
    r = traj[:, 2:] - (2 * traj[:, 1:-1] - traj[:, :-2])
    return 1.0 / float(torch.sqrt((d1 ** 2).mean())), float(torch.sqrt((r ** 2).mean()))


def batch_loss(torch, net, traj, picks, s_in, s_out):
    """Loss on fixed triples (index pairs (trajectory, k)), for validation."""
    ti = [p[0] for p in picks]
    ki = [p[1] for p in picks]
    unm1 = traj[ti, ki].contiguous()
    un = traj[ti, [k + 1 for k in ki]].contiguous()
    tgt = traj[ti, [k + 2 for k in ki]].contiguous()
    loss, _ = net.loss_grad(un, unm1, tgt, 1.0, s_in, s_out)
    return loss


def train(torch, net, traj, iters, batch, lr, s_in, s_out, seed=0):
    """Adam on random minibatches of triples; returns the loss history."""
    rng = np.random.default_rng(seed)
    nt, nk = traj.shape[0], traj.shape[1] - 2
    hist = []
    for it in range(iters):
        pick = rng.integers(0, nt * nk, size=batch)
        ti, ki = pick // nk, pick % nk
        unm1 = traj[ti, ki].contiguous()
        un = traj[ti, ki + 1].contiguous()
        tgt = traj[ti, ki + 2].contiguous()
        loss, _ = net.loss_grad(un, unm1, tgt, 1.0, s_in, s_out)
        net.adam(lr)
        hist.append(loss)
    return hist


def evaluate(torch, w, net, seeds, steps, s_in, s_out, skip=20):
    """PAGD evaluations per step and device time per step, from the
    extrapolated initial iterate (plain) and from the network's proposal
    (learned, through pagd_step_with_guess; inference included).  Both forms
    start after the same `skip` plain steps; the last of them gives the solver
    its record of the extrapolation's first direction, against which each
    proposal is judged (kept at no extra cost when its first direction is no
    larger, else the step starts over from the extrapolation)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"plain": {"evals": [], "ms": 0.0}, "learned": {"evals": [], "ms": 0.0, "used": 0}}
    for seed in seeds:
        for form in ("plain", "learned"):
            S = pagd.solver_for(w)
            S.set_state(torch.from_numpy(w.u0(seed)).cuda())
            S.run(w.dt, skip + 1, w.tol)
            out = torch.empty(w.n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                if form == "plain":
                    its, _ = S.run(w.dt, 1, w.tol, out)
                    res[form]["evals"].append(int(its[0]))
                else:
                    un, unm1, _ = S.get_state()
                    g = net.predict(un, unm1, 1.0, s_in, s_out)
                    its, _, used = S.step_with_guess(out, g, w.dt, w.tol)
                    res[form]["evals"].append(int(its))
                    res[form]["used"] += int(used)
            e1.record()
            torch.cuda.synchronize()
            res[form]["ms"] += e0.elapsed_time(e1)
    n = len(seeds) * steps
    for form in res:
        r = res[form]
        r["evals_per_step"] = float(np.mean(r["evals"]))
        r["steps_per_s"] = n / (r["ms"] / 1000.0)
        del r["evals"]
    res["learned"]["kept_fraction"] = res["learned"]["used"] / n
    return res


def batched_study(torch, w, net, s_in, s_out, seeds, steps, skip=20):
    """Member steps per second of len(seeds) instances of w advanced (a) each
    alone by the single-instance kernel from the extrapolation (plain), (b)
    together by one batched launch per step chunk (batched), and (c) together,
    one batched launch per step with every member started from the network's
    proposal (batched + learned: one batched inference per step, each guess
    judged against its member's record).  All three start from the same states
    after `skip` plain steps."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def start():
        sols = []
        for seed in seeds:
            S = pagd.solver_for(w)
            S.set_state(torch.from_numpy(w.u0(seed)).cuda())
            S.run(w.dt, skip + 1, w.tol)  # the last of these sets the record
            sols.append(S)
        return sols

    m = len(seeds)
    out = {"workload": w.name, "members": m, "steps": steps}
    sols = start()
    torch.cuda.synchronize()
    e0.record()
    ev = 0
    for S in sols:
        its, _ = S.run(w.dt, steps, w.tol)
        ev += int(np.sum(its))
    e1.record()
    torch.cuda.synchronize()
    out["plain"] = {"member_steps_per_s": m * steps / (e0.elapsed_time(e1) / 1000.0), "evals_per_step": ev / (m * steps)}
    B = pagd.Batch(start())
    torch.cuda.synchronize()
    e0.record()
    its, _, status = B.run(w.dt, steps, w.tol)
    e1.record()
    torch.cuda.synchronize()
    out["batched"] = {"member_steps_per_s": m * steps / (e0.elapsed_time(e1) / 1000.0),
                      "evals_per_step": float(its.mean()), "all_ok": bool(np.all(status == 0))}
    sols = start()
    B = pagd.Batch(sols)
    ev, kept = 0, 0
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        st = [S.get_state() for S in sols]
        un = torch.stack([s[0] for s in st])
        unm1 = torch.stack([s[1] for s in st])
        g = net.predict(un, unm1, 1.0, s_in, s_out)
        its, _, status, used = B.step_with_guess([g[i] for i in range(m)], w.dt, w.tol)
        ev += int(np.sum(its))
        kept += int(np.sum(used))
    e1.record()
    torch.cuda.synchronize()
    out["batched_learned"] = {"member_steps_per_s": m * steps / (e0.elapsed_time(e1) / 1000.0),
                              "evals_per_step": ev / (m * steps), "kept_fraction": kept / (m * steps)}
    return out


def run_study(torch, w, train_seeds, val_seeds, test_seeds, steps_train, steps_test, iters, batch=4, lr=1e-3,
              channels=16, layers=4, modes=(16, 16), batched_seeds=None):
    """Collect training and (disjoint) validation trajectories, train, and
    evaluate on test seeds disjoint from both; a dict for the benchmark line."""
    traj = trajectories(torch, w, train_seeds, steps_train)
    vtraj = trajectories(torch, w, val_seeds, max(4, batch))
    s_in, s_out = scales(torch, traj)
    nb = max(batch, len(batched_seeds or ()))
    net = SB.SNO(w.n, channels=channels, layers=layers, modes=modes, batch=nb, seed=1, bf16=True)
    val = [(i % vtraj.shape[0], i % (vtraj.shape[1] - 2)) for i in range(batch)]
    val_before = batch_loss(torch, net, vtraj, val, s_in, s_out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = train(torch, net, traj, iters, batch, lr, s_in, s_out)
    e1.record()
    torch.cuda.synchronize()
    val_after = batch_loss(torch, net, vtraj, val, s_in, s_out)
    del traj, vtraj
    ev = evaluate(torch, w, net, test_seeds, steps_test, s_in, s_out)
    if batched_seeds:
        ev["batched_forms"] = batched_study(torch, w, net, s_in, s_out, batched_seeds, steps_test)
    return {"workload": w.name, "network": f"{layers} spectral layers, {channels} channels, "
            f"{modes[0]}x{modes[1]} modes, GELU, BF16 weights with FP32 accumulation (FP32 Adam master)", "train": {"trajectories": len(train_seeds),
            "steps": steps_train, "iters": iters, "batch": batch, "ms": e0.elapsed_time(e1),
            "loss_first": hist[0], "loss_last": float(np.mean(hist[-10:])),
            "validation_seeds": list(val_seeds), "validation_loss_before": val_before,
            "validation_loss_after": val_after},
            "test": {"seeds": list(test_seeds), "steps": steps_test}, **ev}
