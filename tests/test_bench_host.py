"""Host-side checks of bench.py's reference arm (the FP64 oracle timed on a
host core): one JSON line with the contract's keys on rank 0, nothing on the
other ranks; and of the per-pass roofline helper on the emulation library.
No GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r


def test_reference_arm_prints_one_contract_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_pass_rooflines_runs_every_pass_through_the_probe():
    """bench.pass_rooflines (the per-pass roofline object of the 3D line) on
    the emulation library with a host stand-in for torch: every pass of a
    cubic 3D PFC grid runs through pagd_pass_probe and gets its byte model."""
    import dataclasses

    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from paper_2204_07247_gb300 import inputs as I
    from paper_2204_07247_gb300 import pagd

    class HostTorch:
        class _A:
            def __init__(self, a):
                self.a = a

            def cuda(self):
                return self.a

        @staticmethod
        def from_numpy(a):
            return HostTorch._A(a)

    w = dataclasses.replace(I.PFC3D256, n=(64,) * 3, L=tuple(l / 4 for l in I.PFC3D256.L))
    out = bench.pass_rooflines(HostTorch, pagd, w, 6780.0, count=2, warm=1, lib=pagd.load_emulation())
    assert set(("RI", "CI", "MF", "MI")) <= set(out)
    assert out["bytes_per_point"] == {"RI": 24.1, "CI": 24.2, "MF": 8.05, "MI": 8.05}
    json.dumps(out)
