"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: only the random initial fields
(splitmix64 counter stream) and the named workload settings.  Both the CUDA path
and the CPU oracle receive the same host arrays from here.

u0(x) = mean + amp * U(-1, 1), drawn independently per grid point, row-major
over the grid (last axis fastest).  U is the top 53 bits of
splitmix64(seed + (i + 1) * 0x9E3779B97F4A7C15), the published SplitMix64
finaliser of Steele, Lea and Flood (2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of a SplitMix64 stream started at ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.arange(1, count + 1, dtype=np.uint64) * _GAMMA)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """U[0, 1) doubles from the top 53 bits of the stream."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def noisy_field(shape, mean: float, amp: float, seed: int) -> np.ndarray:
    """mean + amp * U(-1, 1) per grid point, float64, C order."""
    n = int(np.prod(shape))
    u = 2.0 * uniform01(seed, n) - 1.0
    return (mean + amp * u).reshape(shape)


PAPER_ETA = tuple(math.sqrt(0.1 + 0.475 * j) for j in range(5))


@dataclass
class Workload:
    """A named synthetic workload: model, grid, parameters, scheme and solver."""
    name: str
    model: str            # "pfc" or "fch"
    n: tuple              # grid points per axis, last axis fastest
    L: tuple              # domain lengths
    eps: float
    eta1: float = 0.0
    eta2: float = 0.0
    tau: float = 0.0
    M: float = 1.0
    scheme: str = "bdf2"  # bdf2 | mp | lbdf2 | lmp
    precision: str = "fp64"  # fp64 | fp32_mixed
    dt: float = 0.1
    steps: int = 100
    tol: float = 1e-10
    mean: float = 0.0
    amp: float = 0.05
    seeds: tuple = (1, 2, 3, 4)
    s: float = 0.9
    eta: tuple = PAPER_ETA
    max_iter: int = 1000

    def u0(self, seed: int) -> np.ndarray:
        return noisy_field(self.n, self.mean, self.amp, seed)


FOURPI = 4.0 * math.pi

# PFC 2D 64x64 on [0, 32 pi]^2, eps = 0.025, u0 = 0.07 + 0.05 U(-1,1), MP,
# dt = 0.1, 100 steps, FP64, tol 1e-10.
PFC64 = Workload("pfc2d_64_mp_fp64", "pfc", (64, 64), (32 * math.pi, 32 * math.pi), eps=0.025,
                 scheme="mp", precision="fp64", dt=0.1, steps=100, tol=1e-10, mean=0.07, amp=0.05)

# FCH 2D 256x256 on [0, 4 pi]^2, W = (u^2-1)^2/4 (tau = 0), eps = 0.1,
# eta1 = eta2 = eps, u0 = -0.3 + 0.05 U(-1,1), BDF2 (fully implicit, FP32
# iterations with FP64 norms) beside LBDF2, dt = 1e-3, 1000 steps, tol 1e-8.
FCH256 = Workload("fch2d_256_bdf2_fp32mixed", "fch", (256, 256), (FOURPI, FOURPI), eps=0.1,
                  eta1=0.1, eta2=0.1, tau=0.0, scheme="bdf2", precision="fp32_mixed", dt=1e-3,
                  steps=1000, tol=1e-8, mean=-0.3, amp=0.05)

# PFC 3D 256^3 on [0, 64 pi]^3, eps = 0.3, u0 = -0.25 + 0.1 U(-1,1), BDF2,
# dt = 0.5, 200 steps, FP32 iterations with FP64 norms, tol 1e-8; two seeds
# advanced together as one batch.
PFC3D256 = Workload("pfc3d_256_bdf2_fp32mixed", "pfc", (256, 256, 256), (64 * math.pi,) * 3, eps=0.3,
                    scheme="bdf2", precision="fp32_mixed", dt=0.5, steps=200, tol=1e-8, mean=-0.25,
                    amp=0.1, seeds=(1, 2))

# FCH 2D 512x512 on [0, 4 pi]^2, parameters as the 256^2 workload (the
# learned-initial-iterate workload).
FCH512 = Workload("fch2d_512_bdf2_fp32mixed", "fch", (512, 512), (FOURPI, FOURPI), eps=0.1, eta1=0.1, eta2=0.1,
                  tau=0.0, scheme="bdf2", precision="fp32_mixed", dt=1e-3, steps=2000, tol=1e-8, mean=-0.3,
                  amp=0.05)

WORKLOADS = {w.name: w for w in (PFC64, FCH256, PFC3D256, FCH512)}


@dataclass
class BatchWorkload:
    """Independent instances advanced together (one dt, step count and tol)."""
    name: str
    members: list
    dt: float
    steps: int
    tol: float

    def u0s(self):
        return [m.u0(m.seeds[0]) for m in self.members]


def pfc_batch(sizes=(128, 256, 512), per_size=32, seed0=100, steps=500) -> BatchWorkload:
    """Uneven PFC batch: per_size instances at each N in sizes, N x N points on
    [0, N pi / 4]^2 (h = pi / 4), MP, FP32-mixed, dt = 0.1, tol 1e-8.  Instance
    i (sizes in order) has seed seed0 + i: eps ~ U(0.02, 0.3) and
    mean ~ U(0.05, 0.2) are the first two draws of the stream seed0 + i + 2^32,
    and u0 = mean + 0.05 U(-1, 1) comes from the stream seed0 + i."""
    members = []
    i = 0
    for N in sizes:
        for _ in range(per_size):
            seed = seed0 + i
            a, b = uniform01(seed + (1 << 32), 2)
            eps = 0.02 + 0.28 * float(a)
            mean = 0.05 + 0.15 * float(b)
            L = N * math.pi / 4.0
            members.append(Workload(f"pfc2d_{N}_mp_fp32mixed_i{i}", "pfc", (N, N), (L, L), eps=eps,
                                    scheme="mp", precision="fp32_mixed", dt=0.1, steps=steps, tol=1e-8,
                                    mean=mean, amp=0.05, seeds=(seed,)))
            i += 1
    name = "pfc2d_batch{}_{}_mp_fp32mixed".format(len(members), "_".join(str(N) for N in sizes))
    return BatchWorkload(name, members, dt=0.1, steps=steps, tol=1e-8)


# 96 PFC instances, 32 each at 128^2, 256^2 and 512^2, 500 steps
PFC_BATCH96 = pfc_batch()


# Seeded test fields for sketching the difference of two states: with w_j
# iid U(-1, 1) per point, E[(sum_x e(x) w_j(x))^2] = |e|^2 / 3, so the mean of
# 3 p_j^2 over the fields estimates the squared L2 norm of e = u - v from the
# projections p_j of u and of v alone (a Johnson-Lindenstrauss sketch).
SKETCH_SEED = 0x5EED0000
SKETCH_COUNT = 128


def sketch(u: np.ndarray, count: int = SKETCH_COUNT, seed: int = SKETCH_SEED) -> np.ndarray:
    """Projections sum_x u(x) w_j(x) of a field onto `count` seeded U(-1, 1) fields."""
    flat = np.ascontiguousarray(u, dtype=np.float64).ravel()
    out = np.empty(count)
    for j in range(count):
        out[j] = float(np.dot(flat, 2.0 * uniform01(seed + j, flat.size) - 1.0))
    return out


def sketch_rel_l2(p_u: np.ndarray, p_v: np.ndarray, sumsq_v: float) -> float:
    """Estimated |u - v|_2 / |v|_2 from the two sketches and sum_x v(x)^2."""
    d = np.asarray(p_u, dtype=np.float64) - np.asarray(p_v, dtype=np.float64)
    return math.sqrt(3.0 * float(np.mean(d * d)) / sumsq_v)
