"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method (no forces, residuals, actions or
gradients): only workload shapes, lattice starting points and random draws.
Both the CPU oracle and the CUDA library are fed from here, and neither side
imports the other.

Workloads are shaped like the paper's model systems (Sec. IV): a Brownian
harmonic oscillator (k = beta = gamma = 1) and a Lennard-Jones liquid with the
cut-and-force-shifted potential of Eq. (11), here at reduced density 0.85,
T* = 1 and cutoff 2.5 sigma in a periodic cubic box.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 1907


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """One system: `n_chains` independent paths of `T` steps (T+1 slices)."""
    kind: str            # "harmonic" or "lj"
    N: int               # particles
    d: int               # Cartesian dimensions
    T: int               # steps (residuals / force evaluations); slices = T+1
    n_chains: int = 1
    k: float = 1.0       # harmonic constant
    density: float = 0.85
    rc: float = 2.5      # requested LJ cutoff (sigma units)
    eps: float = 1.0
    sigma: float = 1.0

    @property
    def box(self) -> float:
        return box_side(self.N, self.density) if self.kind == "lj" else 0.0

    @property
    def rc_eff(self) -> float:
        """Cutoff used: min(rc, L/2), so that only the nearest image can interact."""
        return min(self.rc, 0.5 * self.box) if self.kind == "lj" else 0.0

    @property
    def units(self) -> int:
        """Particle-timeslices of one action evaluation (N per step per chain)."""
        return self.N * self.T * self.n_chains


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    systems: List[SystemSpec]
    D: float = 1.0
    beta: float = 1.0
    dt: float = 1e-4
    init: str = "euler"          # "euler" (FCC/x0 + EM) or "gaussian" (i.i.d. per slice)
    n_updates: int = 1
    seed: int = SEED_BASE
    note: str = ""

    @property
    def units(self) -> int:
        return sum(s.units for s in self.systems)


def box_side(N: int, density: float) -> float:
    return (N / density) ** (1.0 / 3.0)


def fcc_lattice(N: int, box: float) -> np.ndarray:
    """First N sites of an m^3 FCC lattice filling the box, m = ceil((N/4)^(1/3)).

    Returns positions as [3][N] float64 inside [0, box)."""
    m = max(1, math.ceil((N / 4.0) ** (1.0 / 3.0) - 1e-12))
    while 4 * m ** 3 < N:
        m += 1
    a = box / m
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    sites = []
    for ix in range(m):
        for iy in range(m):
            for iz in range(m):
                for b in basis:
                    sites.append((np.array([ix, iy, iz], dtype=np.float64) + b + 0.25) * a)
                    if len(sites) == N:
                        return np.ascontiguousarray(np.array(sites).T)
    return np.ascontiguousarray(np.array(sites[:N]).T)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def normals(seed: int, shape) -> np.ndarray:
    return rng(seed).standard_normal(shape)


def gaussian_path(seed: int, B: int, T: int, d: int, N: int, var: float) -> np.ndarray:
    """Every slice i.i.d. N(0, var): [B][T+1][d][N]."""
    return normals(seed, (B, T + 1, d, N)) * math.sqrt(var)


def ragged_lj_systems(seed: int, n_systems: int = 32, N_range=(64, 864), T_range=(1024, 32768),
                      density: float = 0.85, n_chains: int = 1) -> List[SystemSpec]:
    """LJ systems with N and T drawn uniformly from the given integer ranges."""
    g = rng(seed)
    Ns = g.integers(N_range[0], N_range[1] + 1, size=n_systems)
    Ts = g.integers(T_range[0], T_range[1] + 1, size=n_systems)
    return [SystemSpec("lj", int(n), 3, int(t), n_chains, density=density)
            for n, t in zip(Ns, Ts)]


# ---------------------------------------------------------------- the five workloads
def workload(name: str, scale: Optional[str] = None) -> Workload:
    """The five configurations.  scale="small" shrinks T and the batch so that
    the CPU oracle finishes in seconds while still spanning several tiles."""
    small = scale == "small"
    s = SEED_BASE
    if name == "ho1d":
        # 1D harmonic oscillator, T = 1024, FP64 plain path, EM from x0 = 0.
        return Workload("ho1d", [SystemSpec("harmonic", 1, 1, 1024, 1)], D=1.0, beta=1.0,
                        dt=0.01, init="euler", n_updates=1000, seed=s + 1)
    if name == "ho3d":
        T = 4096 + 37 if small else 2 ** 20
        B = 3 if small else 64
        return Workload("ho3d", [SystemSpec("harmonic", 1, 3, T, B)], D=1.0, beta=1.0,
                        dt=0.005, init="gaussian", seed=s + 2)
    if name == "lj108":
        T = 160 if small else 4096
        return Workload("lj108", [SystemSpec("lj", 108, 3, T, 1)], D=1.0, beta=1.0, dt=1e-4,
                        init="euler", seed=s + 3)
    if name == "lj500":
        T = 72 if small else 16384
        B = 2 if small else 8
        return Workload("lj500", [SystemSpec("lj", 500, 3, T, B)], D=1.0, beta=1.0, dt=1e-4,
                        init="euler", seed=s + 4)
    if name == "ragged":
        if small:
            systems = ragged_lj_systems(s + 5, n_systems=5, N_range=(64, 300), T_range=(24, 90))
        else:
            systems = ragged_lj_systems(s + 5)
        return Workload("ragged", systems, D=1.0, beta=1.0, dt=1e-4, init="euler",
                        n_updates=100, seed=s + 5)
    if name == "ho_pamd":
        # The oscillator of Sec. IV.A integrated by the PAMD loop of Fig. 2 with the
        # multilevel sampler, in the shape of the paper's Simulation 3
        # (dt = 0.4, N_path = 4096, N_sample = 1, N_shift = 64, levels 4..8); the
        # benchmark runs it with the exact propagator and straight-line regrowth.
        B = 8 if small else 16384
        T = 256 if small else 4096
        return Workload("ho_pamd", [SystemSpec("harmonic", 1, 1, T, B)], D=1.0, beta=1.0,
                        dt=0.4, init="gaussian", seed=s + 6,
                        note="n_sample=1 n_shift=64 l_min=4 l_max=8")
    raise KeyError(name)


WORKLOADS = ("ho1d", "ho3d", "lj108", "lj500", "ragged", "ho_pamd")


def initial_positions(spec: SystemSpec, seed: int) -> np.ndarray:
    """x_0 for every chain, [B][d][N]: FCC for LJ (all chains alike), 0 for the oscillator."""
    if spec.kind == "lj":
        x0 = fcc_lattice(spec.N, spec.box)
        return np.repeat(x0[None], spec.n_chains, axis=0)
    return np.zeros((spec.n_chains, spec.d, spec.N))


def euler_noise(spec: SystemSpec, seed: int, T: Optional[int] = None) -> np.ndarray:
    """Standard normals xi[B][T][d][N] for the Euler-Maruyama start paths."""
    T = spec.T if T is None else T
    return normals(seed, (spec.n_chains, T, spec.d, spec.N))
