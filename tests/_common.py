"""Shared test plumbing: turn the seeded workloads of pamd_inputs into inputs for
both the CPU oracle and the CUDA library (neither imports the other)."""
from __future__ import annotations

import numpy as np

import oracle
import pamd_inputs as inputs


def oracle_potential(spec):
    if spec.kind == "lj":
        return oracle.lennard_jones(spec.box, spec.rc_eff, spec.eps, spec.sigma)
    return oracle.harmonic(spec.k)


def gpu_system(spec, pamd):
    if spec.kind == "lj":
        return pamd.System("lj", spec.N, spec.d, spec.T, spec.n_chains, box=spec.box,
                           rc=spec.rc_eff, eps=spec.eps, sigma=spec.sigma)
    return pamd.System("harmonic", spec.N, spec.d, spec.T, spec.n_chains, k=spec.k)


def start_paths(w, precision="fp32", nthreads=0):
    """Seeded start paths of every system of workload w: list of [B][T+1][d][N]
    float64 arrays (values already rounded to float32 for fp32).  Euler-Maruyama
    starts are generated by the oracle only."""
    out = []
    f32 = precision == "fp32"
    for q, spec in enumerate(w.systems):
        seed = w.seed * 1000 + q
        if w.init == "gaussian":
            p = inputs.gaussian_path(seed, spec.n_chains, spec.T, spec.d, spec.N,
                                     1.0 / (w.beta * spec.k))
            if f32:
                p = p.astype(np.float32).astype(np.float64)
        else:
            x0 = inputs.initial_positions(spec, seed)
            xi = inputs.euler_noise(spec, seed + 500)
            p = oracle.euler_batch(oracle_potential(spec), x0, xi, w.D, w.beta, w.dt,
                                   store_f32=f32, nthreads=nthreads)
        out.append(p)
    return out


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
