"""Runs the small parity shapes through the library that PAMD_LIBRARY selects and
prints one JSON line: the worst errors against the oracle and the library's
bounds-check record.  test_gpu_debug_build runs it with the bounds-checked build.

Covered: action + gradient of every workload at its small size (single and
double precision), the LJ kernel under several tiles, windows and list
capacities (including the overflow paths, a path far from Brownian and the
per-step image shift), a batch split into two block-size classes, path updates
(captured graph and host-buffer pipeline), the multilevel sampler and the PAMD
event, and time slabs.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))


def main():
    import numpy as np
    import torch

    import oracle
    import pamd_inputs as inputs
    import paper_1907_09529_gb300 as pamd
    from _common import gpu_system, oracle_potential, rel, start_paths
    from paper_1907_09529_gb300 import timeslab

    worst = {"fp32": 0.0, "fp64": 0.0}

    def check(w, prob, paths, S, g, prec):
        S, g = S.cpu().numpy(), g.cpu()
        for q, spec in enumerate(w.systems):
            pot = oracle_potential(spec)
            for b in range(spec.n_chains):
                So, go = oracle.action_grad(pot, paths[q][b], w.D, w.beta, w.dt, nthreads=8)
                e = max(abs(S[prob.chain0[q] + b] - So) / abs(So),
                        rel(prob.view(g, q)[b].double().numpy(), go))
                worst[prec] = max(worst[prec], e)

    def run(name, prec, tune=None, env=None):
        env = env or {}
        for k, v in env.items():
            os.environ[k] = v
        pamd.release_cache()
        pamd.tune(*(tune or ()))
        w = inputs.workload(name, "small")
        prob = pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt,
                            precision=prec)
        paths = start_paths(w, prec)
        buf = prob.empty("cuda")
        for q, p in enumerate(paths):
            prob.view(buf, q).copy_(torch.from_numpy(p).to(prob.dtype))
        S, g = pamd.action_grad(prob, buf)
        torch.cuda.synchronize()
        check(w, prob, paths, S, g, prec)
        for k in env:
            os.environ.pop(k)
        pamd.tune()
        return w, prob, buf, S, g

    for name in ("ho3d", "lj108", "lj500", "ragged", "ho1d"):
        for prec in ("fp32", "fp64"):
            run(name, prec)
    for tune in ((1, 0, 0, -1.0, 0), (7, 0, 0, -1.0, 2), (64, 0, 0, -1.0, 40), (16, 0, 8, -1.0, 0)):
        run("lj500", "fp32", tune)
        run("lj108", "fp32", tune)
    run("lj500", "fp32", env={"PAMD_LJ_NO_PIPE": "1"})
    run("ragged", "fp32", env={"PAMD_LJ_PER_STEP_SHIFT": "1"})
    # systems on both sides of N = 512: two block-size classes, each with its own
    # block size and shared memory, sharing the outer-list region
    import dataclasses
    mixed = dataclasses.replace(
        inputs.workload("ragged", "small"), name="mixed",
        systems=[inputs.SystemSpec("lj", 96, 3, 40, 2), inputs.SystemSpec("lj", 530, 3, 33, 1),
                 inputs.SystemSpec("lj", 700, 3, 25, 2)])
    for prec in ("fp32", "fp64"):
        pamd.release_cache()
        prob = pamd.Problem([gpu_system(s, pamd) for s in mixed.systems], mixed.D, mixed.beta,
                            mixed.dt, precision=prec)
        paths = start_paths(mixed, prec)
        buf = prob.empty("cuda")
        for q, p in enumerate(paths):
            prob.view(buf, q).copy_(torch.from_numpy(p).to(prob.dtype))
        S, g = pamd.action_grad(prob, buf)
        torch.cuda.synchronize()
        check(mixed, prob, paths, S, g, prec)
        if prec == "fp32":  # host-buffer pipeline over the two classes
            hb, hg, hS = buf.cpu().pin_memory(), g.cpu().pin_memory(), S.cpu().pin_memory()
            pamd.path_update(prob, hb, hg, hS, 2e-7, n_updates=1, seed=1, counter=3)

    # a path far from Brownian: outer and window lists overflow
    N, T, B = 256, 40, 2
    L = (N / 0.5) ** (1.0 / 3.0)
    rng = inputs.rng(77)
    x = (inputs.fcc_lattice(N, L)[None, None] + 0.12 * rng.standard_normal((B, T + 1, 3, N)))
    x = x.astype(np.float32).astype(np.float64)
    prob = pamd.Problem([pamd.System("lj", N, 3, T, B, box=L, rc=2.5)], 1.0, 1.0, 1e-4)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(x))
    S, g = pamd.action_grad(prob, buf)
    pot = oracle.lennard_jones(L, 2.5)
    for b in range(B):
        So, go = oracle.action_grad(pot, x[b], 1.0, 1.0, 1e-4)
        worst["fp32"] = max(worst["fp32"], abs(S[b].item() - So) / So,
                            rel(prob.view(g, 0)[b].double().cpu().numpy(), go))

    # updates: captured graph, and host buffers (pipelined over chunks)
    w, prob, buf, S, g = run("ragged", "fp32")
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    pamd.path_update(prob, buf, g, S, 2e-7, n_updates=3, seed=1, counter=0, n_accepted=nacc)
    hb, hg, hS = buf.cpu().pin_memory(), g.cpu().pin_memory(), S.cpu().pin_memory()
    pamd.path_update(prob, hb, hg, hS, 2e-7, n_updates=1, seed=1, counter=9)
    # time slabs over three ranks held here
    run_ = timeslab.SlabRun(prob, timeslab.LocalComm(3))
    bufs = [timeslab.scatter(prob, buf, lp) for lp in run_.probs]
    Ss, Gs = run_.action_grad(bufs)
    run_.update(bufs, Gs, Ss, 2e-7, seed=2, counter=3)

    # multilevel sampler and PAMD events (one-line and block kernels, thread fallback)
    for (d, N, T, B) in ((1, 1, 256, 8), (3, 2, 96, 4), (1, 1, 40000, 2)):
        hp = pamd.Problem([pamd.System("harmonic", N, d, T, B)], 1.0, 1.0, 0.4, "fp32",
                          ho_exact_propagator=True)
        pb = hp.empty("cuda")
        hp.view(pb, 0).copy_(torch.randn(hp.view(pb, 0).shape, device="cuda"))
        pamd.fragment_mc(hp, pb, 2, 4, n_steps=2, seed=5, counter=1)
        from paper_1907_09529_gb300 import integrator
        integ = integrator.PamdIntegrator(hp, 8, 1, 2, 4, seed=5)
        integ.run(pb, 2)
    torch.cuda.synchronize()

    checked, count, site, index, bound = pamd._lib.pamd_debug_status()
    print(json.dumps({"worst": worst, "checked": checked, "count": count, "site": site,
                      "index": index, "bound": bound}), flush=True)


if __name__ == "__main__":
    main()
