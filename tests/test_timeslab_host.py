"""Time-slab sharding of one long path (paper Sec. II.B: the forces of different
timesteps are independent): the driver's halo exchange, sums over ranks and
rank-0 accept broadcast, on CPU.

Each rank's slab is evaluated by the CPU oracle (the library needs a GPU): S over
the owned steps from oracle.step_actions, the gradient at the owned slices from
oracle.grad_slices, the update pieces written out from the whole-path MALA rule.
The sharded S, gradient and path updates must equal the oracle's whole-path
action_grad and mala_step on the same noise and uniforms: over two gloo ranks,
and over three slabs held by one process.
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle
import pamd_inputs as inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")

D, BETA, DT, H = 1.0, 1.0, 1e-3, 2e-5


def _whole(pamd):
    """A two-system problem: an LJ liquid (N = 64) and a 2D oscillator; T odd so
    that the slabs are uneven."""
    N = 64
    L = inputs.box_side(N, 0.85)
    return pamd.Problem([pamd.System("lj", N, 3, 23, 2, box=L, rc=min(2.5, L / 2)),
                         pamd.System("harmonic", 3, 2, 23, 2, k=0.8)], D, BETA, DT,
                        precision="fp64")


def _pots(p):
    return [oracle.lennard_jones(s.box, s.rc) if s.kind == "lj" else oracle.harmonic(s.k)
            for s in p.systems]


def _paths(p):
    """Brownian paths (FCC start for the liquid), seeded."""
    rng = inputs.rng(4242)
    out = []
    for s in p.systems:
        if s.kind == "lj":
            x0 = inputs.fcc_lattice(s.N, s.box)[None, None]
        else:
            x0 = rng.standard_normal((s.n_chains, 1, s.d, s.N))
        steps = math.sqrt(2 * D * DT) * rng.standard_normal((s.n_chains, s.T + 1, s.d, s.N))
        steps[:, 0] = 0
        out.append(x0 + np.cumsum(steps, axis=1))
    return out


class OracleBackend:
    """Evaluates one slab with the CPU oracle (slab semantics of include/pamd.h)."""

    def __init__(self, whole):
        self.pots = _pots(whole)

    @staticmethod
    def _free(s):
        return range(1, s.T + 1 - s.halo_hi)  # proposed slices: owned, not the fixed tail

    def action_grad(self, p, pos, S=None, grad=None):
        S = torch.zeros(p.n_chains, dtype=torch.float64)
        grad = torch.zeros_like(pos) if grad is None else grad
        for q, s in enumerate(p.systems):
            own = list(range(s.halo_lo, s.T + 1 - s.halo_hi))
            for b in range(s.n_chains):
                x = p.view(pos, q)[b].numpy()
                S[p.chain0[q] + b] = float(np.sum(oracle.step_actions(
                    self.pots[q], x, D, BETA, DT, list(range(s.halo_lo, s.T)))))
                g = oracle.grad_slices(self.pots[q], x, D, BETA, DT, own)
                p.view(grad, q)[b, own[0]:own[-1] + 1] = torch.from_numpy(g)
        return S, grad

    def propose(self, p, pos, grad, h, seed, counter, noise=None):
        prop = pos.clone()
        qf = torch.zeros(p.n_chains, dtype=torch.float64)
        for q, s in enumerate(p.systems):
            fr = list(self._free(s))
            x, g, z = p.view(pos, q)[:, fr], p.view(grad, q)[:, fr], p.view(noise, q)[:, fr]
            xp = x - h * g + math.sqrt(2 * h) * z
            p.view(prop, q)[:, fr] = xp
            qf[p.chain0[q]:p.chain0[q] + s.n_chains] = ((xp - x + h * g) ** 2).sum(dim=(1, 2, 3))
        return prop, qf

    def reverse(self, p, pos, prop, grad_prop, h):
        qr = torch.zeros(p.n_chains, dtype=torch.float64)
        for q, s in enumerate(p.systems):
            fr = list(self._free(s))
            x, xp, gp = p.view(pos, q)[:, fr], p.view(prop, q)[:, fr], p.view(grad_prop, q)[:, fr]
            qr[p.chain0[q]:p.chain0[q] + s.n_chains] = ((x - xp + h * gp) ** 2).sum(dim=(1, 2, 3))
        return qr

    def accept(self, p, S, S_prop, q_fwd, q_rev, h, seed, counter, log_u=None, n_accepted=None,
               log_alpha=None):
        la = (S - S_prop) - q_rev / (4 * h) + q_fwd / (4 * h)
        acc = (log_u < la).to(torch.int32)
        if n_accepted is not None:
            n_accepted += acc
        if log_alpha is not None:
            log_alpha.copy_(la)
        return acc

    def commit(self, p, pos, grad, S, prop, grad_prop, S_prop, accept):
        for q, s in enumerate(p.systems):
            for b in range(s.n_chains):
                c = p.chain0[q] + b
                if accept[c]:
                    p.view(pos, q)[b].copy_(p.view(prop, q)[b])
                    p.view(grad, q)[b].copy_(p.view(grad_prop, q)[b])
                    S[c] = S_prop[c]


def _reference(p, paths, noise, logus):
    """Whole-path oracle: S, gradient, then successive MALA steps on the same draws."""
    pots = _pots(p)
    out = {"S0": [], "g0": [], "steps": []}
    state = []
    for q, s in enumerate(p.systems):
        for b in range(s.n_chains):
            S, g = oracle.action_grad(pots[q], paths[q][b], D, BETA, DT)
            out["S0"].append(S)
            out["g0"].append(g)
            state.append([paths[q][b].copy(), S, g])
    for k, lu in enumerate(logus):
        rec = []
        c = 0
        for q, s in enumerate(p.systems):
            for b in range(s.n_chains):
                x, S, g = state[c]
                r = oracle.mala_step(pots[q], x, S, g, noise[k][q][b], lu[c], H, D, BETA, DT)
                if r["accepted"]:
                    state[c] = [r["prop"], r["S_prop"], r["grad_prop"]]
                rec.append((r["accepted"], state[c][0].copy(), state[c][1], state[c][2].copy()))
                c += 1
        out["steps"].append(rec)
    return out


def _draws(p, n):
    rng = inputs.rng(77)
    noise = [[rng.standard_normal((s.n_chains, s.T + 1, s.d, s.N)) for s in p.systems]
             for _ in range(n)]
    logus = [np.log(rng.random(p.n_chains)) for _ in range(n)]
    return noise, logus


def _whole_buf(p, arrays):
    buf = p.empty("cpu")
    for q, a in enumerate(arrays):
        p.view(buf, q).copy_(torch.from_numpy(a))
    return buf


def _run_slabs(pamd, comm, n_updates):
    """Drive the slabs this process holds; returns per held rank the owned-slice
    results (S, gradients, paths after each update) gathered into whole buffers."""
    from paper_1907_09529_gb300 import timeslab
    p = _whole(pamd)
    paths = _paths(p)
    noise, logus = _draws(p, n_updates)
    run = timeslab.SlabRun(p, comm, OracleBackend(p))
    whole = _whole_buf(p, paths)
    bufs = [timeslab.scatter(p, whole, lp) for lp in run.probs]
    S, G = run.action_grad(bufs)
    res = {"S0": [s.clone() for s in S],
           "g0": [timeslab.gather_owned(p, torch.zeros(p.span, dtype=torch.float64), lp, g)
                  for lp, g in zip(run.probs, G)], "steps": []}
    for k in range(n_updates):
        nz = [timeslab.scatter(p, _whole_buf(p, noise[k]), lp) for lp in run.probs]
        lu = [torch.from_numpy(logus[k]) for _ in run.probs]
        flags = run.update(bufs, G, S, H, noise=nz, log_u=lu)
        res["steps"].append([(f.clone(), s.clone(),
                              timeslab.gather_owned(p, torch.zeros(p.span, dtype=torch.float64), lp, b),
                              timeslab.gather_owned(p, torch.zeros(p.span, dtype=torch.float64), lp, g))
                             for f, s, lp, b, g in zip(flags, S, run.probs, bufs, G)])
    return p, paths, noise, logus, res


def _check(pamd, p, ref, per_rank, slabs):
    """per_rank: results of every rank (same structure as _run_slabs' res, one entry
    per rank); slabs[r]: rank r's local problem (to know its owned slices)."""
    from paper_1907_09529_gb300 import timeslab
    nc = p.n_chains
    for r, res in enumerate(per_rank):
        S0 = res["S0"]
        for c in range(nc):
            assert abs(float(S0[c]) - ref["S0"][c]) <= 1e-12 * abs(ref["S0"][c])
    # gradients: each rank's owned slices
    for r, res in enumerate(per_rank):
        lp = slabs[r]
        for q, s in enumerate(lp.systems):
            o = timeslab.owned_slices(s)
            g0 = p.view(res["g0"], q)
            for b in range(s.n_chains):
                c = p.chain0[q] + b
                want = ref["g0"][c][s.first_slice + o.start:s.first_slice + o.stop]
                got = g0[b, s.first_slice + o.start:s.first_slice + o.stop].numpy()
                assert np.abs(got - want).max() <= 1e-12 * np.abs(ref["g0"][c]).max()
    n_acc = 0
    for k, rec in enumerate(ref["steps"]):
        for r, res in enumerate(per_rank):
            flags, S, pos, grad = res["steps"][k]
            lp = slabs[r]
            for q, s in enumerate(lp.systems):
                o = timeslab.owned_slices(s)
                lo, hi = s.first_slice + o.start, s.first_slice + o.stop
                for b in range(s.n_chains):
                    c = p.chain0[q] + b
                    acc, x, Sw, g = rec[c]
                    assert bool(flags[c]) == acc, (k, r, c)
                    assert abs(float(S[c]) - Sw) <= 1e-12 * abs(Sw)
                    assert np.abs(p.view(pos, q)[b, lo:hi].numpy() - x[lo:hi]).max() <= 1e-12
                    assert np.abs(p.view(grad, q)[b, lo:hi].numpy() - g[lo:hi]).max() <= \
                        1e-10 * np.abs(g).max()
                    n_acc += int(acc) if r == 0 else 0
    assert 0 < n_acc < len(ref["steps"]) * nc  # both decisions occur


def test_three_slabs_in_one_process_match_the_whole_path():
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import timeslab
    comm = timeslab.LocalComm(3)
    p, paths, noise, logus, res = _run_slabs(pamd, comm, 4)
    ref = _reference(p, paths, noise, logus)
    per_rank = [{"S0": res["S0"][r], "g0": res["g0"][r],
                 "steps": [st[r] for st in res["steps"]]} for r in range(3)]
    _check(pamd, p, ref, per_rank, [timeslab.slab_problem(p, r, 3) for r in range(3)])


def test_slab_bounds_and_layout():
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import timeslab
    assert timeslab.slab_bounds(23, 3) == [0, 7, 15, 23]
    with pytest.raises(ValueError):
        timeslab.slab_bounds(2, 3)
    p = _whole(pamd)
    locs = [timeslab.slab_problem(p, r, 3) for r in range(3)]
    s0, s1, s2 = (lp.systems[0] for lp in locs)
    assert (s0.first_slice, s0.halo_lo, s0.halo_hi, s0.T) == (0, 0, 1, 7)
    assert (s1.first_slice, s1.halo_lo, s1.halo_hi, s1.T) == (6, 1, 1, 9)
    assert (s2.first_slice, s2.halo_lo, s2.halo_hi, s2.T) == (14, 1, 0, 9)
    # owned slices tile the whole path exactly once
    owned = []
    for s in (s0, s1, s2):
        o = timeslab.owned_slices(s)
        owned += list(range(s.first_slice + o.start, s.first_slice + o.stop))
    assert owned == list(range(24))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import timeslab
    import test_timeslab_host as me
    _, _, _, _, res = me._run_slabs(pamd, timeslab.TorchComm(), 3)
    out[rank] = {"S0": res["S0"][0].numpy(), "g0": res["g0"][0].numpy(),
                 "steps": [tuple(t.numpy() for t in st[0]) for st in res["steps"]]}
    dist.destroy_process_group()


def test_two_gloo_ranks_match_the_whole_path():
    import torch.multiprocessing as mp
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import timeslab
    world, port = 2, 29547
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    p = _whole(pamd)
    noise, logus = _draws(p, 3)
    ref = _reference(p, _paths(p), noise, logus)
    per_rank = []
    for r in range(world):
        d = out[r]
        per_rank.append({"S0": torch.from_numpy(d["S0"]), "g0": torch.from_numpy(d["g0"]),
                         "steps": [tuple(torch.from_numpy(a) for a in st) for st in d["steps"]]})
    _check(pamd, p, ref, per_rank, [timeslab.slab_problem(p, r, world) for r in range(world)])
