"""Time-slab sharding of long paths over processes.

The forces along a path are independent across timesteps (paper Sec. II.B; the
method's premise is one processor per timestep, Sec. III), so one long path
splits into contiguous slabs of steps, one per rank.  Rank k of K owns steps
[s_k, s_{k+1}), s_k = floor(k T / K), and slices [s_k, s_{k+1}) of every chain
(the last rank also slice T).  It holds the whole path's slices
[s_k - h, s_{k+1}] (h = 1 for k > 0): one halo slice on each inner edge
(``pamd_system``'s time-slab fields in ``include/pamd.h``).

An evaluation of S and its gradient exchanges the halo slices with the two
neighbours (positions only: the residual of the step before a slab is formed
again from its halo slice, one extra force evaluation per slab and chain), has
each rank evaluate its slab with the library, and sums the parts of S over the
ranks in double precision.  A path update -- the whole-path Metropolis-adjusted
Langevin step that consumes the gradient -- runs in the library's pieces:
proposal on the owned slices (the whole path's noise stream), exchange of the
proposal's halo slices, S and gradient of the proposal, reverse term, one sum
over the ranks of (S', q_fwd, q_rev), accept decisions taken on rank 0 and
broadcast, commit.  With the same seed and counter the sharded run samples the
chain the single-process update does: positions and owned gradients are bitwise
the same; S agrees up to the order of its double-precision sums.

Communication goes through a small interface with two implementations:
``TorchComm`` (one slab per process over torch.distributed: NCCL for CUDA
tensors, gloo for CPU ones) and ``LocalComm`` (several slabs in one process, run
in lockstep; sums in rank order).  The slab evaluator is the library
(``LibraryBackend``); the interface lets a test substitute another evaluator.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import torch

from . import Problem, System, action_grad as _action_grad
from . import mala_accept, mala_commit, mala_propose, mala_reverse


def slab_bounds(T: int, world: int) -> List[int]:
    """Step boundaries s_0 = 0 < s_1 < ... < s_K = T of K slabs."""
    if world < 1 or T < world:
        raise ValueError(f"cannot split {T} steps into {world} slabs of at least one step")
    return [(k * T) // world for k in range(world + 1)]


def slab_system(s: System, rank: int, world: int) -> System:
    """The local system of rank `rank`: its owned slices plus the halo slices."""
    if s.first_slice or s.halo_lo or s.halo_hi:
        raise ValueError("slab_system expects a whole-path system")
    b = slab_bounds(s.T, world)
    lo, hi = b[rank], b[rank + 1]
    h_lo = 1 if rank > 0 else 0
    h_hi = 1 if rank < world - 1 else 0
    return dataclasses.replace(s, T=hi - lo + h_lo, first_slice=lo - h_lo, halo_lo=h_lo,
                               halo_hi=h_hi)


def slab_problem(whole: Problem, rank: int, world: int) -> Problem:
    return Problem([slab_system(s, rank, world) for s in whole.systems], whole.D, whole.beta,
                   whole.dt, precision=whole.precision)


def owned_slices(s: System) -> slice:
    """Local slice indices this rank owns (its gradient there is the whole path's)."""
    return slice(s.halo_lo, s.T + 1 - s.halo_hi)


def scatter(whole: Problem, buf: torch.Tensor, local: Problem, out: Optional[torch.Tensor] = None):
    """Copy a rank's slices (owned and halo) out of a whole-path buffer."""
    if out is None:
        out = local.empty(buf.device)
    for q, s in enumerate(local.systems):
        local.view(out, q).copy_(whole.view(buf, q)[:, s.first_slice:s.first_slice + s.T + 1])
    return out


def gather_owned(whole: Problem, out: torch.Tensor, local: Problem, buf: torch.Tensor):
    """Write a rank's owned slices into a whole-path buffer (tests, checkpoints)."""
    for q, s in enumerate(local.systems):
        o = owned_slices(s)
        whole.view(out, q)[:, s.first_slice + o.start:s.first_slice + o.stop].copy_(
            local.view(buf, q)[:, o])
    return out


class LibraryBackend:
    """Evaluates one slab with the CUDA library."""

    def action_grad(self, p: Problem, pos, S=None, grad=None):
        return _action_grad(p, pos, S, grad)

    def propose(self, p: Problem, pos, grad, h, seed, counter, noise=None):
        return mala_propose(p, pos, grad, h, seed, counter, noise)

    def reverse(self, p: Problem, pos, prop, grad_prop, h):
        return mala_reverse(p, pos, prop, grad_prop, h)

    def accept(self, p: Problem, S, S_prop, q_fwd, q_rev, h, seed, counter, log_u=None,
               n_accepted=None, log_alpha=None):
        return mala_accept(p, S, S_prop, q_fwd, q_rev, h, seed, counter, log_u, n_accepted,
                           log_alpha)

    def commit(self, p: Problem, pos, grad, S, prop, grad_prop, S_prop, accept):
        mala_commit(p, pos, grad, S, prop, grad_prop, S_prop, accept)


class TorchComm:
    """One slab per process over torch.distributed (default group)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.ranks = [self.rank]

    def exchange(self, to_left: Sequence, to_right: Sequence):
        """to_left[0] goes to rank - 1, to_right[0] to rank + 1; returns what the
        left and right neighbours sent this way ([None] at the ends).  The sends
        and receives are posted as one batch: NCCL runs the point-to-point
        operations between two ranks in the order they are posted, so posting
        them one by one (receive, then send, on both sides) would wait forever."""
        d, r = self.dist, self.rank
        ops, from_left, from_right = [], None, None
        if r > 0:
            from_left = torch.empty_like(to_left[0])
            ops.append(d.P2POp(d.irecv, from_left, r - 1))
            ops.append(d.P2POp(d.isend, to_left[0].contiguous(), r - 1))
        if r < self.world - 1:
            from_right = torch.empty_like(to_right[0])
            ops.append(d.P2POp(d.irecv, from_right, r + 1))
            ops.append(d.P2POp(d.isend, to_right[0].contiguous(), r + 1))
        if ops:
            for w in d.batch_isend_irecv(ops):
                w.wait()
        return [from_left], [from_right]

    def allreduce_sum(self, ts: Sequence[torch.Tensor]):
        self.dist.all_reduce(ts[0], op=self.dist.ReduceOp.SUM)
        return [ts[0]]

    def broadcast0(self, ts: Sequence[torch.Tensor]):
        self.dist.broadcast(ts[0], src=0)
        return [ts[0]]


class LocalComm:
    """All `world` slabs in this process, run in lockstep (sums in rank order)."""

    def __init__(self, world: int):
        self.world = world
        self.rank = 0
        self.ranks = list(range(world))

    def exchange(self, to_left: Sequence, to_right: Sequence):
        W = self.world
        from_left = [None] + [to_right[k - 1].clone() for k in range(1, W)]
        from_right = [to_left[k + 1].clone() for k in range(W - 1)] + [None]
        return from_left, from_right

    def allreduce_sum(self, ts: Sequence[torch.Tensor]):
        total = ts[0].clone()
        for t in ts[1:]:
            total += t
        for t in ts:
            t.copy_(total)
        return list(ts)

    def broadcast0(self, ts: Sequence[torch.Tensor]):
        for t in ts[1:]:
            t.copy_(ts[0])
        return list(ts)


class SlabRun:
    """The slabs of one whole-path problem that this process holds."""

    def __init__(self, whole: Problem, comm, backend=None):
        self.whole = whole
        self.comm = comm
        self.backend = backend or LibraryBackend()
        self.probs = [slab_problem(whole, r, comm.world) for r in comm.ranks]

    # ---------------------------------------------------------------- halos
    def _edge(self, p: Problem, buf, first: bool):
        parts = []
        for q, s in enumerate(p.systems):
            o = owned_slices(s)
            t = o.start if first else o.stop - 1
            parts.append(p.view(buf, q)[:, t].reshape(-1))
        return torch.cat(parts)

    def exchange(self, bufs: Sequence[torch.Tensor]):
        """Fill every halo slice from the neighbour that owns it."""
        to_left = [self._edge(p, b, True) for p, b in zip(self.probs, bufs)]
        to_right = [self._edge(p, b, False) for p, b in zip(self.probs, bufs)]
        from_left, from_right = self.comm.exchange(to_left, to_right)
        for p, b, fl, fr in zip(self.probs, bufs, from_left, from_right):
            for src, first in ((fl, True), (fr, False)):
                if src is None:
                    continue
                off = 0
                for q, s in enumerate(p.systems):
                    v = p.view(b, q)
                    t = 0 if first else s.T
                    n = s.n_chains * s.d * s.N
                    v[:, t].copy_(src[off:off + n].view(s.n_chains, s.d, s.N))
                    off += n

    # ---------------------------------------------------------------- action
    def action_grad(self, bufs: Sequence[torch.Tensor], grads=None, exchange: bool = True):
        """Whole-path S of every chain (the same tensor values on every rank) and each
        slab's gradient at its owned slices."""
        if exchange:
            self.exchange(bufs)
        S, G = [], []
        for k, (p, b) in enumerate(zip(self.probs, bufs)):
            s_part, g = self.backend.action_grad(p, b, None, None if grads is None else grads[k])
            S.append(s_part)
            G.append(g)
        return self.comm.allreduce_sum(S), G

    # ---------------------------------------------------------------- update
    def update(self, bufs, grads, S, h: float, seed: int = 0, counter: int = 0, noise=None,
               log_u=None, n_accepted=None, log_alpha=None):
        """One whole-path Metropolis-adjusted Langevin update of every chain, in
        place (bufs, grads, S: per local slab; halos of bufs current on entry)."""
        be = self.backend
        props, qf = [], []
        for k, (p, b, g) in enumerate(zip(self.probs, bufs, grads)):
            pr, q = be.propose(p, b, g, h, seed, counter, None if noise is None else noise[k])
            props.append(pr)
            qf.append(q)
        self.exchange(props)
        Sp, gprops = [], []
        for p, pr in zip(self.probs, props):
            s_part, g = be.action_grad(p, pr)
            Sp.append(s_part)
            gprops.append(g)
        qr = [be.reverse(p, b, pr, gp, h) for p, b, pr, gp in zip(self.probs, bufs, props, gprops)]
        sums = self.comm.allreduce_sum([torch.cat([a, b, c]) for a, b, c in zip(Sp, qf, qr)])
        nc = self.whole.n_chains
        flags = []
        for k, (p, tot) in enumerate(zip(self.probs, sums)):
            Sp[k], qf[k], qr[k] = tot[:nc], tot[nc:2 * nc], tot[2 * nc:]
            flags.append(be.accept(p, S[k], Sp[k], qf[k], qr[k], h, seed, counter,
                                   None if log_u is None else log_u[k],
                                   None if n_accepted is None else n_accepted[k],
                                   None if log_alpha is None else log_alpha[k]))
        mine = [f.clone() for f in flags]
        flags = self.comm.broadcast0(flags)  # rank 0's decisions for every rank
        for m, f in zip(mine, flags):
            if not torch.equal(m, f):
                raise RuntimeError("accept decisions differ between ranks")
        for p, b, g, s, pr, gp, sp, f in zip(self.probs, bufs, grads, S, props, gprops, Sp, flags):
            be.commit(p, b, g, s, pr, gp, sp, f)
        return flags
