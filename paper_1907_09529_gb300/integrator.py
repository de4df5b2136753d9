"""Path-accelerated MD integration loop (paper Fig. 2) for harmonic systems.

Every shifting event runs n_sample multilevel sliding-and-sampling Monte Carlo
steps on each chain's path (Sec. III), then shifts the path by n_shift steps:
the n_shift slices behind the tail become the next points of the integrated
trajectory, and the path is regrown at the nose with free-particle steps (the
sampler's trial distribution).  All of it runs in the library's kernels; this
module only sequences the calls and the double buffer.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import Problem, _check_buf, _ptr, _stream, pamd_event, pamd_shift_regenerate


def shift_regenerate(p: Problem, pos: torch.Tensor, pos_out: torch.Tensor, n_shift: int,
                     traj: Optional[torch.Tensor] = None, seed: int = 0, counter: int = 0,
                     noise: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """One shift of every chain (Fig. 2B); returns the trajectory points
    [sum over systems of chains * n_shift * dim * N] (flat)."""
    _check_buf(p, pos, "pos")
    _check_buf(p, pos_out, "pos_out")
    n = sum(s.n_chains * n_shift * s.d * s.N for s in p.systems)
    if traj is None:
        traj = torch.empty(n, dtype=p.dtype, device=pos.device)
    pamd_shift_regenerate(p.ref, _ptr(pos), _ptr(pos_out), int(n_shift), _ptr(traj), int(seed),
                          int(counter), _ptr(noise), _stream(pos, stream))
    return traj


def event(p: Problem, pos: torch.Tensor, pos_out: torch.Tensor, n_sample: int, n_shift: int,
          l_min: int, l_max: int, traj: torch.Tensor, n_accepted: torch.Tensor,
          n_proposed: torch.Tensor, seed: int = 0, event: int = 0, stream=None) -> None:
    """One shifting event (Fig. 2): n_sample MC steps on `pos`, then the shifted
    and regrown paths into `pos_out` and the trajectory points into `traj`."""
    _check_buf(p, pos, "pos")
    _check_buf(p, pos_out, "pos_out")
    pamd_event(p.ref, _ptr(pos), _ptr(pos_out), int(n_sample), int(n_shift), int(l_min), int(l_max),
               _ptr(traj), int(seed), int(event), _ptr(n_accepted), _ptr(n_proposed),
               _stream(pos, stream))


class PamdIntegrator:
    """The loop of Fig. 2 over all chains of a problem of harmonic systems."""

    def __init__(self, p: Problem, n_shift: int, n_sample: int, l_min: int, l_max: int,
                 seed: int = 0):
        self.p, self.n_shift, self.n_sample = p, int(n_shift), int(n_sample)
        self.l_min, self.l_max, self.seed = int(l_min), int(l_max), int(seed)
        self.events = 0
        self.n_accepted = None
        self.n_proposed = None

    def run(self, pos: torch.Tensor, n_events: int) -> torch.Tensor:
        """Advance every chain by n_events shifting events.  `pos` (the current
        paths) is updated in place.  Returns the integrated trajectory points,
        shape [n_events * n_shift, flat points of one shift]."""
        p = self.p
        if self.n_accepted is None:
            self.n_accepted = torch.zeros(p.n_chains, dtype=torch.int32, device=pos.device)
            self.n_proposed = torch.zeros(p.n_chains, dtype=torch.int32, device=pos.device)
        per = sum(s.n_chains * self.n_shift * s.d * s.N for s in p.systems)
        out = torch.empty((n_events, per), dtype=p.dtype, device=pos.device)
        a, b = pos, torch.empty_like(pos)
        for ev in range(n_events):
            event(p, a, b, self.n_sample, self.n_shift, self.l_min, self.l_max, out[ev],
                  self.n_accepted, self.n_proposed, seed=self.seed, event=self.events + ev)
            a, b = b, a
        if a is not pos:
            pos.copy_(a)
        self.events += n_events
        return out
