"""GB300-native path action for path-accelerated molecular dynamics (arXiv:1907.09529).

Every step of the path -- forces, Euler-Maruyama residuals (Eq. (3)), the action
S (Eq. (4)), its gradient, the Metropolis-adjusted path update and the
Euler-Maruyama reference (Eq. (2)) -- runs in the CUDA kernels of ``libpamd.so``
behind the C ABI of ``include/pamd.h``.  This module only describes problems,
lays out buffers and marshals PyTorch tensors (device or host memory) to that
ABI.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import torch

from . import _lib
from ._lib import (PAMD_FLAG_HO_EXACT_PROPAGATOR, PAMD_FLAG_ONE_CHAIN_PER_LAUNCH,
                   PAMD_FLAG_REGENERATE_FLAT, PAMD_FP32, PAMD_FP64, PAMD_HARMONIC, PAMD_LJ,
                   PamdError, pamd_action, pamd_action_grad, pamd_device_status, pamd_euler_reference,
                   pamd_event, pamd_fragment_mc, pamd_shift_regenerate,
                   pamd_lj_pair_counts, pamd_normals, pamd_path_update, pamd_philox,
                   pamd_action_grad_hs, pamd_cache_stats, pamd_mala_accept, pamd_mala_commit, pamd_mala_propose,
                   pamd_mala_reverse, pamd_release_cache, pamd_tune, pamd_version)

__all__ = [
    "System", "Problem", "action", "action_grad", "path_update", "euler_reference",
    "lj_pair_counts", "philox", "normals", "PamdAction", "PamdError", "tune", "release_cache",
    "pamd_action", "pamd_action_grad", "pamd_path_update", "pamd_euler_reference",
    "pamd_lj_pair_counts", "pamd_philox", "pamd_normals", "pamd_release_cache", "pamd_tune",
    "pamd_version", "pamd_device_status", "device_status", "pamd_fragment_mc", "fragment_mc",
    "fragment_slots", "pamd_shift_regenerate", "pamd_event", "pamd_cache_stats", "cache_stats",
    "mala_propose", "mala_reverse", "mala_accept", "mala_commit", "pamd_mala_propose",
    "pamd_mala_reverse", "pamd_mala_accept", "pamd_mala_commit", "action_grad_hs",
    "pamd_action_grad_hs",
]

ALIGN = 8  # system offsets are rounded to 8 elements (>= 16 bytes)


@dataclasses.dataclass(frozen=True)
class System:
    """n_chains paths of T steps (T+1 slices) of N particles in d dimensions."""
    kind: str            # "harmonic" or "lj"
    N: int
    d: int
    T: int
    n_chains: int = 1
    k: float = 1.0       # harmonic constant
    box: float = 0.0     # LJ periodic box side
    rc: float = 2.5      # LJ cutoff (must be <= box/2)
    eps: float = 1.0
    sigma: float = 1.0
    # time slab (see timeslab.py): whole-path index of local slice 0 and the halo
    # slices below / above the owned ones; zeros for whole paths
    first_slice: int = 0
    halo_lo: int = 0
    halo_hi: int = 0

    @property
    def chain_len(self) -> int:
        return (self.T + 1) * self.d * self.N


class Problem:
    """A batch of systems sharing D, beta, dt, laid out in one flat buffer."""

    def __init__(self, systems: Sequence[System], D: float, beta: float, dt: float,
                 precision: str = "fp32", one_chain_per_launch: bool = False,
                 ho_exact_propagator: bool = False, regenerate_flat: bool = False):
        """ho_exact_propagator: the sampler and the PAMD loop use the oscillator's
        exact transition density as the path action (the action, gradient and
        update entry points then refuse the problem).  regenerate_flat: the
        shift continues the path past the nose as the line x_T instead of
        free-particle steps."""
        self.systems: List[System] = list(systems)
        self.D, self.beta, self.dt = float(D), float(beta), float(dt)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.offsets = []
        off = 0
        for s in self.systems:
            self.offsets.append(off)
            off += s.n_chains * s.chain_len
            off = (off + ALIGN - 1) // ALIGN * ALIGN
        self.span = off
        self.n_chains = sum(s.n_chains for s in self.systems)
        self.chain0 = []
        c = 0
        for s in self.systems:
            self.chain0.append(c)
            c += s.n_chains
        arr = (_lib.pamd_system * len(self.systems))()
        for q, s in enumerate(self.systems):
            kind = PAMD_HARMONIC if s.kind == "harmonic" else PAMD_LJ
            arr[q] = _lib.pamd_system(s.N, s.T, s.d, s.n_chains, self.offsets[q],
                                      _lib.pamd_potential(kind, s.k, s.eps, s.sigma, s.rc, s.box),
                                      s.first_slice, s.halo_lo, s.halo_hi)
        self._systems_arr = arr
        flags = PAMD_FLAG_ONE_CHAIN_PER_LAUNCH if one_chain_per_launch else 0
        if ho_exact_propagator:
            flags |= PAMD_FLAG_HO_EXACT_PROPAGATOR
        if regenerate_flat:
            flags |= PAMD_FLAG_REGENERATE_FLAT
        self.c = _lib.pamd_problem(self.D, self.beta, self.dt, len(self.systems),
                                   ctypes.cast(arr, ctypes.POINTER(_lib.pamd_system)),
                                   PAMD_FP32 if precision == "fp32" else PAMD_FP64, flags)

    @property
    def ref(self):
        return ctypes.byref(self.c)

    @property
    def units(self) -> int:
        """Particle-timeslices of one action evaluation over all chains."""
        return sum(s.N * s.T * s.n_chains for s in self.systems)

    def empty(self, device="cuda", pin: bool = False) -> torch.Tensor:
        if device == "cpu" or (isinstance(device, torch.device) and device.type == "cpu"):
            return torch.zeros(self.span, dtype=self.dtype, pin_memory=pin)
        return torch.zeros(self.span, dtype=self.dtype, device=device)

    def view(self, buf: torch.Tensor, q: int = 0) -> torch.Tensor:
        """[n_chains][T+1][d][N] view of system q inside a flat buffer."""
        s = self.systems[q]
        o = self.offsets[q]
        return buf[o:o + s.n_chains * s.chain_len].view(s.n_chains, s.T + 1, s.d, s.N)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(t: Optional[torch.Tensor], stream=None):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    if t is not None and t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def _check_buf(p: Problem, t: torch.Tensor, name: str):
    if t.dtype != p.dtype or not t.is_contiguous() or t.numel() < p.span:
        raise ValueError(f"{name}: need a contiguous {p.dtype} buffer of >= {p.span} elements")


def action(p: Problem, pos: torch.Tensor, S: Optional[torch.Tensor] = None, stream=None):
    _check_buf(p, pos, "pos")
    if S is None:
        S = torch.empty(p.n_chains, dtype=torch.float64, device=pos.device)
    pamd_action(p.ref, _ptr(pos), _ptr(S), _stream(pos, stream))
    return S


def action_grad(p: Problem, pos: torch.Tensor, S: Optional[torch.Tensor] = None,
                grad: Optional[torch.Tensor] = None, stream=None):
    _check_buf(p, pos, "pos")
    if S is None:
        S = torch.empty(p.n_chains, dtype=torch.float64, device=pos.device)
    if grad is None:
        grad = torch.zeros_like(pos)  # padding between systems stays defined
    pamd_action_grad(p.ref, _ptr(pos), _ptr(S), _ptr(grad), _stream(pos, stream))
    return S, grad


def action_grad_hs(p: Problem, pos: torch.Tensor, sigma_hs: torch.Tensor,
                   S: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None,
                   with_grad: bool = True, stream=None):
    """Action (+inf where a pair lies within its slice's hard-sphere radius) and
    gradient with the hard-sphere path bias of the paper's LJ runs;
    sigma_hs: float64 device tensor, T+1 radii per LJ system in order."""
    _check_buf(p, pos, "pos")
    if S is None:
        S = torch.empty(p.n_chains, dtype=torch.float64, device=pos.device)
    if grad is None and with_grad:
        grad = torch.zeros_like(pos)
    pamd_action_grad_hs(p.ref, _ptr(pos), _ptr(sigma_hs.contiguous()), _ptr(S), _ptr(grad),
                        _stream(pos, stream))
    return S, grad


def path_update(p: Problem, pos: torch.Tensor, grad: torch.Tensor, S: torch.Tensor, h: float,
                n_updates: int = 1, seed: int = 0, counter: int = 0,
                noise: Optional[torch.Tensor] = None, log_u: Optional[torch.Tensor] = None,
                n_accepted: Optional[torch.Tensor] = None,
                log_alpha: Optional[torch.Tensor] = None, stream=None):
    _check_buf(p, pos, "pos")
    _check_buf(p, grad, "grad")
    pamd_path_update(p.ref, _ptr(pos), _ptr(grad), _ptr(S), float(h), int(n_updates),
                     int(seed), int(counter), _ptr(noise), _ptr(log_u), _ptr(n_accepted),
                     _ptr(log_alpha), _stream(pos, stream))


def mala_propose(p: Problem, pos: torch.Tensor, grad: torch.Tensor, h: float, seed: int = 0,
                 counter: int = 0, noise: Optional[torch.Tensor] = None,
                 prop: Optional[torch.Tensor] = None, q_fwd: Optional[torch.Tensor] = None,
                 stream=None):
    """First piece of a path update (pamd_mala_propose): the proposal and this
    slab's part of the forward proposal term, per chain."""
    _check_buf(p, pos, "pos")
    if prop is None:
        prop = torch.empty_like(pos)
    if q_fwd is None:
        q_fwd = torch.empty(p.n_chains, dtype=torch.float64, device=pos.device)
    pamd_mala_propose(p.ref, _ptr(pos), _ptr(grad), _ptr(prop), float(h), int(seed), int(counter),
                      _ptr(noise), _ptr(q_fwd), _stream(pos, stream))
    return prop, q_fwd


def mala_reverse(p: Problem, pos: torch.Tensor, prop: torch.Tensor, grad_prop: torch.Tensor,
                 h: float, q_rev: Optional[torch.Tensor] = None, stream=None):
    """This slab's part of the reverse proposal term, per chain (pamd_mala_reverse)."""
    if q_rev is None:
        q_rev = torch.empty(p.n_chains, dtype=torch.float64, device=pos.device)
    pamd_mala_reverse(p.ref, _ptr(pos), _ptr(prop), _ptr(grad_prop), float(h), _ptr(q_rev),
                      _stream(pos, stream))
    return q_rev


def mala_accept(p: Problem, S: torch.Tensor, S_prop: torch.Tensor, q_fwd: torch.Tensor,
                q_rev: torch.Tensor, h: float, seed: int = 0, counter: int = 0,
                log_u: Optional[torch.Tensor] = None, n_accepted: Optional[torch.Tensor] = None,
                log_alpha: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Metropolis-Hastings decisions from whole-path sums (pamd_mala_accept)."""
    accept = torch.empty(p.n_chains, dtype=torch.int32, device=S.device)
    pamd_mala_accept(p.ref, _ptr(S), _ptr(S_prop), _ptr(q_fwd), _ptr(q_rev), float(h), int(seed),
                     int(counter), _ptr(log_u), _ptr(accept), _ptr(n_accepted), _ptr(log_alpha),
                     _stream(S, stream))
    return accept


def mala_commit(p: Problem, pos: torch.Tensor, grad: torch.Tensor, S: torch.Tensor,
                prop: torch.Tensor, grad_prop: torch.Tensor, S_prop: torch.Tensor,
                accept: torch.Tensor, stream=None):
    """Accepted chains take the proposal, its gradient and action (pamd_mala_commit)."""
    pamd_mala_commit(p.ref, _ptr(pos), _ptr(grad), _ptr(S), _ptr(prop), _ptr(grad_prop),
                     _ptr(S_prop), _ptr(accept), _stream(pos, stream))


def euler_reference(p: Problem, pos: torch.Tensor, seed: int = 0, counter: int = 0,
                    noise: Optional[torch.Tensor] = None, stream=None):
    _check_buf(p, pos, "pos")
    pamd_euler_reference(p.ref, _ptr(pos), int(seed), int(counter), _ptr(noise),
                         _stream(pos, stream))
    return pos


def fragment_slots(p: Problem, l_min: int) -> int:
    """Per-chain stride of the log_u array of fragment_mc."""
    return max(s.T for s in p.systems) // (1 << l_min) + 2


def fragment_mc(p: Problem, pos: torch.Tensor, l_min: int, l_max: int, n_steps: int = 1,
                seed: int = 0, counter: int = 0, levels: Optional[torch.Tensor] = None,
                offsets: Optional[torch.Tensor] = None, noise: Optional[torch.Tensor] = None,
                log_u: Optional[torch.Tensor] = None, n_accepted: Optional[torch.Tensor] = None,
                n_proposed: Optional[torch.Tensor] = None, stream=None):
    """Multilevel sliding-and-sampling MC steps (Sec. III) of harmonic paths."""
    _check_buf(p, pos, "pos")
    if n_accepted is None:
        n_accepted = torch.zeros(p.n_chains, dtype=torch.int32, device=pos.device)
    if n_proposed is None:
        n_proposed = torch.zeros(p.n_chains, dtype=torch.int32, device=pos.device)
    pamd_fragment_mc(p.ref, _ptr(pos), int(l_min), int(l_max), int(n_steps), int(seed),
                     int(counter), _ptr(levels), _ptr(offsets), _ptr(noise), _ptr(log_u),
                     _ptr(n_accepted), _ptr(n_proposed), _stream(pos, stream))
    return n_accepted, n_proposed


def lj_pair_counts(p: Problem, pos: torch.Tensor, stream=None) -> torch.Tensor:
    n = sum(s.n_chains * (s.T + 1) for s in p.systems if s.kind == "lj")
    counts = torch.zeros(n, dtype=torch.int64, device=pos.device)
    pamd_lj_pair_counts(p.ref, _ptr(pos), _ptr(counts), _stream(pos, stream))
    return counts


def philox(ctr, key, n: int, device="cuda") -> torch.Tensor:
    out = torch.empty(4 * n, dtype=torch.int32, device=device)
    pamd_philox(*[int(c) for c in ctr], *[int(k) for k in key], int(n), _ptr(out), _stream(out))
    return out


def normals(seed: int, counter: int, stream_id: int, chain: int, n: int, e0: int = 0,
            device="cuda") -> torch.Tensor:
    out = torch.empty(n, dtype=torch.float32, device=device)
    pamd_normals(int(seed), int(counter), int(stream_id), int(chain), int(e0), int(n), _ptr(out),
                 _stream(out))
    return out


def tune(tile_steps: int = 0, threads_per_particle: int = 0, max_neighbours: int = 0,
         skin: float = -1.0, window_steps: int = 0):
    """Launch-shape override for the LJ kernels (zeros: automatic); see pamd_tune."""
    pamd_tune(tile_steps, threads_per_particle, max_neighbours, skin, window_steps)


def release_cache():
    pamd_release_cache()


def cache_stats():
    """(cached plans, captured update graphs) held by the library."""
    return pamd_cache_stats()


def device_status(stream=None):
    """Raise PamdError if an action computed since the last check was not finite."""
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    pamd_device_status(s)


class PamdAction(torch.autograd.Function):
    """S = PamdAction.apply(pos, problem): per-chain action with the hand-written
    adjoint (the kernel's path gradient) as backward."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, p: Problem):
        S, grad = action_grad(p, pos.detach().contiguous())
        ctx.save_for_backward(grad)
        ctx.problem = p
        return S

    @staticmethod
    def backward(ctx, gS: torch.Tensor):
        (grad,) = ctx.saved_tensors
        p = ctx.problem
        out = torch.zeros_like(grad)
        for q, s in enumerate(p.systems):
            c0 = p.chain0[q]
            w = gS[c0:c0 + s.n_chains].to(grad.dtype).view(-1, 1, 1, 1)
            p.view(out, q).copy_(p.view(grad, q) * w)
        return out, None
