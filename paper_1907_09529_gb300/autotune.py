"""Autotuner for the Lennard-Jones action kernel's launch shape.

For a problem it times ``pamd_action_grad`` (CUDA events, on the current stream)
over a grid of candidate shapes -- steps per tile, threads per particle, list
capacity, Verlet skin (double precision), neighbour-list window (single
precision) -- and keeps the fastest.  Results do not depend on the tile, list
capacity, skin or window (the candidate order inside every sum is fixed); the
threads per particle change how a particle's sums are split, so results differ
by rounding only.  The choice can be cached per problem signature in a small
JSON file.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, Iterable, Optional, Tuple

import torch

from . import Problem, action_grad, tune

Shape = Tuple[int, int, int, float, int]  # tile, threads/particle, max neighbours, skin, window

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuned.json")


def signature(p: Problem) -> str:
    parts = [p.precision, f"{p.D:g},{p.beta:g},{p.dt:g}"]
    for s in p.systems:
        parts.append(f"{s.kind}:{s.N}x{s.T}x{s.n_chains}:{s.box:.6g}:{s.rc:g}")
    return "|".join(parts)


def candidates(tiles=(16, 32, 64), tpps=(0,), skins=(-1.0,), maxnb=(0,),
               windows=(8, 16, 32)) -> Iterable[Shape]:
    for t, q, m, s, w in itertools.product(tiles, tpps, maxnb, skins, windows):
        yield (t, q, m, s, w)


def time_shape(p: Problem, pos: torch.Tensor, shape: Shape, reps: int = 3) -> float:
    tune(*shape)
    S, g = action_grad(p, pos)  # builds the plan for this shape, warms up
    stream = torch.cuda.current_stream(pos.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        action_grad(p, pos, S, g)
    e1.record(stream)
    torch.cuda.synchronize(pos.device)
    return e0.elapsed_time(e1) / reps


def autotune(p: Problem, pos: torch.Tensor, shapes: Optional[Iterable[Shape]] = None,
             reps: int = 3, cache: Optional[str] = DEFAULT_CACHE, verbose: bool = False
             ) -> Tuple[Shape, Dict[str, float]]:
    """Time every candidate shape on (p, pos); leave the fastest one active and
    return it with all timings (ms per action+gradient call)."""
    sig = signature(p)
    if cache and os.path.exists(cache):
        try:
            with open(cache) as fh:
                known = json.load(fh)
            if sig in known:
                best = tuple(known[sig]["shape"])
                tune(*best)
                return best, known[sig]["timings"]
        except (OSError, ValueError, KeyError):
            pass
    timings: Dict[str, float] = {}
    best, best_ms = None, float("inf")
    for shape in (shapes if shapes is not None else candidates()):
        ms = time_shape(p, pos, shape, reps)
        timings[json.dumps(shape)] = ms
        if verbose:
            print(f"  shape tile={shape[0]} tpp={shape[1]} maxnb={shape[2]} skin={shape[3]} "
                  f"window={shape[4]}: {ms:.3f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = shape, ms
    tune(*best)
    if cache:
        try:
            known = {}
            if os.path.exists(cache):
                with open(cache) as fh:
                    known = json.load(fh)
            known[sig] = {"shape": list(best), "timings": timings}
            with open(cache, "w") as fh:
                json.dump(known, fh, indent=1)
        except (OSError, ValueError):
            pass
    return best, timings
