"""Checkpoint and resume of a path-sampling run.

The state of a run is the path, its cached gradient and action, the Philox seed
and the counter of the next update, and the per-chain acceptance counts.  The
random numbers of update u are a pure function of (seed, counter + u), so a run
resumed from a checkpoint draws exactly the numbers an unbroken run would have
drawn and reproduces it bit for bit.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from . import Problem


@dataclasses.dataclass
class RunState:
    pos: torch.Tensor
    grad: torch.Tensor
    S: torch.Tensor
    n_accepted: torch.Tensor
    seed: int
    counter: int


def _signature(p: Problem) -> dict:
    return {"precision": p.precision, "D": p.D, "beta": p.beta, "dt": p.dt,
            "systems": [dataclasses.asdict(s) for s in p.systems], "span": p.span}


def save(path: str, p: Problem, state: RunState) -> None:
    torch.save({"problem": _signature(p), "pos": state.pos.detach().cpu(),
                "grad": state.grad.detach().cpu(), "S": state.S.detach().cpu(),
                "n_accepted": state.n_accepted.detach().cpu(), "seed": int(state.seed),
                "counter": int(state.counter)}, path)


def load(path: str, p: Problem, device="cuda") -> RunState:
    d = torch.load(path, map_location="cpu")
    if d["problem"] != _signature(p):
        raise ValueError("checkpoint was written for a different problem")
    return RunState(pos=d["pos"].to(device), grad=d["grad"].to(device), S=d["S"].to(device),
                    n_accepted=d["n_accepted"].to(device), seed=d["seed"], counter=d["counter"])
