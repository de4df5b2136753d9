"""The hard-sphere path bias of the paper's Lennard-Jones runs (Sec. IV.B) through
pamd_action_grad_hs, against the oracle.

The overlap decision is an integer outcome decided in floating point: it is
compared with the oracle's mirror of the kernels' single-precision rule
(oracle.hs_overlap_f32, slice by slice) for single-precision paths, and with the
oracle's double-precision test for double-precision paths.  A finite action is
the plain LJ action (checked against the oracle and, bit for bit, against
pamd_action_grad), and the gradient is the LJ gradient in every case.
"""
import math

import numpy as np
import pytest

import oracle
import pamd_inputs as inputs
from _common import gpu_system, oracle_potential, rel, start_paths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pamd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    pamd.tune()
    return pamd


def _setup(pamd, name, precision):
    if name == "mixed":  # LJ systems on both sides of N = 512: two block-size classes
        import dataclasses
        w = dataclasses.replace(
            inputs.workload("ragged", "small"), name="mixed",
            systems=[inputs.SystemSpec("lj", 96, 3, 30, 2), inputs.SystemSpec("lj", 600, 3, 20, 2)])
    else:
        w = inputs.workload(name, "small")
    prob = pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt,
                        precision=precision)
    paths = start_paths(w, precision)
    buf = prob.empty("cuda")
    for q, p in enumerate(paths):
        prob.view(buf, q).copy_(torch.from_numpy(p).to(prob.dtype))
    return w, prob, paths, buf


def _schedules(w, kind, top):
    """Per LJ system: T+1 radii.  ramp: 0 at the tail rising to `top` at the nose
    (the shape of the paper's schedule); nose: `top` at the last slice only;
    mid: `top` at the middle slice only."""
    out = []
    for s in w.systems:
        if s.kind != "lj":
            continue
        sig = np.zeros(s.T + 1)
        if kind == "ramp":
            sig = top * np.linspace(0.0, 1.0, s.T + 1)
        elif kind == "nose":
            sig[s.T] = top
        elif kind == "mid":
            sig[s.T // 2] = top
        out.append(sig)
    return out


@pytest.mark.parametrize("name,precision", [("lj500", "fp32"), ("ragged", "fp32"),
                                            ("lj108", "fp64")])
def test_zero_radius_is_the_plain_action(pamd, name, precision):
    w, prob, paths, buf = _setup(pamd, name, precision)
    sig = torch.from_numpy(np.concatenate(_schedules(w, "zero", 0.0))).cuda()
    S0, g0 = pamd.action_grad(prob, buf)
    S, g = pamd.action_grad_hs(prob, buf, sig)
    torch.cuda.synchronize()
    assert torch.equal(S, S0) and torch.equal(g, g0)


@pytest.mark.parametrize("name,precision", [("lj108", "fp32"), ("ragged", "fp32"),
                                            ("lj108", "fp64"), ("mixed", "fp32")])
def test_overlaps_match_the_oracle(pamd, parity_report, name, precision):
    w, prob, paths, buf = _setup(pamd, name, precision)
    S0, g0 = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    n_inf = n_fin = 0
    for kind, top in [("ramp", 0.85), ("ramp", 1.0), ("ramp", 1.15), ("nose", 1.1),
                      ("mid", 1.05), ("ramp", 3.0)]:
        sched = _schedules(w, kind, top)
        sig = torch.from_numpy(np.concatenate(sched)).cuda()
        S, g = pamd.action_grad_hs(prob, buf, sig)
        S_only, _ = pamd.action_grad_hs(prob, buf, sig, with_grad=False)
        torch.cuda.synchronize()
        assert torch.equal(g, g0)  # the bias adds nothing to the gradient
        assert torch.equal(S_only, S)
        S = S.cpu().numpy()
        lj = 0
        for q, spec in enumerate(w.systems):
            if spec.kind != "lj":
                continue
            sg = sched[lj]
            lj += 1
            pot = oracle_potential(spec)
            for b in range(spec.n_chains):
                x = paths[q][b]
                if precision == "fp32":
                    x32 = x.astype(np.float32)
                    want = any(oracle.hs_overlap_f32(spec.box, spec.rc_eff, sg[t], x32[t])
                               for t in range(spec.T + 1) if sg[t] > 0)
                else:
                    want = oracle.hs_first_overlap(pot, x, sg) >= 0
                c = prob.chain0[q] + b
                if want:
                    assert S[c] == math.inf, (kind, top, q, b)
                    n_inf += 1
                else:
                    assert S[c] == float(S0[c].item())
                    So = oracle.action_grad(pot, x, w.D, w.beta, w.dt, grad=False, nthreads=8)
                    assert abs(S[c] - So) <= (1e-5 if precision == "fp32" else 1e-12) * So
                    n_fin += 1
    assert n_inf > 0 and n_fin > 0  # both outcomes occur
    parity_report.record(f"{name}_hardsphere_{precision}",
                         "test_overlaps_match_the_oracle (overlap decisions equal)",
                         chains_infinite=n_inf, chains_finite=n_fin)


def test_biased_proposal_with_an_overlap_is_rejected(pamd):
    """Pieces of the path update with the biased action: a proposal whose path has
    an overlapping pair (S' = +inf) is never accepted."""
    w, prob, paths, buf = _setup(pamd, "lj108", "fp32")
    sig = torch.from_numpy(np.concatenate(_schedules(w, "zero", 0.0))).cuda()
    S, g = pamd.action_grad_hs(prob, buf, sig)
    prop, qf = pamd.mala_propose(prob, buf, g, 2e-7, seed=3, counter=1)
    big = torch.from_numpy(np.concatenate(_schedules(w, "ramp", 3.0))).cuda()
    Sp, gp = pamd.action_grad_hs(prob, prop, big)
    qr = pamd.mala_reverse(prob, buf, prop, gp, 2e-7)
    acc = pamd.mala_accept(prob, S, Sp, qf, qr, 2e-7, seed=3, counter=1)
    torch.cuda.synchronize()
    assert bool(torch.isinf(Sp).all()) and int(acc.sum()) == 0
