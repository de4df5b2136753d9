"""Time slabs on the GPU: one path split in time over three slabs held by this
process (timeslab.LocalComm), each evaluated by the library's slab entry points.

Against the whole-path library calls on the same inputs (themselves checked
against the oracle by the parity tests): the gradient at every owned slice and
the positions after each update are bitwise equal, accept decisions and counts
are equal, and S agrees to 1e-12 where every per-thread sum is double (the LJ
kernels, FP64 data: only the order of the double-precision parts differs) and
to 1e-7 for the single-precision oscillator kernel, whose per-thread partials
over a few elements are single precision before the double-precision sum (a
slab groups the elements differently).  The update pieces on whole paths equal
pamd_path_update bit for bit.
"""
import numpy as np
import pytest

import pamd_inputs as inputs
from _common import gpu_system, start_paths

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
    w = inputs.workload(name, "small")
    prob = pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt,
                        precision=precision)
    buf = prob.empty("cuda")
    for q, p in enumerate(start_paths(w, precision)):
        prob.view(buf, q).copy_(torch.from_numpy(p).to(prob.dtype))
    return w, prob, buf


CASES = [("lj500", "fp32"), ("ragged", "fp32"), ("ho3d", "fp32"), ("lj108", "fp64")]


@pytest.mark.parametrize("name,precision", CASES)
def test_update_pieces_equal_path_update(pamd, name, precision):
    w, prob, buf = _setup(pamd, name, precision)
    h = 1e-5 if name == "ho3d" else 2e-6  # large enough that some proposals are rejected
    S0, g0 = pamd.action_grad(prob, buf)
    ref_pos, ref_g, ref_S = buf.clone(), g0.clone(), S0.clone()
    ref_acc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    ref_la = torch.zeros(prob.n_chains, dtype=torch.float64, device="cuda")
    pos, g, S = buf.clone(), g0.clone(), S0.clone()
    acc = torch.zeros_like(ref_acc)
    la = torch.zeros_like(ref_la)
    for k in range(3):
        pamd.path_update(prob, ref_pos, ref_g, ref_S, h, 1, seed=5, counter=40 + k,
                         n_accepted=ref_acc, log_alpha=ref_la)
        prop, qf = pamd.mala_propose(prob, pos, g, h, seed=5, counter=40 + k)
        Sp, gp = pamd.action_grad(prob, prop)
        qr = pamd.mala_reverse(prob, pos, prop, gp, h)
        flags = pamd.mala_accept(prob, S, Sp, qf, qr, h, seed=5, counter=40 + k, n_accepted=acc,
                                 log_alpha=la)
        pamd.mala_commit(prob, pos, g, S, prop, gp, Sp, flags)
    torch.cuda.synchronize()
    assert int(ref_acc.sum()) > 0
    assert torch.equal(pos, ref_pos) and torch.equal(g, ref_g) and torch.equal(S, ref_S)
    assert torch.equal(acc, ref_acc) and torch.equal(la, ref_la)


@pytest.mark.parametrize("name,precision", CASES)
def test_three_slabs_match_the_whole_path(pamd, parity_report, name, precision):
    from paper_1907_09529_gb300 import timeslab
    w, prob, buf = _setup(pamd, name, precision)
    h = 1e-5 if name == "ho3d" else 2e-6
    S_ref, g_ref = pamd.action_grad(prob, buf)
    tol = 1e-7 if precision == "fp32" and any(s.kind == "harmonic" for s in prob.systems) else 1e-12
    run = timeslab.SlabRun(prob, timeslab.LocalComm(3))
    bufs = [timeslab.scatter(prob, buf, lp) for lp in run.probs]
    S, G = run.action_grad(bufs)
    torch.cuda.synchronize()

    def check(S_ref, g_ref, pos_ref=None):
        worst = 0.0
        for k, lp in enumerate(run.probs):
            worst = max(worst, float(((S[k] - S_ref).abs() / S_ref.abs()).max()))
            assert torch.allclose(S[k], S_ref, rtol=tol, atol=0)
            for q, s in enumerate(lp.systems):
                o = timeslab.owned_slices(s)
                lo, hi = s.first_slice + o.start, s.first_slice + o.stop
                assert torch.equal(lp.view(G[k], q)[:, o], prob.view(g_ref, q)[:, lo:hi])
                if pos_ref is not None:
                    assert torch.equal(lp.view(bufs[k], q)[:, o], prob.view(pos_ref, q)[:, lo:hi])
        return worst

    worst = check(S_ref, g_ref)
    # three sharded updates (Philox noise over the whole path) against the whole-path update
    acc_ref = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    accs = [torch.zeros_like(acc_ref) for _ in run.probs]
    pos_ref, gr, Sr = buf.clone(), g_ref.clone(), S_ref.clone()
    for k in range(3):
        pamd.path_update(prob, pos_ref, gr, Sr, h, 1, seed=9, counter=70 + k, n_accepted=acc_ref)
        run.update(bufs, G, S, h, seed=9, counter=70 + k, n_accepted=accs)
        torch.cuda.synchronize()
        worst = max(worst, check(Sr, gr, pos_ref))
        for a in accs:
            assert torch.equal(a, acc_ref)
    assert int(acc_ref.sum()) > 0
    parity_report.record(f"{name}_timeslab3_{precision}",
                         "test_three_slabs_match_the_whole_path (S vs the whole-path call; "
                         "gradients and paths bitwise)", S_rel=worst)


def test_slab_problems_are_refused_where_whole_paths_are_needed(pamd):
    from paper_1907_09529_gb300 import timeslab
    w, prob, buf = _setup(pamd, "lj500", "fp32")
    lp = timeslab.slab_problem(prob, 1, 3)
    b = timeslab.scatter(prob, buf, lp)
    S, g = pamd.action_grad(lp, b)
    with pytest.raises(pamd.PamdError) as ei:
        pamd.path_update(lp, b, g, S, 1e-7)
    assert ei.value.status == -2
    with pytest.raises(pamd.PamdError):
        pamd.euler_reference(lp, b)
    sig = torch.zeros(sum(s.T + 1 for s in lp.systems if s.kind == "lj"), dtype=torch.float64,
                      device="cuda")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.action_grad_hs(lp, b, sig)
    assert ei.value.status == -2
