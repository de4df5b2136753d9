"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP32 data with FP64 accumulation, 1e-5 relative on S and on the
gradient (per chain, 2-norm) plus a max-abs bound of 1e-5 * max|g|; plain FP64,
1e-12 relative.  Index work (pair counts, Philox words) is compared bit for bit.
"""
import dataclasses
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
    pamd.tune()  # automatic launch shapes
    return pamd


def _problem(pamd, w, precision, one=False):
    return pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt,
                        precision=precision, one_chain_per_launch=one)


def _upload(pamd, prob, paths, device="cuda"):
    buf = prob.empty(device)
    for q, p in enumerate(paths):
        prob.view(buf, q).copy_(torch.from_numpy(p).to(prob.dtype))
    return buf


def _workload(name):
    """The small workloads, plus "mixed": LJ systems on both sides of N = 512, which
    a single-precision plan launches in two block-size classes."""
    if name == "mixed":
        base = inputs.workload("ragged", "small")
        systems = [inputs.SystemSpec("lj", 96, 3, 40, 2), inputs.SystemSpec("lj", 530, 3, 33, 1),
                   inputs.SystemSpec("lj", 700, 3, 25, 2)]
        return dataclasses.replace(base, name="mixed", systems=systems)
    return inputs.workload(name, "small")


def _check_against_oracle(w, prob, paths, S, g, tol_rel, nthreads=8):
    S = S.cpu().numpy()
    g = g.cpu()
    worst = (0.0, 0.0, 0.0)
    for q, spec in enumerate(w.systems):
        pot = oracle_potential(spec)
        gq = prob.view(g, q).double().numpy()
        for b in range(spec.n_chains):
            So, go = oracle.action_grad(pot, paths[q][b], w.D, w.beta, w.dt, nthreads=nthreads)
            c = prob.chain0[q] + b
            es = abs(S[c] - So) / abs(So)
            eg = rel(gq[b], go)
            emax = np.abs(gq[b] - go).max() / np.abs(go).max()
            assert es <= tol_rel, (q, b, es)
            assert eg <= tol_rel, (q, b, eg)
            assert emax <= tol_rel, (q, b, emax)
            worst = (max(worst[0], es), max(worst[1], eg), max(worst[2], emax))
    return worst


@pytest.mark.parametrize("name", ["ho3d", "lj108", "lj500", "ragged"])
def test_fp32_action_grad_matches_oracle(pamd, parity_report, name):
    w = inputs.workload(name, "small")
    paths = start_paths(w, "fp32")
    prob = _problem(pamd, w, "fp32")
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    es, eg, em = _check_against_oracle(w, prob, paths, S, g, 1e-5)
    parity_report.record(f"{name}_small", "test_fp32_action_grad_matches_oracle", S_rel=es,
                         grad_rel_2norm=eg, grad_rel_maxabs=em)
    # action-only entry point gives the same S
    S2 = pamd.action(prob, buf)
    torch.cuda.synchronize()
    assert torch.allclose(S2, S, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name,one", [("ho1d", True), ("ho1d", False), ("lj108", True),
                                      ("ragged", False)])
def test_fp64_plain_matches_oracle(pamd, parity_report, name, one):
    w = inputs.workload(name, "small")
    paths = start_paths(w, "fp64")
    prob = _problem(pamd, w, "fp64", one=one)
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    es, eg, em = _check_against_oracle(w, prob, paths, S, g, 1e-12)
    parity_report.record(f"{name}_small_fp64", "test_fp64_plain_matches_oracle", S_rel=es,
                         grad_rel_2norm=eg, grad_rel_maxabs=em)


def test_edge_cases_tiny_paths(pamd):
    """T = 1 (two slices), N = 2 LJ particles, odd sizes and ragged tails."""
    L = 6.0
    systems = [pamd.System("lj", 2, 3, 1, 1, box=L, rc=2.5),
               pamd.System("lj", 3, 3, 5, 2, box=L, rc=3.0),
               pamd.System("harmonic", 1, 1, 1, 1, k=2.0),
               pamd.System("harmonic", 5, 2, 4097, 2, k=0.5)]
    prob = pamd.Problem(systems, 0.9, 1.1, 1e-3)
    rng = inputs.rng(5)
    paths = []
    for s in systems:
        base = rng.uniform(0, L, size=(s.n_chains, 1, s.d, s.N)) if s.kind == "lj" else 0
        p = base + 0.05 * rng.standard_normal((s.n_chains, s.T + 1, s.d, s.N))
        if s.kind == "lj":  # keep pairs apart
            p[:, :, :, :] += np.arange(s.N)[None, None, None, :] * 1.3
        paths.append(p.astype(np.float32).astype(np.float64))
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S, g = S.cpu().numpy(), g.cpu()
    for q, s in enumerate(systems):
        pot = (oracle.lennard_jones(s.box, s.rc) if s.kind == "lj" else oracle.harmonic(s.k))
        for b in range(s.n_chains):
            So, go = oracle.action_grad(pot, paths[q][b], 0.9, 1.1, 1e-3)
            c = prob.chain0[q] + b
            assert abs(S[c] - So) <= 1e-5 * abs(So)
            assert rel(prob.view(g, q)[b].double().numpy(), go) <= 1e-5


@pytest.mark.parametrize("name", ["lj108", "lj500"])
def test_results_independent_of_tiling(pamd, name):
    """Candidate order is fixed, so S and the gradient are bitwise the same for any
    tile, neighbour-list window (down to one list per step pair) and list
    capacity (including the overflow path, where a particle scans every
    candidate).  In lj108's box the lists reach past L/2; in lj500's they do not."""
    w = inputs.workload(name, "small")
    paths = start_paths(w, "fp32")
    outs = []
    try:
        for tile, tpp, maxnb, window in [(32, 0, 0, 0), (1, 0, 0, 0), (7, 0, 0, 2),
                                         (64, 0, 0, 40), (16, 0, 8, 0), (33, 0, 0, 5)]:
            pamd.tune(tile, tpp, maxnb, -1.0, window)
            prob = _problem(pamd, w, "fp32")
            buf = _upload(pamd, prob, paths)
            S, g = pamd.action_grad(prob, buf)
            torch.cuda.synchronize()
            outs.append((S.cpu(), prob.view(g, 0).cpu()))
    finally:
        pamd.tune()
    for S, g in outs[1:]:
        assert torch.equal(S, outs[0][0])
        assert torch.equal(g, outs[0][1])


@pytest.mark.parametrize("tpp", [0, 1, 2, 4])
def test_threads_per_particle_match_the_oracle(pamd, tpp):
    """Every width of the per-particle thread group against the oracle: forced
    widths 1, 2 and 4, and the automatic choice (0), which gives the two tiny
    systems added to the small ragged batch (N = 16, 20) groups of 8 threads.
    Candidate classes are split over the group below 8 threads and lie in one
    class per thread at 8.  A list capacity of 24 sends most particles down the
    overflow paths."""
    base = inputs.workload("ragged", "small")
    tiny = [inputs.SystemSpec("lj", n, 3, 40, 1) for n in (16, 20)]
    w = dataclasses.replace(base, systems=list(base.systems) + tiny)
    paths = start_paths(w, "fp32")
    try:
        for maxnb in (0, 24):
            pamd.tune(0, tpp, maxnb, -1.0, 0)
            prob = _problem(pamd, w, "fp32")
            buf = _upload(pamd, prob, paths)
            S, g = pamd.action_grad(prob, buf)
            torch.cuda.synchronize()
            _check_against_oracle(w, prob, paths, S, g, 1e-5)
    finally:
        pamd.tune()


@pytest.mark.parametrize("one_class", [False, True])
def test_block_size_classes_match_the_oracle(pamd, parity_report, one_class):
    """A single-precision batch of LJ systems with N on both sides of 512 runs in two
    persistent launches (the N <= 512 system in 384-thread blocks, four threads per
    particle, with the pipelined gradient pass; the others in 704-thread blocks);
    PAMD_LJ_ONE_CLASS keeps one launch of 704-thread blocks.  Both against the
    oracle, and in one chain per launch."""
    import os
    w = _workload("mixed")
    paths = start_paths(w, "fp32")
    try:
        if one_class:
            os.environ["PAMD_LJ_ONE_CLASS"] = "1"
        for one in (False, True):
            pamd.release_cache()
            prob = _problem(pamd, w, "fp32", one=one)
            buf = _upload(pamd, prob, paths)
            S, g = pamd.action_grad(prob, buf)
            torch.cuda.synchronize()
            es, eg, em = _check_against_oracle(w, prob, paths, S, g, 1e-5)
            if not one and not one_class:
                parity_report.record("mixed_classes", "test_block_size_classes_match_the_oracle",
                                     S_rel=es, grad_rel_2norm=eg, grad_rel_maxabs=em)
    finally:
        os.environ.pop("PAMD_LJ_ONE_CLASS", None)
        pamd.release_cache()


def test_lj_far_from_brownian_paths_use_the_fallbacks(pamd):
    """Slices that jump by ~0.3 sigma (a jittered FCC lattice at every step) make
    the item-wide outer lists and the window lists overflow the capacities the
    plan sizes for Brownian steps: particles then build their window lists from
    every candidate and evaluate every candidate.  S and the gradient must still
    match the oracle, and be bitwise independent of tile and window."""
    N, T, B, rho = 256, 40, 2, 0.5
    L = (N / rho) ** (1.0 / 3.0)
    x0 = inputs.fcc_lattice(N, L)
    rng = inputs.rng(77)
    paths = (x0[None, None] + 0.12 * rng.standard_normal((B, T + 1, 3, N)))
    paths = paths.astype(np.float32).astype(np.float64)
    D, beta, dt = 1.0, 1.0, 1e-4
    system = pamd.System("lj", N, 3, T, B, box=L, rc=2.5)
    prob = pamd.Problem([system], D, beta, dt)
    pot = oracle.lennard_jones(L, 2.5)
    outs = []
    try:
        for tile, window in [(16, 0), (40, 2), (7, 24)]:
            pamd.tune(tile, 0, 0, -1.0, window)
            buf = _upload(pamd, prob, [paths])
            S, g = pamd.action_grad(prob, buf)
            torch.cuda.synchronize()
            outs.append((S.cpu(), g.cpu()))
    finally:
        pamd.tune()
    for S, g in outs[1:]:
        assert torch.equal(S, outs[0][0]) and torch.equal(g, outs[0][1])
    S, g = outs[0]
    for b in range(B):
        So, go = oracle.action_grad(pot, paths[b], D, beta, dt)
        gb = prob.view(g, 0)[b].double().numpy()
        assert abs(S[b].item() - So) <= 1e-5 * abs(So)
        assert rel(gb, go) <= 1e-5
        assert np.abs(gb - go).max() <= 1e-5 * np.abs(go).max()


def test_pair_counts_bit_exact(pamd):
    w = inputs.workload("lj500", "small")
    paths = start_paths(w, "fp32")
    spec = w.systems[0]
    prob = _problem(pamd, w, "fp32")
    buf = _upload(pamd, prob, paths)
    counts = pamd.lj_pair_counts(prob, buf).cpu().numpy()
    T = spec.T
    for b in range(spec.n_chains):
        for t in range(0, T + 1, 7):
            ref = oracle.pair_count_f32(spec.box, spec.rc_eff, paths[0][b, t].astype(np.float32))
            assert counts[b * (T + 1) + t] == ref


def test_philox_and_normals_match_oracle(pamd):
    ctr, key = (0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)
    n = 1000
    words = pamd.philox(ctr, key, n).cpu().numpy().view(np.uint32).reshape(n, 4)
    for q in (0, 1, 517, n - 1):
        c = list(ctr)
        c[0] = (c[0] + q) & 0xFFFFFFFF
        assert np.array_equal(words[q], oracle.philox(c, key))
    z = pamd.normals(seed=1234567, counter=3, stream_id=1, chain=5, n=4099, e0=13).cpu().numpy()
    zo = oracle.normals(1234567, 3, 1, 5, 4099, e0=13)
    assert np.all(np.abs(z - zo) <= 2e-6 * (1 + np.abs(zo)))


def test_euler_reference_matches_oracle(pamd):
    # plain FP64 oscillator: exact recursion
    w = inputs.workload("ho1d")
    spec = w.systems[0]
    prob = _problem(pamd, w, "fp64")
    xi = inputs.euler_noise(spec, 77)
    noise = np.zeros((1, spec.T + 1, 1, 1))
    noise[:, 1:] = xi
    buf = prob.empty("cuda")
    nbuf = prob.empty("cuda")
    prob.view(nbuf, 0).copy_(torch.from_numpy(noise))
    pamd.euler_reference(prob, buf, noise=nbuf)
    torch.cuda.synchronize()
    ref = oracle.euler(oracle_potential(spec), np.zeros((1, 1)), xi[0], w.D, w.beta, w.dt)
    got = prob.view(buf, 0)[0].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1, np.abs(ref).max())
    # FP32 LJ, short path (chaos has no time to amplify roundoff)
    w = inputs.workload("lj108", "small")
    spec = w.systems[0]
    T = 30
    spec = inputs.SystemSpec("lj", spec.N, 3, T, 2)
    prob = pamd.Problem([gpu_system(spec, pamd)], w.D, w.beta, w.dt)
    x0 = inputs.initial_positions(spec, 1)
    xi = inputs.euler_noise(spec, 78)
    noise = np.zeros((2, T + 1, 3, spec.N))
    noise[:, 1:] = xi
    buf = prob.empty("cuda")
    prob.view(buf, 0)[:, 0].copy_(torch.from_numpy(x0).float())
    nbuf = prob.empty("cuda")
    prob.view(nbuf, 0).copy_(torch.from_numpy(noise).float())
    pamd.euler_reference(prob, buf, noise=nbuf)
    torch.cuda.synchronize()
    ref = oracle.euler_batch(oracle_potential(spec), x0, noise[:, 1:].astype(np.float32), w.D,
                             w.beta, w.dt, store_f32=True)
    got = prob.view(buf, 0).cpu().double().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-5
    # Philox noise stream: the invariant S = sum xi^2 / 2 holds up to FP32 rounding
    buf2 = prob.empty("cuda")
    prob.view(buf2, 0)[:, 0].copy_(torch.from_numpy(x0).float())
    pamd.euler_reference(prob, buf2, seed=99, counter=5)
    S, _ = pamd.action_grad(prob, buf2)
    zs = [pamd.normals(99, 5, 0, c, T * 3 * spec.N, e0=3 * spec.N).double().cpu()
          for c in range(2)]
    for c in range(2):
        assert abs(S[c].item() - 0.5 * float((zs[c] ** 2).sum())) <= 1e-3 * S[c].item()


def _mala_case(pamd, w, precision, h, seed):
    paths = start_paths(w, precision)
    prob = _problem(pamd, w, precision)
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    rng = inputs.rng(seed)
    eta = [rng.standard_normal(p.shape) for p in paths]
    if precision == "fp32":
        eta = [e.astype(np.float32).astype(np.float64) for e in eta]
    logu = np.log(rng.random(prob.n_chains))
    nbuf = _upload(pamd, prob, eta)
    lu = torch.from_numpy(logu).cuda()
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    la = torch.zeros(prob.n_chains, dtype=torch.float64, device="cuda")
    S0, g0 = S.clone(), g.clone()
    pamd.path_update(prob, buf, g, S, h, 1, noise=nbuf, log_u=lu, n_accepted=nacc, log_alpha=la)
    torch.cuda.synchronize()
    return prob, paths, eta, logu, S0.cpu().numpy(), g0.cpu(), buf.cpu(), g.cpu(), S.cpu().numpy(), \
        nacc.cpu().numpy(), la.cpu().numpy()


def test_mala_update_fp64_matches_oracle(pamd):
    w = inputs.workload("ho1d")
    prob, paths, eta, logu, S0, g0, pos1, g1, S1, nacc, la = _mala_case(pamd, w, "fp64", 2e-4, 3)
    spec = w.systems[0]
    pot = oracle_potential(spec)
    go = prob.view(g0, 0)[0].numpy()
    r = oracle.mala_step(pot, paths[0][0], S0[0], go, eta[0][0], logu[0], 2e-4, w.D, w.beta, w.dt)
    assert abs(la[0] - r["log_alpha"]) <= 1e-9 * (1 + abs(r["log_alpha"]))
    assert bool(nacc[0]) == r["accepted"]
    expect = r["prop"] if r["accepted"] else paths[0][0]
    assert np.max(np.abs(prob.view(pos1, 0)[0].numpy() - expect)) <= 1e-12
    if r["accepted"]:
        assert abs(S1[0] - r["S_prop"]) <= 1e-12 * r["S_prop"]


def test_mala_update_fp32_matches_oracle(pamd):
    w = inputs.workload("lj108", "small")
    h = 2e-6
    prob, paths, eta, logu, S0, g0, pos1, g1, S1, nacc, la = _mala_case(pamd, w, "fp32", h, 4)
    spec = w.systems[0]
    pot = oracle_potential(spec)
    go = prob.view(g0, 0)[0].double().numpy()
    r = oracle.mala_step(pot, paths[0][0], S0[0], go, eta[0][0], logu[0], h, w.D, w.beta, w.dt,
                         store_f32=True, nthreads=8)
    # log alpha agrees to the FP32 rounding of the proposal (a few 1e-3 absolute here)
    assert abs(la[0] - r["log_alpha"]) <= 5e-3 * (1 + abs(r["log_alpha"]))
    if abs(logu[0] - r["log_alpha"]) > 1e-2:
        assert bool(nacc[0]) == r["accepted"]
    expect = r["prop"] if nacc[0] else paths[0][0]
    got = prob.view(pos1, 0)[0].double().numpy()
    assert np.max(np.abs(got - expect)) <= 4 * np.spacing(np.float32(np.abs(expect).max()))


def test_path_update_keeps_cached_action_consistent(pamd):
    """After many updates (captured as a CUDA graph) the cached S and grad equal a
    fresh evaluation of the updated path, and the tail slice never moved."""
    w = inputs.workload("lj108", "small")
    paths = start_paths(w, "fp32")
    prob = _problem(pamd, w, "fp32")
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    x0 = prob.view(buf, 0)[:, 0].clone()
    pamd.path_update(prob, buf, g, S, 1e-6, n_updates=20, seed=11, counter=100, n_accepted=nacc)
    pamd.path_update(prob, buf, g, S, 1e-6, n_updates=20, seed=11, counter=120, n_accepted=nacc)
    torch.cuda.synchronize()
    S2, g2 = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    assert torch.equal(S2, S)
    assert torch.equal(g2, g)
    assert torch.equal(prob.view(buf, 0)[:, 0], x0)
    assert 0 < int(nacc.sum()) <= 40 * prob.n_chains


def test_host_buffers_match_device_buffers(pamd):
    w = inputs.workload("ragged", "small")
    paths = start_paths(w, "fp32")
    prob = _problem(pamd, w, "fp32")
    dbuf = _upload(pamd, prob, paths)
    hbuf = dbuf.cpu().pin_memory()
    Sd, gd = pamd.action_grad(prob, dbuf)
    torch.cuda.synchronize()
    Sh = torch.zeros(prob.n_chains, dtype=torch.float64).pin_memory()
    gh = torch.zeros_like(hbuf).pin_memory()
    pamd.action_grad(prob, hbuf, Sh, gh)
    assert torch.equal(Sh, Sd.cpu())
    assert torch.equal(gh, gd.cpu())
    # pageable host memory works too
    hp = dbuf.cpu()
    Sp, gp = pamd.action_grad(prob, hp)
    assert torch.equal(Sp, Sd.cpu()) and torch.equal(gp, gd.cpu())


@pytest.mark.parametrize("name,precision,n_updates",
                         [("ragged", "fp32", 1), ("ragged", "fp64", 2), ("lj500", "fp32", 3),
                          ("ho3d", "fp32", 2), ("mixed", "fp32", 2)])
def test_path_update_host_buffers_match_device_buffers(pamd, name, precision, n_updates):
    """With host buffers the update is pipelined over chunks of chains (copies of one
    chunk overlap the updates of another); every chain must come out bit for bit as
    from one update over device buffers.  The host-side S, acceptance counts and
    log alpha are covered, and a mix of host and device buffers.  "mixed" runs two
    block-size classes per chunk."""
    w = _workload(name)
    paths = start_paths(w, precision)
    prob = _problem(pamd, w, precision)
    h = 2e-7 if name != "ho3d" else 1e-5
    d_pos = _upload(pamd, prob, paths)
    start = d_pos.cpu()
    S0, g0 = pamd.action_grad(prob, d_pos)
    torch.cuda.synchronize()
    h_pos, h_grad = d_pos.cpu().pin_memory(), g0.cpu().pin_memory()
    h_S = S0.cpu().pin_memory()
    h_acc = torch.zeros(prob.n_chains, dtype=torch.int32).pin_memory()
    h_la = torch.zeros(prob.n_chains, dtype=torch.float64).pin_memory()
    d_acc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    d_la = torch.zeros(prob.n_chains, dtype=torch.float64, device="cuda")
    for rep in range(2):
        pamd.path_update(prob, d_pos, g0, S0, h, n_updates, seed=11, counter=7 + rep,
                         n_accepted=d_acc, log_alpha=d_la)
        pamd.path_update(prob, h_pos, h_grad, h_S, h, n_updates, seed=11, counter=7 + rep,
                         n_accepted=h_acc, log_alpha=h_la)
    torch.cuda.synchronize()
    assert int(d_acc.sum()) > 0 and not torch.equal(d_pos.cpu(), start)
    assert torch.equal(h_pos, d_pos.cpu())
    assert torch.equal(h_grad, g0.cpu())
    assert torch.equal(h_S, S0.cpu())
    assert torch.equal(h_acc, d_acc.cpu())
    assert torch.equal(h_la, d_la.cpu())
    # mixed: host path, device gradient cache and counts
    m_pos = h_pos.clone().pin_memory()
    m_grad, m_S, m_acc = g0.clone(), S0.clone(), d_acc.clone()
    pamd.path_update(prob, d_pos, g0, S0, h, 1, seed=12, counter=1, n_accepted=d_acc)
    pamd.path_update(prob, m_pos, m_grad, m_S, h, 1, seed=12, counter=1, n_accepted=m_acc)
    torch.cuda.synchronize()
    assert torch.equal(m_pos, d_pos.cpu())
    assert torch.equal(m_grad, g0) and torch.equal(m_S, S0) and torch.equal(m_acc, d_acc)


def test_autograd_function_and_finite_differences(pamd):
    """PamdAction: backward is the hand-written adjoint; it matches central finite
    differences of the kernel's own action (h = 1e-3, FP64 path) and the oracle."""
    w = inputs.workload("lj108", "small")
    spec = inputs.SystemSpec("lj", 108, 3, 24, 1)
    w = inputs.Workload("lj108", [spec], dt=1e-4)
    paths = start_paths(w, "fp64")
    prob = _problem(pamd, w, "fp64")
    buf = _upload(pamd, prob, paths).requires_grad_(True)
    S = pamd.PamdAction.apply(buf, prob)
    S.sum().backward()
    g = buf.grad.detach()
    rng = inputs.rng(17)
    for _ in range(4):
        v = torch.from_numpy(rng.standard_normal(prob.span)).cuda()
        v /= v.norm()
        hh = 1e-3
        Sp = pamd.action(prob, (buf.detach() + hh * v).contiguous())
        Sm = pamd.action(prob, (buf.detach() - hh * v).contiguous())
        fd = float((Sp - Sm).sum()) / (2 * hh)
        an = float((g * v).sum())
        assert abs(fd - an) <= 1e-4 * (abs(an) + 1e-3 * float(g.norm()))
    So, go = oracle.action_grad(oracle_potential(spec), paths[0][0], w.D, w.beta, w.dt)
    assert rel(prob.view(g.cpu(), 0)[0].numpy(), go) <= 1e-12
    # fp32 through autograd, weighted backward
    prob32 = _problem(pamd, w, "fp32")
    b32 = _upload(pamd, prob32, [p.astype(np.float32).astype(np.float64) for p in paths])
    b32.requires_grad_(True)
    S32 = pamd.PamdAction.apply(b32, prob32)
    (3.0 * S32).sum().backward()
    _, g32 = pamd.action_grad(prob32, b32.detach())
    assert torch.allclose(b32.grad, 3.0 * g32, rtol=1e-6, atol=0)


def test_invalid_arguments_are_rejected(pamd):
    with pytest.raises(pamd.PamdError):
        prob = pamd.Problem([pamd.System("lj", 10, 3, 4, 1, box=4.0, rc=2.5)], 1, 1, 1e-4)
        pamd.action(prob, prob.empty("cuda"))  # rc > box/2
    with pytest.raises(pamd.PamdError):
        prob = pamd.Problem([pamd.System("lj", 2000, 3, 4, 1, box=40.0, rc=2.5)], 1, 1, 1e-4)
        pamd.action(prob, prob.empty("cuda"))  # N beyond the supported maximum
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, 8, 1)], 1, 1, 1e-2)
    buf = prob.empty("cuda")
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pamd.PamdError):
        pamd.path_update(prob, buf, buf.clone(), S, h=-1.0)


def test_misaligned_device_buffers_are_refused(pamd):
    """A device buffer at an address that is not 16-byte aligned is refused with
    PAMD_ERR_ARG by every entry point that takes path-shaped buffers, before any
    other check: each problem here is also unsupported (an LJ system of N = 2000,
    an oscillator slice of 9000 elements for the allocation-free call), so a
    missing alignment check would report PAMD_ERR_UNSUPPORTED instead, still
    without launching anything."""
    import ctypes
    from paper_1907_09529_gb300 import _lib
    lj = pamd.Problem([pamd.System("lj", 2000, 3, 2, 1, box=20.0, rc=2.5)], 1.0, 1.0, 1e-4)
    base = torch.zeros(lj.span + 64, dtype=torch.float32, device="cuda")
    bad = base[1:]  # 4 bytes past a 16-byte boundary
    assert bad.data_ptr() % 16 == 4
    good = torch.zeros_like(base)
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    sig = torch.zeros(3, dtype=torch.float64, device="cuda")
    calls = [lambda: pamd.action(lj, bad),
             lambda: pamd.action_grad(lj, bad),
             lambda: pamd.action_grad(lj, good, S, bad),
             lambda: pamd.action_grad_hs(lj, bad, sig),
             lambda: pamd.path_update(lj, bad, good, S, 1e-6),
             lambda: pamd.euler_reference(lj, bad),
             lambda: pamd.mala_propose(lj, good, good, 1e-6, prop=bad),
             lambda: pamd.mala_reverse(lj, good, bad, good, 1e-6),
             lambda: pamd.mala_commit(lj, bad, good, S, good, good, S,
                                      torch.zeros(1, dtype=torch.int32, device="cuda")),
             lambda: pamd.lj_pair_counts(lj, bad)]
    for k, call in enumerate(calls):
        with pytest.raises(pamd.PamdError) as ei:
            call()
        assert ei.value.status == -1, (k, ei.value.status)
    ho = pamd.Problem([pamd.System("harmonic", 3000, 3, 2, 1)], 1.0, 1.0, 1e-3)
    hbase = torch.zeros(ho.span + 64, dtype=torch.float32, device="cuda")
    with pytest.raises(pamd.PamdError) as ei:
        _lib.pamd_ho_action_grad_noalloc(ho.ref, ctypes.c_void_p(hbase[1:].data_ptr()),
                                         ctypes.c_void_p(S.data_ptr()),
                                         ctypes.c_void_p(hbase.data_ptr()), None)
    assert ei.value.status == -1
    torch.cuda.synchronize()


def test_nonfinite_action_is_reported(pamd):
    """Two particles on top of each other give an infinite action; the library
    flags it on the device and pamd_device_status reports it once."""
    prob = pamd.Problem([pamd.System("lj", 4, 3, 3, 1, box=6.0, rc=2.5)], 1.0, 1.0, 1e-4)
    buf = prob.empty("cuda")
    v = prob.view(buf, 0)
    v[0, :, :, :] = torch.tensor([[0.5, 2.0, 3.5, 5.0]] * 3, device="cuda")
    v[0, :, :, 1] = v[0, :, :, 0]  # particles 0 and 1 coincide at every slice
    pamd.device_status()  # clear anything earlier
    S, g = pamd.action_grad(prob, buf)
    with pytest.raises(pamd.PamdError) as ei:
        pamd.device_status()
    assert ei.value.status == -5
    pamd.device_status()  # cleared


def test_checkpoint_resume_is_bitwise_identical(pamd, tmp_path):
    """20 updates in one run == 10 updates, checkpoint, reload, 10 more updates."""
    from paper_1907_09529_gb300 import checkpoint
    w = inputs.workload("lj108", "small")
    paths = start_paths(w, "fp32")
    prob = _problem(pamd, w, "fp32")

    def fresh():
        buf = _upload(pamd, prob, paths)
        S, g = pamd.action_grad(prob, buf)
        return checkpoint.RunState(buf, g, S, torch.zeros(prob.n_chains, dtype=torch.int32,
                                                         device="cuda"), seed=5, counter=1000)

    a = fresh()
    pamd.path_update(prob, a.pos, a.grad, a.S, 1e-6, n_updates=20, seed=a.seed, counter=a.counter,
                     n_accepted=a.n_accepted)
    b = fresh()
    pamd.path_update(prob, b.pos, b.grad, b.S, 1e-6, n_updates=10, seed=b.seed, counter=b.counter,
                     n_accepted=b.n_accepted)
    b.counter += 10
    f = str(tmp_path / "run.pt")
    checkpoint.save(f, prob, b)
    c = checkpoint.load(f, prob)
    pamd.path_update(prob, c.pos, c.grad, c.S, 1e-6, n_updates=10, seed=c.seed, counter=c.counter,
                     n_accepted=c.n_accepted)
    torch.cuda.synchronize()
    assert torch.equal(prob.view(a.pos, 0), prob.view(c.pos, 0))
    assert torch.equal(a.S, c.S) and torch.equal(a.n_accepted, c.n_accepted)
    assert torch.equal(prob.view(a.grad, 0), prob.view(c.grad, 0))


def test_update_graph_is_captured_once(pamd):
    """Repeated multi-update calls on the same buffers replay one cached graph: the
    cache must not grow call after call (the graph key compares its fields, not the
    bytes of a padded struct)."""
    w = inputs.workload("lj108", "small")
    paths = start_paths(w, "fp32")
    pamd.release_cache()
    prob = _problem(pamd, w, "fp32")
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    for rep in range(4):
        pamd.path_update(prob, buf, g, S, 1e-6, n_updates=3, seed=3, counter=10 * rep,
                         n_accepted=nacc)
    torch.cuda.synchronize()
    n_plans, n_graphs = pamd.cache_stats()
    assert (n_plans, n_graphs) == (1, 1)
    pamd.path_update(prob, buf, g, S, 1e-6, n_updates=2, seed=3, counter=99, n_accepted=nacc)
    torch.cuda.synchronize()
    assert pamd.cache_stats() == (1, 2)


@pytest.mark.parametrize("name", ["lj500", "ragged"])
def test_pipelined_gradient_pass_equals_two_pass_form(pamd, name):
    """The pipelined gradient walk (the Hessian-vector product of one step pair
    interleaved with the force of the next) only reorders independent arithmetic,
    and a window whose particles stay within (L/2 - rc)/4 of its reference uses the
    image shift rounded once per list entry, which is then the shift rounded at
    every slice: S and the gradient are bitwise the same with either form and
    either shift rule."""
    import os
    w = inputs.workload(name, "small")
    paths = start_paths(w, "fp32")
    outs = []
    try:
        for env in ({}, {"PAMD_LJ_NO_PIPE": "1"}, {"PAMD_LJ_PER_STEP_SHIFT": "1"},
                    {"PAMD_LJ_NO_PIPE": "1", "PAMD_LJ_PER_STEP_SHIFT": "1"}):
            for key in ("PAMD_LJ_NO_PIPE", "PAMD_LJ_PER_STEP_SHIFT"):
                os.environ.pop(key, None)
            os.environ.update(env)
            pamd.release_cache()
            prob = _problem(pamd, w, "fp32")
            buf = _upload(pamd, prob, paths)
            S, g = pamd.action_grad(prob, buf)
            S1 = pamd.action(prob, buf)
            torch.cuda.synchronize()
            outs.append((S.cpu(), g.cpu(), S1.cpu()))
    finally:
        for key in ("PAMD_LJ_NO_PIPE", "PAMD_LJ_PER_STEP_SHIFT"):
            os.environ.pop(key, None)
        pamd.release_cache()
    for S, g, S1 in outs[1:]:
        assert torch.equal(outs[0][0], S)
        assert torch.equal(outs[0][1], g)
        assert torch.equal(outs[0][2], S1)


@pytest.mark.parametrize("precision,n_updates", [("fp64", 8), ("fp32", 6)])
def test_ragged_path_updates_match_oracle_step_by_step(pamd, parity_report, precision,
                                                       n_updates):
    """A ragged batch of five LJ systems through successive pamd_path_update calls
    with explicit noise and log uniforms: at every step each chain's log alpha,
    accept decision, updated path, action and gradient agree with the oracle's MALA
    step (oracle.mala_step) started from the library's current path.  The uniform
    of a chain is redrawn when it falls within twice the stated agreement of log
    alpha (1e-9 in FP64; 5e-3 in FP32, where each side rounds the proposal to
    float), relative to 1 + |log alpha|, so that every decision is determined."""
    w = inputs.workload("ragged", "small")
    h = 2e-7
    f32 = precision == "fp32"
    paths = start_paths(w, precision)
    prob = _problem(pamd, w, precision)
    buf = _upload(pamd, prob, paths)
    S, g = pamd.action_grad(prob, buf)
    pots = [oracle_potential(s) for s in w.systems]
    rng = inputs.rng(2024 + n_updates)
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    la = torch.zeros(prob.n_chains, dtype=torch.float64, device="cuda")
    tol_la = 5e-3 if f32 else 1e-9
    margin = 2 * tol_la
    worst = {"log_alpha_abs": 0.0, "path_maxabs": 0.0, "S_rel": 0.0, "grad_rel_2norm": 0.0}
    n_acc = 0
    for k in range(n_updates):
        x = [prob.view(buf, q).cpu().double().numpy() for q in range(len(w.systems))]
        eta, logu, ref = [], np.zeros(prob.n_chains), {}
        for q, s in enumerate(w.systems):
            e = rng.standard_normal(x[q].shape)
            if f32:
                e = e.astype(np.float32).astype(np.float64)
            eta.append(e)
            for b in range(s.n_chains):
                c = prob.chain0[q] + b
                So, go = oracle.action_grad(pots[q], x[q][b], w.D, w.beta, w.dt, nthreads=8)
                lu = math.log(rng.random())
                r = oracle.mala_step(pots[q], x[q][b], So, go, e[b], lu, h, w.D, w.beta, w.dt,
                                     store_f32=f32, nthreads=8)
                # log alpha does not depend on u: redraw u until the decision is clear
                while abs(lu - r["log_alpha"]) <= margin * (1 + abs(r["log_alpha"])):
                    lu = math.log(rng.random())
                logu[c] = lu
                ref[c] = (q, b, lu < r["log_alpha"], r)
        nbuf = _upload(pamd, prob, eta)
        pamd.path_update(prob, buf, g, S, h, 1, noise=nbuf, log_u=torch.from_numpy(logu).cuda(),
                         n_accepted=nacc, log_alpha=la)
        torch.cuda.synchronize()
        la_k, S_k, g_k = la.cpu().numpy(), S.cpu().numpy(), g.cpu()
        for c, (q, b, accepted, r) in ref.items():
            d_la = abs(la_k[c] - r["log_alpha"])
            assert d_la <= tol_la * (1 + abs(r["log_alpha"])), (k, c, la_k[c], r["log_alpha"])
            got = prob.view(buf, q)[b].cpu().double().numpy()
            expect = r["prop"] if accepted else x[q][b]
            ep = np.abs(got - expect).max()
            lim = (4 * np.spacing(np.float32(np.abs(expect).max())) if f32
                   else 1e-12 * max(1.0, np.abs(expect).max()))
            assert ep <= lim, (k, c, accepted, ep)
            # cached action and gradient of the updated path against the oracle's
            So, go = oracle.action_grad(pots[q], got, w.D, w.beta, w.dt, nthreads=8)
            tol = 1e-5 if f32 else 1e-12
            es = abs(S_k[c] - So) / So
            eg = rel(prob.view(g_k, q)[b].double().numpy(), go)
            assert es <= tol and eg <= tol, (k, c, es, eg)
            n_acc += int(accepted)
            worst["log_alpha_abs"] = max(worst["log_alpha_abs"], d_la)
            worst["path_maxabs"] = max(worst["path_maxabs"], ep)
            worst["S_rel"] = max(worst["S_rel"], es)
            worst["grad_rel_2norm"] = max(worst["grad_rel_2norm"], eg)
    assert int(nacc.sum()) == n_acc and n_acc > 0
    parity_report.record(f"ragged_updates_{precision}",
                         f"test_ragged_path_updates_match_oracle_step_by_step ({n_updates} "
                         f"updates, 5 systems)", **worst)
