"""Parity at the full workload sizes, in the launch configuration the benchmark
times (default plan), against the CPU oracle.

Where the oracle cannot redo everything in seconds, it checks every chain's S
and the gradient at sampled slices (each computed locally from x_{t-1}, x_t,
x_{t+1}), or a property that holds at any size (the Euler-Maruyama invariant
S = sum xi^2 / 2).
"""
import math

import numpy as np
import pytest

import oracle
import pamd_inputs as inputs
from _common import gpu_system, oracle_potential, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pamd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    pamd.tune()
    return pamd


def _problem(pamd, w, precision="fp32"):
    return pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt,
                        precision=precision)


def test_ho3d_full_size(pamd, parity_report):
    """3D oscillator, T = 2^20, 64 chains: every chain's S and gradient."""
    w = inputs.workload("ho3d")
    spec = w.systems[0]
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    view = prob.view(buf, 0)
    paths = []
    for b in range(spec.n_chains):
        x = inputs.gaussian_path(w.seed * 1000 + b, 1, spec.T, 3, 1, 1.0)[0]
        x = x.astype(np.float32)
        view[b].copy_(torch.from_numpy(x))
        paths.append(x)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    pot = oracle_potential(spec)
    nth = oracle.max_threads()
    for b in range(spec.n_chains):
        So, go = oracle.action_grad(pot, paths[b].astype(np.float64), w.D, w.beta, w.dt,
                                    nthreads=nth)
        es = abs(S[b] - So) / So
        assert es <= 1e-5, b
        parity_report.record("ho3d", "test_ho3d_full_size", S_rel=es)
        if b % 8 == 0:
            gb = prob.view(g, 0)[b].double().cpu().numpy()
            eg, em = rel(gb, go), np.abs(gb - go).max() / np.abs(go).max()
            assert eg <= 1e-5 and em <= 1e-5
            parity_report.record("ho3d", "test_ho3d_full_size", grad_rel_2norm=eg,
                                 grad_rel_maxabs=em)


@pytest.fixture(scope="module")
def lj500_paths():
    """LJ N = 500, T = 16384, 8 chains: the oracle's Euler-Maruyama start paths
    (rounded to float32), shared by the full-size lj500 tests."""
    w = inputs.workload("lj500")
    spec = w.systems[0]
    pot = oracle_potential(spec)
    x0 = inputs.initial_positions(spec, 1)
    xi = inputs.euler_noise(spec, w.seed)
    paths = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True,
                               nthreads=oracle.max_threads())
    return w, spec, pot, paths


def test_lj500_full_size(pamd, parity_report, lj500_paths):
    """LJ N = 500, T = 16384, 8 chains (oracle Euler-Maruyama start paths): every
    chain's S, and the gradient at 48 sampled slices per chain, incl. both ends."""
    w, spec, pot, paths = lj500_paths
    nth = oracle.max_threads()
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths).float())
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    gv = prob.view(g, 0)
    rng = inputs.rng(123)
    for b in range(spec.n_chains):
        So = oracle.action_grad(pot, paths[b], w.D, w.beta, w.dt, grad=False, nthreads=nth)
        es = abs(S[b] - So) / So
        assert es <= 1e-5, (b, S[b], So)
        ts = np.unique(np.concatenate([[0, 1, spec.T - 1, spec.T, 31, 32, 33],
                                       rng.integers(0, spec.T + 1, 41)]))
        go = oracle.grad_slices(pot, paths[b], w.D, w.beta, w.dt, ts)
        gk = gv[b, torch.from_numpy(ts).long()].double().cpu().numpy()
        eg, em = rel(gk, go), np.abs(gk - go).max() / np.abs(go).max()
        assert eg <= 1e-5 and em <= 1e-5, b
        parity_report.record("lj500", "test_lj500_full_size (S of every chain; gradient at "
                             "48 sampled slices per chain)", S_rel=es, grad_rel_2norm=eg,
                             grad_rel_maxabs=em)


def test_lj500_hardsphere_full_size(pamd, parity_report, lj500_paths):
    """The hard-sphere path bias at full size: radii at 98 sampled slices (the tail
    and the nose among them) at four levels around the liquid's closest approach.
    Every chain's overlap decision equals the oracle's mirror of the kernels'
    single-precision rule at those slices, a finite S is the plain action bit for
    bit, and both outcomes occur."""
    w, spec, pot, paths = lj500_paths
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths).float())
    S0, _ = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S0 = S0.cpu().numpy()
    rng = inputs.rng(321)
    ts = np.unique(np.concatenate([[0, spec.T], rng.integers(1, spec.T, 96)]))
    n_inf = n_fin = 0
    for level in (0.75, 0.85, 0.90, 0.95):
        sig = np.zeros(spec.T + 1)
        sig[ts] = level
        S, _ = pamd.action_grad_hs(prob, buf, torch.from_numpy(sig).cuda(), with_grad=False)
        torch.cuda.synchronize()
        S = S.cpu().numpy()
        for b in range(spec.n_chains):
            x32 = paths[b].astype(np.float32)
            want = any(oracle.hs_overlap_f32(spec.box, spec.rc_eff, level, x32[t]) for t in ts)
            if want:
                assert S[b] == math.inf, (level, b)
                n_inf += 1
            else:
                assert S[b] == S0[b], (level, b)
                n_fin += 1
    assert n_inf > 0 and n_fin > 0
    parity_report.record("lj500_hardsphere", "test_lj500_hardsphere_full_size (overlap "
                         "decisions equal at 98 sampled slices, four radii)",
                         chains_infinite=n_inf, chains_finite=n_fin)


def test_lj500_timeslabs_full_size(pamd, parity_report, lj500_paths):
    """One lj500 path split into four time slabs held by this process, at full size:
    the gradient at every owned slice equals the whole-path call's bit for bit, and
    each chain's S (the slabs' FP64 parts summed) agrees to 1e-12."""
    from paper_1907_09529_gb300 import timeslab
    w, spec, pot, paths = lj500_paths
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths).float())
    S_ref, g_ref = pamd.action_grad(prob, buf)
    run = timeslab.SlabRun(prob, timeslab.LocalComm(4))
    bufs = [timeslab.scatter(prob, buf, lp) for lp in run.probs]
    S, G = run.action_grad(bufs)
    torch.cuda.synchronize()
    worst = 0.0
    for k, lp in enumerate(run.probs):
        worst = max(worst, float(((S[k] - S_ref).abs() / S_ref.abs()).max()))
        s = lp.systems[0]
        o = timeslab.owned_slices(s)
        lo, hi = s.first_slice + o.start, s.first_slice + o.stop
        assert torch.equal(lp.view(G[k], 0)[:, o], prob.view(g_ref, 0)[:, lo:hi]), k
    assert worst <= 1e-12
    parity_report.record("lj500_timeslab4", "test_lj500_timeslabs_full_size (S vs the whole-path "
                         "call; owned gradients bitwise)", S_rel=worst)


def test_lj108_full_size(pamd, parity_report):
    """LJ N = 108, T = 4096: complete S and gradient."""
    w = inputs.workload("lj108")
    spec = w.systems[0]
    pot = oracle_potential(spec)
    x0 = inputs.initial_positions(spec, 1)
    xi = inputs.euler_noise(spec, w.seed)
    paths = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True)
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths).float())
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    So, go = oracle.action_grad(pot, paths[0], w.D, w.beta, w.dt, nthreads=oracle.max_threads())
    es = abs(S[0].item() - So) / So
    gk = prob.view(g, 0)[0].double().cpu().numpy()
    eg, em = rel(gk, go), np.abs(gk - go).max() / np.abs(go).max()
    assert es <= 1e-5 and eg <= 1e-5 and em <= 1e-5
    parity_report.record("lj108", "test_lj108_full_size", S_rel=es, grad_rel_2norm=eg,
                         grad_rel_maxabs=em)


def test_ragged_full_size(pamd, parity_report):
    """32 LJ systems of N in [64, 864], T in [1024, 32768], one persistent launch:
    the Euler-Maruyama invariant on every chain (paths from the library's own
    Euler-Maruyama with Philox noise), and oracle parity on three systems whose
    paths the oracle generates."""
    w = inputs.workload("ragged")
    prob = _problem(pamd, w)
    buf = prob.empty("cuda")
    for q, s in enumerate(w.systems):
        prob.view(buf, q)[:, 0].copy_(torch.from_numpy(inputs.initial_positions(s, 1)).float())
    pamd.euler_reference(prob, buf, seed=77, counter=0)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    for q, s in enumerate(w.systems):
        c = prob.chain0[q]
        z = pamd.normals(77, 0, 0, c, s.T * 3 * s.N, e0=3 * s.N).double()
        half = 0.5 * float((z ** 2).sum())
        # residuals equal sqrt(2 D dt) xi up to the FP32 rounding of the stored slices
        assert abs(S[c] - half) <= 1e-4 * half, (q, S[c], half)
        parity_report.record("ragged", "test_ragged_full_size (Euler-Maruyama invariant, all "
                             "32 systems)", S_vs_invariant_rel=abs(S[c] - half) / half)
    # oracle parity on the three shortest systems, paths generated by the oracle
    order = sorted(range(len(w.systems)), key=lambda q: w.systems[q].T * w.systems[q].N)[:3]
    nth = oracle.max_threads()
    refs = {}
    for q in order:
        s = w.systems[q]
        pot = oracle_potential(s)
        x0 = inputs.initial_positions(s, 2)
        xi = inputs.euler_noise(s, w.seed * 1000 + q)
        p = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True, nthreads=nth)
        prob.view(buf, q).copy_(torch.from_numpy(p).float())
        refs[q] = (pot, p)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    for q, (pot, p) in refs.items():
        s = w.systems[q]
        So = oracle.action_grad(pot, p[0], w.D, w.beta, w.dt, grad=False, nthreads=nth)
        es = abs(S[prob.chain0[q]] - So) / So
        assert es <= 1e-5
        ts = np.array([0, 1, s.T // 2, s.T - 1, s.T])
        go = oracle.grad_slices(pot, p[0], w.D, w.beta, w.dt, ts)
        gk = prob.view(g, q)[0, torch.from_numpy(ts).long()].double().cpu().numpy()
        eg, em = rel(gk, go), np.abs(gk - go).max() / np.abs(go).max()
        assert eg <= 1e-5 and em <= 1e-5
        parity_report.record("ragged", "test_ragged_full_size (oracle on three systems; "
                             "gradient at 5 slices)", S_rel=es, grad_rel_2norm=eg,
                             grad_rel_maxabs=em)


def test_ho1d_thousand_updates_fp64(pamd, parity_report):
    """1D oscillator, T = 1024, plain FP64: 1000 seeded path updates with the
    noise and uniforms passed in, against the oracle's MALA on the same draws."""
    w = inputs.workload("ho1d")
    spec = w.systems[0]
    pot = oracle_potential(spec)
    h = 1e-3
    x0 = np.zeros((1, 1, 1))
    xi = inputs.euler_noise(spec, 9)
    path = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt)[0]
    prob = _problem(pamd, w, "fp64")
    buf = prob.empty("cuda")
    prob.view(buf, 0)[0].copy_(torch.from_numpy(path))
    S, g = pamd.action_grad(prob, buf)
    So, go = oracle.action_grad(pot, path, w.D, w.beta, w.dt)
    rng = inputs.rng(10)
    nbuf = prob.empty("cuda")
    lu = torch.zeros(1, dtype=torch.float64, device="cuda")
    nacc = torch.zeros(1, dtype=torch.int32, device="cuda")
    acc_o = 0
    x = path
    for it in range(1000):
        eta = rng.standard_normal(path.shape)
        logu = math.log(rng.random())
        prob.view(nbuf, 0)[0].copy_(torch.from_numpy(eta))
        lu.fill_(logu)
        pamd.path_update(prob, buf, g, S, h, 1, noise=nbuf, log_u=lu, n_accepted=nacc)
        r = oracle.mala_step(pot, x, So, go, eta, logu, h, w.D, w.beta, w.dt)
        if r["accepted"]:
            x, So, go = r["prop"], r["S_prop"], r["grad_prop"]
            acc_o += 1
    torch.cuda.synchronize()
    assert int(nacc.item()) == acc_o
    assert 100 < acc_o <= 1000
    got = prob.view(buf, 0)[0].cpu().numpy()
    ep = np.abs(got - x).max() / max(1.0, np.abs(x).max())
    assert ep <= 1e-10
    assert abs(S.item() - So) <= 1e-10 * So
    gk = prob.view(g, 0)[0].cpu().numpy()
    parity_report.record("ho1d", "test_ho1d_thousand_updates_fp64 (after 1000 updates)",
                         path_after_1000_updates_maxabs=ep, S_after_1000_updates_rel=abs(S.item() - So) / So,
                         grad_after_1000_updates_rel_2norm=rel(gk, go))


def test_lj108_autograd_finite_differences_full_size(pamd, parity_report):
    """LJ N = 108, T = 4096 through PamdAction (torch.autograd.Function): the
    backward (the hand-written adjoint) against central finite differences of the
    action with h = 1e-3, in the plain FP64 form, along four random unit
    directions of the whole path; the single-precision gradient through the same
    Function against the FP64 one."""
    w = inputs.workload("lj108")
    spec = w.systems[0]
    pot = oracle_potential(spec)
    x0 = inputs.initial_positions(spec, 1)
    xi = inputs.euler_noise(spec, w.seed)
    paths = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True)
    prob = _problem(pamd, w, "fp64")
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths))
    x = buf.clone().requires_grad_(True)
    S = pamd.PamdAction.apply(x, prob)
    S.sum().backward()
    g = x.grad.detach()
    rng = inputs.rng(4096)
    hh = 1e-3
    worst = 0.0
    for _ in range(4):
        v = torch.from_numpy(rng.standard_normal(prob.span)).cuda()
        v /= v.norm()
        Sp = pamd.action(prob, (buf + hh * v).contiguous())
        Sm = pamd.action(prob, (buf - hh * v).contiguous())
        fd = float((Sp - Sm).sum()) / (2 * hh)
        an = float((g * v).sum())
        err = abs(fd - an) / (abs(an) + 1e-3 * float(g.norm()))
        worst = max(worst, err)
        assert err <= 1e-4, (fd, an)
    # the FP64 adjoint itself against the oracle's gradient
    So, go = oracle.action_grad(pot, paths[0], w.D, w.beta, w.dt, nthreads=oracle.max_threads())
    e64 = rel(prob.view(g, 0)[0].cpu().numpy(), go)
    assert e64 <= 1e-12 and abs(S.item() - So) <= 1e-12 * So
    # float32 positions through the same Function: gradient against the FP64 one
    p32 = _problem(pamd, w, "fp32")
    b32 = p32.empty("cuda")
    p32.view(b32, 0).copy_(torch.from_numpy(paths).float())
    b32.requires_grad_(True)
    S32 = pamd.PamdAction.apply(b32, p32)
    S32.sum().backward()
    e32 = rel(p32.view(b32.grad, 0)[0].double().cpu().numpy(), go)
    assert e32 <= 1e-5 and abs(S32.item() - So) <= 1e-5 * So
    parity_report.record("lj108", "test_lj108_autograd_finite_differences_full_size",
                         fd_vs_adjoint_rel=worst, fp64_grad_rel_2norm=e64,
                         fp64_S_rel=abs(S.item() - So) / So,
                         autograd_fp32_grad_rel_2norm=e32)
