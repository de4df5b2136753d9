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


def test_ho3d_full_size(pamd):
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
        assert abs(S[b] - So) <= 1e-5 * So, b
        if b % 8 == 0:
            gb = prob.view(g, 0)[b].double().cpu().numpy()
            assert rel(gb, go) <= 1e-5
            assert np.abs(gb - go).max() <= 1e-5 * np.abs(go).max()


def test_lj500_full_size(pamd):
    """LJ N = 500, T = 16384, 8 chains (oracle Euler-Maruyama start paths): every
    chain's S, and the gradient at 48 sampled slices per chain, incl. both ends."""
    w = inputs.workload("lj500")
    spec = w.systems[0]
    pot = oracle_potential(spec)
    nth = oracle.max_threads()
    x0 = inputs.initial_positions(spec, 1)
    xi = inputs.euler_noise(spec, w.seed)
    paths = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True, nthreads=nth)
    del xi
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
        assert abs(S[b] - So) <= 1e-5 * So, (b, S[b], So)
        ts = np.unique(np.concatenate([[0, 1, spec.T - 1, spec.T, 31, 32, 33],
                                       rng.integers(0, spec.T + 1, 41)]))
        go = oracle.grad_slices(pot, paths[b], w.D, w.beta, w.dt, ts)
        gk = gv[b, torch.from_numpy(ts).long()].double().cpu().numpy()
        assert rel(gk, go) <= 1e-5, b
        assert np.abs(gk - go).max() <= 1e-5 * np.abs(go).max(), b


def test_lj108_full_size(pamd):
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
    assert abs(S[0].item() - So) <= 1e-5 * So
    gk = prob.view(g, 0)[0].double().cpu().numpy()
    assert rel(gk, go) <= 1e-5
    assert np.abs(gk - go).max() <= 1e-5 * np.abs(go).max()


def test_ragged_full_size(pamd):
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
        assert abs(S[prob.chain0[q]] - So) <= 1e-5 * So
        ts = np.array([0, 1, s.T // 2, s.T - 1, s.T])
        go = oracle.grad_slices(pot, p[0], w.D, w.beta, w.dt, ts)
        gk = prob.view(g, q)[0, torch.from_numpy(ts).long()].double().cpu().numpy()
        assert rel(gk, go) <= 1e-5


def test_ho1d_thousand_updates_fp64(pamd):
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
    assert np.abs(got - x).max() <= 1e-10 * max(1.0, np.abs(x).max())
    assert abs(S.item() - So) <= 1e-10 * So
