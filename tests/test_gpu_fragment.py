"""Multilevel sliding-and-sampling Monte Carlo (Sec. III, Fig. 5) on the GPU:
parity with the oracle on the same fragmentation, normals and uniforms, and
the stationary path distribution of the oscillator."""
import math

import numpy as np
import pytest

import oracle
import pamd_inputs as inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pamd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    return pamd


@pytest.mark.parametrize("precision,T,d,l_min,l_max,dt", [
    ("fp64", 16, 1, 3, 3, 0.4),     # the paper's oscillator Simulation 1 shape
    ("fp64", 256, 1, 4, 5, 0.4),    # Simulation 2 shape
    ("fp64", 1024, 3, 2, 6, 0.01),
    ("fp32", 256, 1, 4, 5, 0.4),
])
def test_fragment_step_matches_oracle(pamd, precision, T, d, l_min, l_max, dt):
    B, D, beta = 4, 1.0, 1.0
    rng = inputs.rng(200 + T + d)
    prob = pamd.Problem([pamd.System("harmonic", 1, d, T, B, k=1.0)], D, beta, dt,
                        precision=precision)
    paths = rng.standard_normal((B, T + 1, d, 1))
    noise = rng.standard_normal((B, T + 1, d, 1))
    if precision == "fp32":
        paths = paths.astype(np.float32).astype(np.float64)
        noise = noise.astype(np.float32).astype(np.float64)
    levels = rng.integers(l_min, l_max + 1, size=B)
    offsets = np.array([rng.integers(0, 1 << l) for l in levels])
    F = pamd.fragment_slots(prob, l_min)
    log_u = np.log(rng.random((B, F)))
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths).to(prob.dtype))
    nbuf = prob.empty("cuda")
    prob.view(nbuf, 0).copy_(torch.from_numpy(noise).to(prob.dtype))
    acc, prop = pamd.fragment_mc(prob, buf, l_min, l_max, 1,
                                 levels=torch.from_numpy(levels).int().cuda(),
                                 offsets=torch.from_numpy(offsets).int().cuda(), noise=nbuf,
                                 log_u=torch.from_numpy(log_u.reshape(-1)).cuda())
    torch.cuda.synchronize()
    got = prob.view(buf, 0).double().cpu().numpy()
    pot = oracle.harmonic(1.0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for b in range(B):
        x = paths[b].copy()
        nf, na, npr = oracle.fragment_step(pot, x, int(levels[b]), int(offsets[b]), noise[b],
                                           log_u[b, :oracle.n_fragments(T, int(levels[b]),
                                                                        int(offsets[b]))],
                                           D, beta, dt)
        assert int(acc[b]) == na and int(prop[b]) == npr, (b, int(acc[b]), na)
        assert np.abs(got[b] - x).max() <= tol * max(1.0, np.abs(x).max()), b
        assert np.array_equal(got[b][0], paths[b][0])


def test_fragment_mc_samples_oscillator_paths(pamd):
    """20000 chains of T = 8 steps, 600 Philox-driven MC steps at levels 1..2:
    x_4 and x_8 across chains follow the exact AR(1) marginals of exp(-S)."""
    B, T, dt, x0v = 20000, 8, 0.1, 1.0
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, T, B, k=1.0)], 1.0, 1.0, dt,
                        precision="fp32")
    buf = prob.empty("cuda")
    prob.view(buf, 0)[:, 0].fill_(x0v)
    acc, prop = pamd.fragment_mc(prob, buf, 1, 2, n_steps=600, seed=2024, counter=0)
    torch.cuda.synchronize()
    x = prob.view(buf, 0)[:, :, 0, 0].double().cpu().numpy()
    assert np.all(x[:, 0] == x0v)
    rate = float(acc.sum()) / float(prop.sum())
    assert 0.3 < rate < 1.0
    a = 1 - dt
    for t in (4, 8):
        m = a ** t * x0v
        v = 2 * dt * (1 - a ** (2 * t)) / (1 - a ** 2)
        assert abs(x[:, t].mean() - m) < 5 * math.sqrt(v / B)
        assert abs(x[:, t].var() - v) < 5 * v * math.sqrt(2 / B)


def test_fragment_mc_rejects_lennard_jones(pamd):
    prob = pamd.Problem([pamd.System("lj", 8, 3, 16, 1, box=6.0, rc=2.5)], 1.0, 1.0, 1e-4)
    with pytest.raises(pamd.PamdError) as ei:
        pamd.fragment_mc(prob, prob.empty("cuda"), 1, 2)
    assert ei.value.status == -2


def test_shift_regenerate_matches_oracle(pamd):
    from paper_1907_09529_gb300 import integrator
    B, T, d, n_shift, D, dt = 3, 16, 2, 5, 0.7, 0.2
    rng = inputs.rng(301)
    prob = pamd.Problem([pamd.System("harmonic", 1, d, T, B)], D, 1.0, dt, precision="fp64")
    paths = rng.standard_normal((B, T + 1, d, 1))
    z = rng.standard_normal((B, n_shift, d, 1))
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths))
    out = prob.empty("cuda")
    traj = integrator.shift_regenerate(prob, buf, out, n_shift,
                                       noise=torch.from_numpy(z.reshape(-1)).cuda())
    torch.cuda.synchronize()
    traj = traj.view(B, n_shift, d, 1).cpu().numpy()
    got = prob.view(out, 0).cpu().numpy()
    for b in range(B):
        o, tr = oracle.shift_regenerate(paths[b], n_shift, z[b], D, dt)
        assert np.abs(got[b] - o).max() <= 1e-13
        assert np.array_equal(traj[b], tr)


def test_pamd_loop_reproduces_the_euler_chain_statistics(pamd):
    """The integrated trajectories of 4096 PAMD chains (N_path = 16, N_shift = 1,
    N_sample = 16, levels 1..3, dt = 0.1) have the stationary variance
    2 D dt / (1 - a^2) and lag-1 autocorrelation a = 1 - beta D k dt of the
    Euler-Maruyama chain whose path measure the sampler draws from."""
    from paper_1907_09529_gb300.integrator import PamdIntegrator
    B, T, dt = 4096, 16, 0.1
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, T, B, k=1.0)], 1.0, 1.0, dt,
                        precision="fp32")
    buf = prob.empty("cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    prob.view(buf, 0).copy_(torch.randn(prob.view(buf, 0).shape, generator=g, device="cuda"))
    integ = PamdIntegrator(prob, n_shift=1, n_sample=16, l_min=1, l_max=3, seed=77)
    integ.run(buf, 300)  # equilibrate
    traj = integ.run(buf, 1500).double().cpu().numpy()  # [events, chains]
    a = 1 - dt
    var_em = 2 * dt / (1 - a * a)
    x = traj
    v = (x ** 2).mean()
    c1 = (x[1:] * x[:-1]).mean() / v
    # effective samples ~ B * events / (2 tau), tau ~ 1/(1-a) = 10 steps
    n_eff = B * x.shape[0] / 20
    assert abs(v - var_em) < 6 * var_em * (2 / n_eff) ** 0.5 + 0.01 * var_em
    assert abs(c1 - a) < 0.01
    rate = float(integ.n_accepted.sum()) / float(integ.n_proposed.sum())
    assert 0.3 < rate < 1.0
