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
    ("fp32", 4096, 1, 4, 8, 0.4),   # Simulation 3 shape
    ("fp32", 2048, 1, 3, 7, 0.4),   # 5 warps per chain
    ("fp32", 1000, 1, 1, 4, 0.1),   # level 1: up to three fragments per quad
    ("fp64", 40000, 1, 5, 9, 0.4),  # too large for one CTA: thread-per-fragment kernel
    ("fp32", 30000, 2, 3, 6, 0.05),
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


def test_flat_regeneration_matches_oracle(pamd):
    """PAMD_FLAG_REGENERATE_FLAT: the regrown nose is the line x_T, i.e. the
    oracle's regeneration with zero noise, exactly."""
    from paper_1907_09529_gb300 import integrator
    B, T, d, n_shift = 3, 40, 2, 9
    rng = inputs.rng(303)
    prob = pamd.Problem([pamd.System("harmonic", 1, d, T, B)], 0.7, 1.0, 0.2, precision="fp64",
                        regenerate_flat=True)
    paths = rng.standard_normal((B, T + 1, d, 1))
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths))
    out = prob.empty("cuda")
    traj = integrator.shift_regenerate(prob, buf, out, n_shift, seed=5, counter=1)
    torch.cuda.synchronize()
    got = prob.view(out, 0).cpu().numpy()
    for b in range(B):
        o, tr = oracle.shift_regenerate(paths[b], n_shift, np.zeros((n_shift, d, 1)), 0.7, 0.2)
        assert np.array_equal(got[b], o)
    assert np.array_equal(traj.view(B, n_shift, d, 1).cpu().numpy(), paths[:, 1:n_shift + 1])


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


def test_fragment_mc_skips_invalid_cuts(pamd):
    """A chain given a level outside [l_min, l_max] or an offset outside
    [0, 2^level) keeps its path and proposes nothing; the others still move."""
    B, T = 4, 64
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, T, B)], 1.0, 1.0, 0.1, precision="fp64")
    rng = inputs.rng(404)
    paths = rng.standard_normal((B, T + 1, 1, 1))
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(paths))
    levels = torch.tensor([1, 5, 3, 3], dtype=torch.int32, device="cuda")
    offsets = torch.tensor([0, 0, 8, -1], dtype=torch.int32, device="cuda")
    F = pamd.fragment_slots(prob, 2)
    log_u = torch.full((B * F,), -np.inf, dtype=torch.float64, device="cuda")  # accept all
    acc, prop = pamd.fragment_mc(prob, buf, 2, 4, 1, levels=levels, offsets=offsets,
                                 log_u=log_u)
    torch.cuda.synchronize()
    got = prob.view(buf, 0).cpu().numpy()
    assert prop.tolist() == [0, 0, 0, 0] and acc.tolist() == [0, 0, 0, 0]
    assert np.array_equal(got, paths)
    levels[1], offsets[1] = 4, 15
    acc, prop = pamd.fragment_mc(prob, buf, 2, 4, 1, levels=levels, offsets=offsets,
                                 log_u=log_u)
    torch.cuda.synchronize()
    got = prob.view(buf, 0).cpu().numpy()
    assert prop.tolist() == [0, 5, 0, 0] and acc.tolist() == [0, 5, 0, 0]
    assert np.array_equal(got[[0, 2, 3]], paths[[0, 2, 3]])
    assert not np.array_equal(got[1, 16:], paths[1, 16:])


def _philox_log_u(seed, counter, chain, f):
    w = oracle.philox([f, chain, counter & 0xFFFFFFFF, ((counter >> 32) & 0xFFFF) | (5 << 16)],
                      [seed & 0xFFFFFFFF, seed >> 32])
    mant = (int(w[0]) >> 5) * 67108864 + (int(w[1]) >> 6)
    return math.log((mant + 1.0) * 2.0 ** -53)


def test_fragment_mc_full_size_sampled_chains(pamd):
    """The Simulation 3 shape at full batch (16384 chains, N_path = 4096,
    levels 4..8, Philox-driven): sampled chains match the oracle fed with the
    same Philox cut (stream 3), trial normals (stream 4) and uniforms (stream 5)."""
    w = inputs.workload("ho_pamd")
    spec = w.systems[0]
    B, T = spec.n_chains, spec.T
    l_min, l_max, seed, counter = 4, 8, 0x5EED1907, 11
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, T, B)], w.D, w.beta, w.dt,
                        precision="fp32")
    buf = prob.empty("cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    prob.view(buf, 0).copy_(torch.randn(prob.view(buf, 0).shape, generator=g, device="cuda"))
    before = prob.view(buf, 0).double().cpu().numpy()
    acc, prop = pamd.fragment_mc(prob, buf, l_min, l_max, 1, seed=seed, counter=counter)
    torch.cuda.synchronize()
    after = prob.view(buf, 0).double().cpu().numpy()
    pot = oracle.harmonic(1.0)
    rng = inputs.rng(77)
    sample = sorted(set(rng.integers(0, B, size=24).tolist()) | {0, B - 1})
    for c in sample:
        wc = oracle.philox([0, c, counter, 3 << 16], [seed & 0xFFFFFFFF, seed >> 32])
        l = l_min + int(wc[0]) % (l_max - l_min + 1)
        o = int(wc[1]) % (1 << l)
        nf = oracle.n_fragments(T, l, o)
        z = oracle.normals(seed, counter, 4, c, T + 1).astype(np.float32).astype(np.float64)
        lu = np.array([_philox_log_u(seed, counter, c, f) for f in range(nf)])
        x = before[c].copy()
        _, na, npr = oracle.fragment_step(pot, x, l, o, z.reshape(T + 1, 1, 1), lu,
                                          w.D, w.beta, w.dt)
        assert (int(acc[c]), int(prop[c])) == (na, npr), c
        assert np.abs(after[c] - x).max() <= 2e-5 * max(1.0, np.abs(x).max()), c
    assert float(acc.sum()) > 0


@pytest.mark.parametrize("precision,d,T,n_sample,n_shift,l_min,l_max,opts", [
    ("fp32", 1, 4096, 1, 64, 4, 8, ""),    # fused epilogue (one-line paths)
    ("fp32", 1, 256, 3, 16, 2, 5, ""),
    ("fp64", 1, 1024, 2, 7, 3, 6, ""),
    ("fp32", 3, 512, 2, 10, 2, 4, ""),     # several lines: separate shift kernels
    ("fp64", 1, 40000, 1, 33, 5, 9, ""),   # too large for one CTA: separate kernels
    ("fp32", 1, 4096, 1, 64, 4, 8, "exact,flat"),
    ("fp32", 3, 512, 2, 10, 2, 4, "exact,flat"),
    ("fp64", 1, 1024, 2, 7, 3, 6, "flat"),
])
def test_event_matches_separate_calls(pamd, precision, d, T, n_sample, n_shift, l_min, l_max,
                                      opts):
    """pamd_event equals n_sample pamd_fragment_mc steps followed by
    pamd_shift_regenerate, bit for bit, for paths, trajectory and counts."""
    from paper_1907_09529_gb300 import integrator
    B, seed, ev = 5, 97531, 3
    prob = pamd.Problem([pamd.System("harmonic", 1, d, T, B),
                         pamd.System("harmonic", 1, d, T // 2, 2)], 1.0, 1.0, 0.3,
                        precision=precision, ho_exact_propagator="exact" in opts,
                        regenerate_flat="flat" in opts)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    a = prob.empty("cuda")
    for q in range(2):
        prob.view(a, q).copy_(torch.randn(prob.view(a, q).shape, generator=g, device="cuda"))
    a2 = a.clone()
    n = sum(s.n_chains * n_shift * s.d * s.N for s in prob.systems)
    acc1 = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    prop1 = torch.zeros_like(acc1)
    acc2, prop2 = acc1.clone(), prop1.clone()
    out1, out2 = prob.empty("cuda"), prob.empty("cuda")
    traj1 = torch.empty(n, dtype=prob.dtype, device="cuda")
    traj2 = torch.empty_like(traj1)
    pamd.fragment_mc(prob, a, l_min, l_max, n_sample, seed=seed, counter=ev * n_sample,
                     n_accepted=acc1, n_proposed=prop1)
    integrator.shift_regenerate(prob, a, out1, n_shift, traj=traj1, seed=seed, counter=ev)
    integrator.event(prob, a2, out2, n_sample, n_shift, l_min, l_max, traj2, acc2, prop2,
                     seed=seed, event=ev)
    torch.cuda.synchronize()
    for q in range(2):
        assert torch.equal(prob.view(a, q), prob.view(a2, q))
        assert torch.equal(prob.view(out1, q), prob.view(out2, q))
    assert torch.equal(traj1, traj2)
    assert torch.equal(acc1, acc2) and torch.equal(prop1, prop2)
    assert int(prop1.sum()) > 0


def test_fallback_kernel_beyond_one_grid_of_chains(pamd):
    """33 elements per slice (11 particles in 3D) take the thread-per-fragment
    kernel, which launches at most 65535 chains at a time: chains on both sides
    of that boundary match the oracle fed the same Philox draws."""
    B, T, N, l_min, l_max, seed, counter = 70000, 16, 11, 2, 3, 4242, 5
    prob = pamd.Problem([pamd.System("harmonic", N, 3, T, B, k=0.8)], 1.0, 1.0, 0.05,
                        precision="fp64")
    buf = prob.empty("cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    prob.view(buf, 0).copy_(torch.randn(prob.view(buf, 0).shape, generator=g, device="cuda",
                                        dtype=torch.float64))
    before = prob.view(buf, 0)
    picks = [0, 1, 65534, 65535, 65536, 69999]
    start = {c: before[c].cpu().numpy().copy() for c in picks}
    acc, prop = pamd.fragment_mc(prob, buf, l_min, l_max, 1, seed=seed, counter=counter)
    torch.cuda.synchronize()
    pot = oracle.harmonic(0.8)
    M = 3 * N
    for c in picks:
        wc = oracle.philox([0, c, counter, 3 << 16], [seed & 0xFFFFFFFF, seed >> 32])
        l = l_min + int(wc[0]) % (l_max - l_min + 1)
        o = int(wc[1]) % (1 << l)
        nf = oracle.n_fragments(T, l, o)
        z = oracle.normals(seed, counter, 4, c, (T + 1) * M).astype(np.float32).astype(np.float64)
        lu = np.array([_philox_log_u(seed, counter, c, f) for f in range(nf)])
        x = start[c].copy()
        _, na, npr = oracle.fragment_step(pot, x, l, o, z.reshape(T + 1, 3, N), lu, 1.0, 1.0, 0.05)
        assert (int(acc[c]), int(prop[c])) == (na, npr), c
        # the kernel's Philox normals are FP32 (Box-Muller in single precision), the
        # oracle's are FP64 rounded to FP32: they agree to about an ulp
        got = prob.view(buf, 0)[c].cpu().numpy()
        assert np.abs(got - x).max() <= 2e-5 * max(1.0, np.abs(x).max()), c
