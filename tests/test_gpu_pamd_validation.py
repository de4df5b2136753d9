"""The oscillator's exact-propagator option of the multilevel sampler and the
PAMD loop (Sec. IV.A, Table of oscillator parameters), on the GPU.

The sampler with PAMD_FLAG_HO_EXACT_PROPAGATOR samples the path measure of the
exact transition density (the oscillator marginal of Sec. II); the PAMD loop
run at the paper's three oscillator parameter sets (dt = 0.4) then reproduces
the exact dynamics: the error measures of Sec. IV.A, E_eq (equilibrium density)
and E_dyn (decay constant of the autocovariance fitted on t in [0, 4]), stay
below the paper's 3 % accuracy requirement."""
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
    ("fp64", 256, 1, 4, 5, 0.4),     # one-line kernel
    ("fp32", 4096, 1, 4, 8, 0.4),
    ("fp64", 512, 3, 2, 4, 0.2),     # several lines per slice
    ("fp64", 40000, 1, 5, 9, 0.4),   # thread-per-fragment fallback
])
def test_exact_propagator_step_matches_oracle(pamd, precision, T, d, l_min, l_max, dt):
    B, D, beta, k = 4, 1.0, 1.0, 1.3
    rng = inputs.rng(700 + T + d)
    prob = pamd.Problem([pamd.System("harmonic", 1, d, T, B, k=k)], D, beta, dt,
                        precision=precision, ho_exact_propagator=True)
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
    pot = oracle.harmonic(k)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for b in range(B):
        x = paths[b].copy()
        nf = oracle.n_fragments(T, int(levels[b]), int(offsets[b]))
        _, na, npr = oracle.fragment_step(pot, x, int(levels[b]), int(offsets[b]), noise[b],
                                          log_u[b, :nf], D, beta, dt, exact_ho=True)
        assert int(acc[b]) == na and int(prop[b]) == npr, (b, int(acc[b]), na)
        assert np.abs(got[b] - x).max() <= tol * max(1.0, np.abs(x).max()), b


def test_eq3_entry_points_refuse_the_exact_propagator(pamd):
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, 64, 2)], 1.0, 1.0, 0.4,
                        ho_exact_propagator=True)
    buf = prob.empty("cuda")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.action(prob, buf)
    assert ei.value.status == -2
    with pytest.raises(pamd.PamdError) as ei:
        pamd.action_grad(prob, buf)
    assert ei.value.status == -2
    with pytest.raises(pamd.PamdError) as ei:
        pamd.euler_reference(prob, buf)
    assert ei.value.status == -2


def _error_measures(traj, dt, lag_max_t=4.0):
    """E_eq: L2 distance between the sampled and the exact (standard normal)
    position densities.  E_dyn: |kappa - kappa_s| with kappa_s from a linear fit
    of log C(t) on t in [0, lag_max_t] (Sec. IV.A).  traj: [points, series]."""
    x = traj.astype(np.float64)
    edges = np.linspace(-5.0, 5.0, 101)
    w = edges[1] - edges[0]
    h, _ = np.histogram(x.ravel(), bins=edges)
    ps = h / (x.size * w)
    cdf = np.array([0.5 * (1 + math.erf(e / math.sqrt(2))) for e in edges])
    p = np.diff(cdf) / w
    e_eq = math.sqrt(((ps - p) ** 2).sum() * w)
    lags = np.arange(0, int(round(lag_max_t / dt)) + 1)
    n = x.shape[0]
    c = np.array([(x[: n - L] * x[L:]).mean() for L in lags])
    slope = np.polyfit(lags * dt, np.log(c), 1)[0]
    return e_eq, abs(1.0 + slope), c[0]


@pytest.mark.parametrize("name,n_path,n_sample,n_shift,l_min,l_max,chains,events,flat", [
    ("Simulation 1", 16, 2, 2, 3, 3, 8192, 2400, False),
    ("Simulation 2", 256, 1, 8, 4, 5, 8192, 640, False),
    ("Simulation 3", 4096, 1, 64, 4, 8, 4096, 160, True),
])
def test_pamd_reproduces_oscillator_dynamics(pamd, name, n_path, n_sample, n_shift, l_min,
                                              l_max, chains, events, flat):
    """The paper's oscillator runs (dt = 0.4, k = beta = gamma = 1) through the
    PAMD loop with the exact propagator: E_eq and E_dyn below 3 %.  Simulations 1
    and 2 regrow the nose from the trial distribution (Sec. III); Simulation 3,
    with one MC step per 64-step shift, needs the straight-line regrowth of
    Fig. 2B (with free-particle regrowth its E_dyn is about 10 %)."""
    from paper_1907_09529_gb300.integrator import PamdIntegrator
    dt = 0.4
    prob = pamd.Problem([pamd.System("harmonic", 1, 1, n_path, chains, k=1.0)], 1.0, 1.0, dt,
                        precision="fp32", ho_exact_propagator=True, regenerate_flat=flat)
    buf = prob.empty("cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(2019)
    prob.view(buf, 0).copy_(torch.randn(prob.view(buf, 0).shape, generator=g, device="cuda"))
    integ = PamdIntegrator(prob, n_shift=n_shift, n_sample=n_sample, l_min=l_min, l_max=l_max,
                           seed=1907)
    burn = max(2 * n_path // n_shift, 50)  # the start path has left the sampled window
    integ.run(buf, burn)
    traj = integ.run(buf, events)          # [events, chains * n_shift]
    torch.cuda.synchronize()
    x = traj.view(events, chains, n_shift).permute(0, 2, 1).reshape(events * n_shift, chains)
    e_eq, e_dyn, x2 = _error_measures(x.cpu().numpy(), dt)
    print(f"{name}: E_eq = {100 * e_eq:.2f} %, E_dyn = {100 * e_dyn:.2f} %, <x^2> = {x2:.4f}, "
          f"acceptance {float(integ.n_accepted.sum()) / float(integ.n_proposed.sum()):.3f}")
    assert e_eq < 0.03 and e_dyn < 0.03
