"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form, an invariant,
finite differences, symbolic differentiation, or published known answers.
None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
import pamd_inputs as inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _lj_tiny(seed, N, T, box, rc, jitter=0.12, step=0.03):
    """A tiny LJ path: jittered simple-cubic start, small random-walk slices."""
    g = inputs.rng(seed)
    m = math.ceil(N ** (1 / 3))
    a = box / m
    sites = np.array([[i, j, k] for i in range(m) for j in range(m) for k in range(m)][:N],
                     dtype=float).T * a + 0.5 * a
    x0 = sites + jitter * g.standard_normal(sites.shape)
    pos = [x0]
    for _ in range(T):
        pos.append(pos[-1] + step * g.standard_normal(x0.shape))
    return np.array(pos)


def _min_pair_gap_to_rc(pos, box, rc):
    """Smallest | |r_ij| - rc | over all slices and pairs (minimum image)."""
    gap = np.inf
    rmin = np.inf
    for x in pos:
        d = x[:, :, None] - x[:, None, :]
        d -= box * np.round(d / box)
        r = np.sqrt((d ** 2).sum(0))
        iu = np.triu_indices(x.shape[1], 1)
        gap = min(gap, np.abs(r[iu] - rc).min())
        rmin = min(rmin, r[iu].min())
    return gap, rmin


# ---------------------------------------------------------------- random numbers
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_are_standard_gaussian():
    """Box-Muller normals: moments and a Kolmogorov-Smirnov test against N(0,1)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    z = oracle.normals(seed=12345, counter=7, stream=1, chain=3, n=200000)
    n = len(z)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # distinct streams / chains / counters give different draws
    assert not np.array_equal(z[:8], oracle.normals(12345, 7, 1, 4, 8))
    assert not np.array_equal(z[:8], oracle.normals(12345, 8, 1, 3, 8))
    assert not np.array_equal(z[:8], oracle.normals(12345, 7, 2, 3, 8))
    # offset access is consistent with a contiguous draw
    np.testing.assert_array_equal(z[101:133], oracle.normals(12345, 7, 1, 3, 32, e0=101))
    u = np.array([oracle.uniform(99, c, 2, 0) for c in range(20000)])
    assert 0.0 < u.min() and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))


# ---------------------------------------------------------------- Lennard-Jones, Eq. (11)
def test_lj_pair_function_closed_forms():
    """u(sigma)=0, u min = -eps at 2^(1/6) sigma, and U(rc) = U'(rc) = 0 (force shift)."""
    p = oracle.lennard_jones(box=20.0, rc=2.5, eps=1.3, sigma=0.9)
    rmin = 2 ** (1 / 6) * 0.9
    # U = u - u(rc) - (r - rc) u'(rc): recover u and u' independently of the oracle's sums
    assert abs(oracle.lj_pair_energy(p, 2.5)) < 1e-15
    assert abs(oracle.lj_pair_dU(p, 2.5)) < 1e-15
    assert oracle.lj_pair_energy(p, 2.5000001) == 0.0
    # derivatives by central differences of the energy
    for r in (0.85, 1.0, 1.3, 2.0, 2.4):
        h = 1e-5
        dU = (oracle.lj_pair_energy(p, r + h) - oracle.lj_pair_energy(p, r - h)) / (2 * h)
        assert abs(dU - oracle.lj_pair_dU(p, r)) < 1e-6 * max(1, abs(dU))
        d2U = (oracle.lj_pair_dU(p, r + h) - oracle.lj_pair_dU(p, r - h)) / (2 * h)
        assert abs(d2U - oracle.lj_pair_d2U(p, r)) < 1e-5 * max(1, abs(d2U))
    # U = u - u(rc) - (r - rc) u'(rc) with u from its closed form; u(sigma) = 0, u(rmin) = -eps
    def u_closed(r):
        q = 0.9 / r
        return 4 * 1.3 * (q ** 12 - q ** 6)
    dudr_rc = 4 * 1.3 * (-12 * 0.9 ** 12 / 2.5 ** 13 + 6 * 0.9 ** 6 / 2.5 ** 7)
    for r in (0.9, rmin, 1.7):
        expect = u_closed(r) - u_closed(2.5) - (r - 2.5) * dudr_rc
        assert abs(oracle.lj_pair_energy(p, r) - expect) < 1e-12 * max(1, abs(expect))
    assert abs(u_closed(0.9)) < 1e-15 and abs(u_closed(rmin) + 1.3) < 1e-12


def test_lj_force_is_minus_gradient_and_newton3():
    p = oracle.lennard_jones(box=4.2, rc=2.0)
    x = _lj_tiny(5, 8, 0, 4.2, 2.0)[0]
    F = oracle.force(p, x)
    # Newton's third law: total force vanishes
    assert np.abs(F.sum(axis=1)).max() < 1e-10 * np.abs(F).max()
    # F = -dV/dx by central differences (Richardson-extrapolated)
    h = 1e-4
    num = np.zeros_like(x)
    for c in range(3):
        for n in range(8):
            def dV(hh):
                xp, xm = x.copy(), x.copy()
                xp[c, n] += hh
                xm[c, n] -= hh
                return (oracle.potential_energy(p, xp) - oracle.potential_energy(p, xm)) / (2 * hh)
            num[c, n] = -(4 * dV(h / 2) - dV(h)) / 3
    assert _rel(F, num) < 1e-8


def test_lj_hvp_properties():
    """H symmetric, translation null space, and Hv = -(F(x+ev) - F(x-ev)) / (2e)."""
    p = oracle.lennard_jones(box=4.2, rc=2.0)
    x = _lj_tiny(6, 8, 0, 4.2, 2.0)[0]
    g = inputs.rng(7)
    u = g.standard_normal(x.shape)
    v = g.standard_normal(x.shape)
    Hu, Hv = oracle.hvp(p, x, u), oracle.hvp(p, x, v)
    assert abs((u * Hv).sum() - (v * Hu).sum()) < 1e-10 * abs((u * Hv).sum())
    assert np.abs(Hv.sum(axis=1)).max() < 1e-10 * np.abs(Hv).max()
    const = np.ones_like(x) * np.array([[0.3], [-1.1], [0.7]])
    assert np.abs(oracle.hvp(p, x, const)).max() < 1e-10
    e = 1e-5
    fd = -(oracle.force(p, x + e * v) - oracle.force(p, x - e * v)) / (2 * e)
    assert _rel(Hv, fd) < 1e-7


def test_harmonic_force_and_hvp():
    p = oracle.harmonic(k=2.5)
    x = inputs.normals(3, (3, 4))
    np.testing.assert_allclose(oracle.force(p, x), -2.5 * x, rtol=0, atol=0)
    np.testing.assert_allclose(oracle.hvp(p, x, x), 2.5 * x, rtol=0, atol=0)
    assert abs(oracle.potential_energy(p, x) - 1.25 * (x ** 2).sum()) < 1e-12


# ---------------------------------------------------------------- invariant (i): EM residuals
@pytest.mark.parametrize("kind", ["harmonic", "lj"])
def test_em_invariant_residuals_equal_scaled_noise(kind):
    """On an Euler-Maruyama path (Eq. (2)) every residual of Eq. (3) equals
    sqrt(2 D dt) xi_t, hence S = sum xi^2 / 2."""
    D, beta, dt = 0.7, 1.3, 0.01
    if kind == "harmonic":
        p = oracle.harmonic(1.4)
        x0 = inputs.normals(11, (3, 2))
    else:
        p = oracle.lennard_jones(box=inputs.box_side(32, 0.85), rc=1.6)
        x0 = inputs.fcc_lattice(32, inputs.box_side(32, 0.85))
        dt = 1e-4
    T = 50
    xi = inputs.normals(12, (T,) + x0.shape)
    pos = oracle.euler(p, x0, xi, D, beta, dt)
    r = oracle.residuals(p, pos, D, beta, dt)
    scale = math.sqrt(2 * D * dt)
    assert np.abs(r - scale * xi).max() < 1e-12 * max(1.0, np.abs(pos).max())
    S = oracle.action_grad(p, pos, D, beta, dt, grad=False)
    assert abs(S - 0.5 * (xi ** 2).sum()) < 1e-10 * S


def test_em_invariant_single_precision_storage_bound():
    """With slices rounded to FP32 the invariant holds up to the rounding of x:
    |r_t - sqrt(2 D dt) xi_t| <= ulp(x)/2 (+ tiny) per component."""
    N = 108
    L = inputs.box_side(N, 0.85)
    p = oracle.lennard_jones(L, 2.5)
    x0 = inputs.fcc_lattice(N, L)
    T, D, beta, dt = 40, 1.0, 1.0, 1e-4
    xi = inputs.normals(13, (T, 3, N))
    pos = oracle.euler(p, x0, xi, D, beta, dt, store_f32=True)
    assert np.array_equal(pos, pos.astype(np.float32).astype(np.float64))
    r = oracle.residuals(p, pos, D, beta, dt)
    err = np.abs(r - math.sqrt(2 * D * dt) * xi)
    bound = 0.5 * np.spacing(np.abs(pos[1:]).astype(np.float32)).astype(np.float64) * 1.01 + 1e-12
    assert (err <= bound).all()


# ---------------------------------------------------------------- invariant (ii): HO closed form
def test_em_harmonic_ar1_statistics_and_ou_limit():
    """EM on the oscillator is an exact AR(1): mean a^t x0, var 2Ddt(1-a^2t)/(1-a^2);
    for small dt it approaches the OU transition density, Eq. (7)."""
    B, T, dt, x0v = 20000, 50, 0.05, 1.0
    p = oracle.harmonic(1.0)
    x0 = np.full((B, 1, 1), x0v)
    xi = inputs.normals(21, (B, T, 1, 1))
    pos = oracle.euler_batch(p, x0, xi, 1.0, 1.0, dt)[:, :, 0, 0]
    a = 1 - dt
    t = np.arange(T + 1)
    mean = a ** t * x0v
    var = 2 * dt * (1 - a ** (2 * t)) / (1 - a ** 2)
    se_m = np.sqrt(np.maximum(var, 1e-30) / B)
    zm = (pos.mean(0)[1:] - mean[1:]) / se_m[1:]
    assert np.abs(zm).max() < 5
    zv = (pos.var(0)[1:] - var[1:]) / (var[1:] * math.sqrt(2 / B))
    assert np.abs(zv).max() < 5
    # OU limit (Eq. (7), k = beta = gamma = 1): small dt, t = 1
    dt2, n = 0.002, 500
    xi2 = inputs.normals(22, (B, n, 1, 1))
    xs = oracle.euler_batch(p, np.full((B, 1, 1), x0v), xi2, 1.0, 1.0, dt2)[:, -1, 0, 0]
    m_ou, v_ou = math.exp(-1.0) * x0v, 1 - math.exp(-2.0)
    assert abs(xs.mean() - m_ou) < 5 * math.sqrt(v_ou / B) + 2 * dt2
    assert abs(xs.var() - v_ou) < 5 * v_ou * math.sqrt(2 / B) + 2 * dt2


@pytest.mark.slow
def test_mala_samples_the_path_distribution():
    """MALA on exp(-S) with x_0 fixed reproduces the AR(1) marginals of the
    oscillator path (exp(-S) is the EM path density up to a constant)."""
    T, dt, x0v, h = 8, 0.1, 1.0, 0.03
    p = oracle.harmonic(1.0)
    a = 1 - dt
    pos = np.zeros((T + 1, 1, 1))
    pos[0] = x0v
    S, g = oracle.action_grad(p, pos, 1.0, 1.0, dt)
    g_rng = inputs.rng(31)
    n_steps, burn = 60000, 2000
    samples = []
    acc = 0
    for it in range(n_steps):
        eta = g_rng.standard_normal(pos.shape)
        lu = math.log(g_rng.random())
        res = oracle.mala_step(p, pos, S, g, eta, lu, h, 1.0, 1.0, dt)
        if res["accepted"]:
            pos, S, g = res["prop"], res["S_prop"], res["grad_prop"]
            acc += 1
        if it >= burn:
            samples.append(pos[[4, 8], 0, 0].copy())
    samples = np.array(samples)
    assert 0.3 < acc / n_steps < 0.98
    for col, t in enumerate((4, 8)):
        m = a ** t * x0v
        v = 2 * dt * (1 - a ** (2 * t)) / (1 - a ** 2)
        xs = samples[:, col]
        nb = 50
        bm = xs[: len(xs) // nb * nb].reshape(nb, -1).mean(1)
        bv = ((xs[: len(xs) // nb * nb] - m) ** 2).reshape(nb, -1).mean(1)
        assert abs(bm.mean() - m) < 5 * bm.std(ddof=1) / math.sqrt(nb)
        assert abs(bv.mean() - v) < 5 * bv.std(ddof=1) / math.sqrt(nb)


def test_mala_log_alpha_is_antisymmetric():
    """log alpha(x->y) = -log alpha(y->x) when each proposal lands on the other path."""
    p = oracle.lennard_jones(box=4.2, rc=2.0)
    D, beta, dt, h = 1.0, 1.0, 1e-3, 1e-4
    x = _lj_tiny(41, 8, 4, 4.2, 2.0)
    y = x.copy()
    y[1:] += 0.01 * inputs.normals(42, y[1:].shape)
    Sx, gx = oracle.action_grad(p, x, D, beta, dt)
    Sy, gy = oracle.action_grad(p, y, D, beta, dt)
    eta_xy = (y - x + h * gx) / math.sqrt(2 * h)
    eta_yx = (x - y + h * gy) / math.sqrt(2 * h)
    r1 = oracle.mala_step(p, x, Sx, gx, eta_xy, 0.0, h, D, beta, dt)
    r2 = oracle.mala_step(p, y, Sy, gy, eta_yx, 0.0, h, D, beta, dt)
    np.testing.assert_allclose(r1["prop"], y, atol=1e-12)
    assert abs(r1["S_prop"] - Sy) < 1e-9 * Sy
    assert abs(r1["log_alpha"] + r2["log_alpha"]) < 1e-7 * (abs(r1["log_alpha"]) + 1)
    # the tail slice never moves
    np.testing.assert_array_equal(r1["prop"][0], x[0])


# ---------------------------------------------------------------- invariant (iii): finite differences
def _fd_grad(p, pos, D, beta, dt, h):
    g = np.zeros_like(pos)
    it = np.nditer(pos, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        def diff(hh):
            a, b = pos.copy(), pos.copy()
            a[idx] += hh
            b[idx] -= hh
            return (oracle.action_grad(p, a, D, beta, dt, grad=False)
                    - oracle.action_grad(p, b, D, beta, dt, grad=False)) / (2 * hh)
        g[idx] = (4 * diff(h / 2) - diff(h)) / 3
    return g


def test_harmonic_gradient_matches_finite_differences():
    """S is quadratic for the oscillator: central differences are exact up to rounding."""
    p = oracle.harmonic(1.7)
    pos = inputs.normals(51, (6, 3, 2))
    D, beta, dt = 0.8, 1.2, 0.05
    S, g = oracle.action_grad(p, pos, D, beta, dt)
    assert _rel(g, _fd_grad(p, pos, D, beta, dt, 1e-3)) < 1e-9


def test_lj_gradient_matches_finite_differences():
    p = oracle.lennard_jones(box=4.2, rc=2.0)
    D, beta, dt = 1.0, 1.0, 2e-3
    pos = _lj_tiny(52, 6, 3, 4.2, 2.0)
    gap, rmin = _min_pair_gap_to_rc(pos, 4.2, 2.0)
    assert gap > 4e-3 and rmin > 0.8
    S, g = oracle.action_grad(p, pos, D, beta, dt)
    fd = _fd_grad(p, pos, D, beta, dt, 1e-3)
    assert _rel(g, fd) < 1e-7


def test_constant_path_closed_form():
    """x_t = c: r_t = a k c, S = T a^2 k^2 |c|^2/(4 D dt), interior grad = (r - (1 - a k) r)/(2Ddt)."""
    k, D, beta, dt, T = 1.5, 0.9, 1.1, 0.02, 7
    p = oracle.harmonic(k)
    c = np.array([[0.3], [-0.8], [1.9]])
    pos = np.repeat(c[None], T + 1, axis=0)
    a = beta * D * dt
    S, g = oracle.action_grad(p, pos, D, beta, dt)
    r = a * k * c
    assert abs(S - T * (r ** 2).sum() / (4 * D * dt)) < 1e-13 * S
    np.testing.assert_allclose(g[0], (-r + a * k * r) / (2 * D * dt), rtol=1e-12)
    np.testing.assert_allclose(g[3], (r - r + a * k * r) / (2 * D * dt), rtol=1e-12)
    np.testing.assert_allclose(g[T], r / (2 * D * dt), rtol=1e-12)


def test_action_invariant_under_translation():
    """A common shift of every slice by a box vector, or any constant, leaves S unchanged (LJ)."""
    L = 4.2
    p = oracle.lennard_jones(box=L, rc=2.0)
    pos = _lj_tiny(61, 8, 4, L, 2.0)
    S = oracle.action_grad(p, pos, 1.0, 1.0, 1e-3, grad=False)
    shift = np.array([[L], [-2 * L], [0.0]])
    assert abs(oracle.action_grad(p, pos + shift, 1.0, 1.0, 1e-3, grad=False) - S) < 1e-10 * S
    assert abs(oracle.action_grad(p, pos + 0.377, 1.0, 1.0, 1e-3, grad=False) - S) < 1e-10 * S
    # moving one particle by a box vector at every slice changes nothing either
    pos2 = pos.copy()
    pos2[:, 1, 3] += L
    assert abs(oracle.action_grad(p, pos2, 1.0, 1.0, 1e-3, grad=False) - S) < 1e-10 * S


def test_threaded_oracle_is_bit_identical():
    L = inputs.box_side(64, 0.85)
    p = oracle.lennard_jones(L, min(2.5, L / 2))
    pos = _lj_tiny(71, 64, 12, L, 2.0, step=0.01)
    S1, g1 = oracle.action_grad(p, pos, 1.0, 1.0, 1e-4, nthreads=1)
    S4, g4 = oracle.action_grad(p, pos, 1.0, 1.0, 1e-4, nthreads=4)
    assert S1 == S4
    assert np.array_equal(g1, g4)
    ts = [0, 3, 12]
    np.testing.assert_array_equal(oracle.grad_slices(p, pos, 1.0, 1.0, 1e-4, ts), g1[ts])
    sa = oracle.step_actions(p, pos, 1.0, 1.0, 1e-4, list(range(12)))
    assert abs(sa.sum() - S1) < 1e-12 * S1


# ---------------------------------------------------------------- brute force, written out symbolically
def test_two_particle_path_symbolic():
    """N = 2 particles, T = 2 steps, open boundaries: S and dS/dx from sympy
    differentiation of Eqs. (3), (4) and (11) written out from scratch."""
    sp = pytest.importorskip("sympy")
    eps, sig, rc = 1.0, 1.0, 2.5
    D, beta, dt = 1.0, 1.0, 0.01
    a = beta * D * dt
    X = [[[sp.Symbol(f"x{t}{c}{n}") for n in range(2)] for c in range(3)] for t in range(3)]
    rs = sp.Symbol("r", positive=True)
    u = 4 * eps * ((sig / rs) ** 12 - (sig / rs) ** 6)
    du = sp.diff(u, rs)
    U = u - u.subs(rs, rc) - (rs - rc) * du.subs(rs, rc)

    def V(x):
        r = sp.sqrt(sum((x[c][0] - x[c][1]) ** 2 for c in range(3)))
        return U.subs(rs, r)

    S = 0
    for t in range(2):
        v = V(X[t])
        for c in range(3):
            for n in range(2):
                F = -sp.diff(v, X[t][c][n])
                S += (X[t + 1][c][n] - X[t][c][n] - a * F) ** 2
    S = S / (4 * D * dt)
    flat = [X[t][c][n] for t in range(3) for c in range(3) for n in range(2)]
    pos = np.array([[[0.1, 1.25], [0.2, 0.05], [-0.1, 0.35]],
                    [[0.12, 1.22], [0.18, 0.08], [-0.07, 0.33]],
                    [[0.09, 1.26], [0.22, 0.03], [-0.12, 0.36]]])
    vals = dict(zip(flat, pos.reshape(-1).tolist()))
    S_ref = float(S.subs(vals).evalf(30))
    g_ref = np.array([float(sp.diff(S, s).subs(vals).evalf(30)) for s in flat]).reshape(pos.shape)
    p = oracle.lennard_jones(box=0.0, rc=rc)
    S_or, g_or = oracle.action_grad(p, pos, D, beta, dt)
    assert abs(S_or - S_ref) < 1e-12 * abs(S_ref)
    assert _rel(g_or, g_ref) < 1e-12


# ---------------------------------------------------------------- index rule
def test_pair_count_f32_agrees_with_exact_distances():
    """The single-precision cutoff count equals the exact count whenever no pair
    distance lies within 1e-4 of the cutoff."""
    for N, seed in ((108, 81), (500, 82), (250, 83)):
        L = inputs.box_side(N, 0.85)
        rc = min(2.5, L / 2)
        x = inputs.fcc_lattice(N, L) + 0.15 * inputs.normals(seed, (3, N))
        x += L * inputs.rng(seed + 1).integers(-2, 3, size=(3, N))  # unwrapped images
        x32 = x.astype(np.float32)
        xd = x32.astype(np.float64)
        d = xd[:, :, None] - xd[:, None, :]
        d -= L * np.round(d / L)
        r = np.sqrt((d ** 2).sum(0))
        np.fill_diagonal(r, np.inf)
        if np.abs(r - rc).min() < 1e-4:
            continue
        assert oracle.pair_count_f32(L, rc, x32) == int((r <= rc).sum())


# ---------------------------------------------------------------- multilevel sliding-and-sampling MC
@pytest.mark.slow
@pytest.mark.parametrize("levels,exact,dt", [((1, 1), False, 0.1), ((2, 3), False, 0.1),
                                             ((2, 3), True, 0.4)])
def test_fragment_mc_samples_the_path_distribution(levels, exact, dt):
    """Repeated multilevel fragment MC steps (free-particle trials) leave the
    oscillator path distribution exp(-S) with x_0 fixed invariant: sampled x_4
    and x_8 match the exact AR(1) marginals of the chain S describes -- the
    Euler-Maruyama chain (coefficient 1 - dt) for Eq. (3), the exact
    Ornstein-Uhlenbeck transition (coefficient e^{-dt}, variance 1 - e^{-2t}
    at time t) for the oscillator's exact propagator."""
    T, x0v = 8, 1.0
    p = oracle.harmonic(1.0)
    a = math.exp(-dt) if exact else 1 - dt
    pos = np.zeros((T + 1, 1, 1))
    pos[0] = x0v
    g = inputs.rng(91 + levels[0])
    n_steps, burn = 30000, 500
    samples = []
    acc = prop = 0
    for it in range(n_steps):
        l = int(g.integers(levels[0], levels[1] + 1))
        o = int(g.integers(0, 1 << l))
        z = g.standard_normal(pos.shape)
        nf = oracle.n_fragments(T, l, o)
        lu = np.log(g.random(nf))
        nf2, na, npr = oracle.fragment_step(p, pos, l, o, z, lu, 1.0, 1.0, dt, exact_ho=exact)
        assert nf2 == nf
        acc += na
        prop += npr
        if it >= burn:
            samples.append(pos[[4, 8], 0, 0].copy())
    assert np.all(pos[0] == x0v)
    assert 0.2 < acc / prop < 1.0
    samples = np.array(samples)
    for col, t in enumerate((4, 8)):
        m = a ** t * x0v
        step_var = (1 - a * a) if exact else 2 * dt
        v = step_var * (1 - a ** (2 * t)) / (1 - a ** 2)
        xs = samples[:, col]
        nb = 50
        k = len(xs) // nb * nb
        bm = xs[:k].reshape(nb, -1).mean(1)
        bv = ((xs[:k] - m) ** 2).reshape(nb, -1).mean(1)
        assert abs(bm.mean() - m) < 5 * bm.std(ddof=1) / math.sqrt(nb)
        assert abs(bv.mean() - v) < 5 * bv.std(ddof=1) / math.sqrt(nb)


def test_fragment_layout_and_fixed_endpoints():
    """Endpoints shared by fragments (and the tail) never move; the nose does."""
    T = 16
    p = oracle.harmonic(1.0)
    pos = inputs.normals(5, (T + 1, 1, 1))
    before = pos.copy()
    z = inputs.normals(6, pos.shape)
    lu = np.full(oracle.n_fragments(T, 2, 1), -np.inf)  # accept everything
    nf, na, npr = oracle.fragment_step(p, pos, 2, 1, z, lu, 1.0, 1.0, 0.1)
    assert nf == 5  # [0,1] [1,5] [5,9] [9,13] [13,16]
    for e in (0, 1, 5, 9, 13):
        assert pos[e, 0, 0] == before[e, 0, 0]
    assert pos[16, 0, 0] != before[16, 0, 0]
    assert na == npr == 4  # [0,1] has no interior point


def test_fragment_trials_are_free_particle_bridges_and_walks():
    """With every fragment accepted the step returns its trial path.  Over many
    normals its interior points follow the free-particle path distribution with
    the fragment ends fixed (Sec. III): a Brownian bridge of covariance
    2 D dt (t - a)(b - s)/(b - a) (t <= s) about the straight line between the
    ends, and for the nose a random walk of covariance 2 D dt (min(t, s) - a)."""
    T, D, dt, level, offset = 16, 0.7, 0.3, 3, 5   # fragments [0,5] [5,13] [13,16]
    p = oracle.harmonic(1.0)
    base = inputs.normals(41, (T + 1, 1, 1))
    g = inputs.rng(42)
    n = 40000
    lu = np.full(oracle.n_fragments(T, level, offset), -np.inf)
    out = np.empty((n, T + 1))
    for i in range(n):
        pos = base.copy()
        nf, na, npr = oracle.fragment_step(p, pos, level, offset, g.standard_normal(pos.shape),
                                           lu, D, 1.0, dt)
        out[i] = pos[:, 0, 0]
    assert nf == 3 and na == npr == 3
    for e in (0, 5, 13):
        assert np.all(out[:, e] == base[e, 0, 0])
    x = base[:, 0, 0]
    q = 2 * D * dt
    for a, b, nose in ((0, 5, False), (5, 13, False), (13, 16, True)):
        ts = np.arange(a + 1, b + 1 if nose else b)
        ys = out[:, ts]
        mean = np.full(len(ts), x[a]) if nose else x[a] + (ts - a) / (b - a) * (x[b] - x[a])
        tt, ss = np.meshgrid(ts, ts, indexing="ij")
        lo, hi = np.minimum(tt, ss), np.maximum(tt, ss)
        cov = q * (lo - a) if nose else q * (lo - a) * (b - hi) / (b - a)
        emp = np.cov(ys, rowvar=False)
        sd = np.sqrt(np.diag(cov))
        assert np.all(np.abs(ys.mean(0) - mean) < 5 * sd / math.sqrt(n))
        assert np.all(np.abs(emp - cov) < 6 * np.outer(sd, sd) * math.sqrt(2.0 / n) + 1e-12)


def test_shift_regenerate_grows_free_particle_walks():
    """Shift and regeneration (Fig. 2B): the kept slices move n_shift steps
    toward the tail, the trajectory gets x_1..x_{n_shift}, and the regrown nose
    is a free-particle random walk from the old nose: over many draws its mean
    is x_T and its covariance 2 D dt min(i, j) (the sampler's trial
    distribution, Sec. III)."""
    T, n_shift, D, dt = 12, 5, 0.6, 0.25
    pos = inputs.normals(61, (T + 1, 1, 1))
    g = inputs.rng(62)
    n = 40000
    nose = np.empty((n, n_shift))
    for i in range(n):
        out, traj = oracle.shift_regenerate(pos, n_shift, g.standard_normal((n_shift, 1, 1)), D, dt)
        if i == 0:
            assert np.array_equal(out[:T - n_shift + 1], pos[n_shift:])
            assert np.array_equal(traj, pos[1:n_shift + 1])
        nose[i] = out[T - n_shift + 1:, 0, 0]
    ks = np.arange(1, n_shift + 1)
    cov = 2 * D * dt * np.minimum.outer(ks, ks)
    sd = np.sqrt(np.diag(cov))
    assert np.all(np.abs(nose.mean(0) - pos[T, 0, 0]) < 5 * sd / math.sqrt(n))
    assert np.all(np.abs(np.cov(nose, rowvar=False) - cov) < 6 * np.outer(sd, sd) * math.sqrt(2.0 / n))


def _hs_path(T, box, d_pair, t_pair, rng_seed=3):
    """Four particles far apart in a box of side `box`, except that particles 0
    and 1 sit exactly d_pair apart along x at slice t_pair (elsewhere 2.0 apart);
    particle 3 sits across the periodic boundary from particle 2 (min image 1.6)."""
    g = inputs.rng(rng_seed)
    pos = np.zeros((T + 1, 3, 4))
    for t in range(T + 1):
        c = np.array([4.0, 4.0, 4.0]) + 1e-3 * g.standard_normal(3)
        sep = d_pair if t == t_pair else 2.0
        pos[t, :, 0] = c
        pos[t, :, 1] = c + np.array([sep, 0.0, 0.0])
        pos[t, :, 2] = [0.3, 8.5, 8.5]
        pos[t, :, 3] = [box - 1.3, 8.5, 8.5]   # 1.6 from particle 2 through the face
    return pos


def test_hard_sphere_bias_closed_forms():
    """The hard-sphere path bias (Sec. IV.B): infinite exactly when a pair within
    the cutoff is at r <= sigma_HS(t) at some slice, the plain LJ action (bit for
    bit) otherwise; minimum image; sigma_HS above rc acts as rc."""
    T, box, rc = 6, 12.0, 2.5
    pot = oracle.lennard_jones(box, rc)
    D, beta, dt = 1.0, 1.0, 1e-3
    pos = _hs_path(T, box, 0.95, 4)
    S_lj, g_lj = oracle.action_grad(pot, pos, D, beta, dt)
    zero = np.zeros(T + 1)
    assert oracle.hs_first_overlap(pot, pos, zero) == -1
    S, g = oracle.action_grad_hs(pot, pos, zero, D, beta, dt)
    assert S == S_lj and np.array_equal(g, g_lj)
    # the pair 0.95 apart at slice 4: caught by sigma 0.96 at that slice only
    sig = zero.copy()
    sig[4] = 0.96
    assert oracle.hs_first_overlap(pot, pos, sig) == 4
    S, g = oracle.action_grad_hs(pot, pos, sig, D, beta, dt)
    assert S == math.inf and np.array_equal(g, g_lj)
    sig[4] = 0.94
    assert oracle.hs_first_overlap(pot, pos, sig) == -1
    assert oracle.action_grad_hs(pot, pos, sig, D, beta, dt)[0] == S_lj
    # sigma 1.9 everywhere: the 2.0 pairs pass, the 1.6 pair through the face overlaps
    sig = np.full(T + 1, 1.9)
    sig[4] = 0.0
    assert oracle.hs_first_overlap(pot, pos, sig) == 0
    # sigma 1.9 only at the nose: still caught there (every slice counts, x_T too)
    sig = zero.copy()
    sig[T] = 1.9
    assert oracle.hs_first_overlap(pot, pos, sig) == T
    # sigma above rc acts as rc: the 2.0 pairs (inside rc) overlap, nothing beyond rc does
    far = pos.copy()
    far[:, :, 3] = [6.0, 1.0, 1.0]                 # the face pair moved out of range
    sig = zero.copy()
    sig[2] = 3.0
    assert oracle.hs_first_overlap(pot, far, sig) == 2
    far[:, 0, 1] = far[:, 0, 0] + 2.6              # pair 0-1 beyond rc = 2.5
    assert oracle.hs_first_overlap(pot, far, sig) == -1


def test_hard_sphere_overlap_f32_agrees_away_from_the_threshold():
    """The single-precision mirror of the overlap decision equals the exact one
    whenever no pair distance is within 1e-4 of sigma."""
    box, rc = 6.0, 2.5
    pot = oracle.lennard_jones(box, rc)
    g = inputs.rng(11)
    checked = 0
    for trial in range(40):
        x = g.uniform(0, box, size=(3, 16))
        dmin = np.inf
        for i in range(16):
            for j in range(i + 1, 16):
                dv = x[:, i] - x[:, j]
                dv -= box * np.round(dv / box)
                dmin = min(dmin, float(np.linalg.norm(dv)))
        for sigma in (0.5, 0.8, 1.0, 1.2):
            if abs(dmin - sigma) < 1e-4:
                continue
            exact = oracle.hs_first_overlap(pot, x[None], [sigma]) == 0
            assert oracle.hs_overlap_f32(box, rc, sigma, x.astype(np.float32)) == exact
            checked += 1
    assert checked > 100
