/*
 * pamd_oracle.c -- plain, slow CPU reference for the discretised
 * Brownian-dynamics path action of path-accelerated molecular dynamics
 * (Rosa-Raices, Zhang & Miller, arXiv:1907.09529).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * file.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA library: every formula below is written out again from
 * the paper.
 *
 * Arithmetic: IEEE double, round to nearest, no fast-math and no FMA
 * contraction (built with -ffp-contract=off).  The only single-precision
 * function is or_pair_count_f32, which mirrors the GPU's cutoff decision
 * (an integer outcome decided in the kernel's precision).
 *
 * Layout of one chain's path: pos[t][c][n], t = 0..T (T+1 slices,
 * T steps), c = 0..d-1 (Cartesian component), n = 0..N-1 (particle).
 * A slice holds M = d*N doubles.
 *
 * Notation (paper Sec. II.A): drift coefficient gamma^-1 = beta*D
 * (Einstein relation under Eq. (1)); F = -grad V; a = beta*D*dt.
 *   residual   r_t = x_{t+1} - x_t - a F(x_t)                 (Eq. (3))
 *   action     S   = sum_{t=0}^{T-1} |r_t|^2 / (4 D dt)        (Eqs. (3)-(4))
 *   gradient   dS/dx_t = [r_{t-1} - r_t + a H(x_t) r_t]/(2 D dt)
 *              with r_{-1} = r_T = 0, H = Hessian of V.
 * The normalisation of K in Eq. (3) is dropped: it does not depend on X.
 *
 * Parity status: every function here is pinned by tests that do not use
 * this file's own formulas (closed forms, invariants, finite differences,
 * symbolic differentiation, published Philox known-answer vectors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Potential parameters.  kind 0: harmonic V = k/2 |x|^2 per coordinate
 * (the paper's oscillator, Sec. IV.A, taken isotropic in d dimensions).
 * kind 1: cut-and-force-shifted Lennard-Jones, Eq. (11), in a periodic
 * cubic box of side `box` (box <= 0: no periodic images). */
typedef struct {
    int kind;
    double k;
    double eps, sigma, rc, box;
} or_potential;

enum { OR_HARMONIC = 0, OR_LJ = 1 };

/* ---------------------------------------------------------------- */
/* Lennard-Jones pair functions, Eq. (11): u(r) = 4 eps [(s/r)^12 - (s/r)^6] */

static double lj_u(const or_potential* p, double r)
{
    double q = p->sigma / r;
    double q6 = pow(q, 6.0);
    return 4.0 * p->eps * (q6 * q6 - q6);
}

/* u'(r) = 4 eps [-12 s^12 / r^13 + 6 s^6 / r^7] */
static double lj_du(const or_potential* p, double r)
{
    double q = p->sigma / r;
    double q6 = pow(q, 6.0);
    return 4.0 * p->eps * (-12.0 * q6 * q6 + 6.0 * q6) / r;
}

/* u''(r) = 4 eps [156 s^12 / r^14 - 42 s^6 / r^8] */
static double lj_d2u(const or_potential* p, double r)
{
    double q = p->sigma / r;
    double q6 = pow(q, 6.0);
    return 4.0 * p->eps * (156.0 * q6 * q6 - 42.0 * q6) / (r * r);
}

/* Eq. (11): U(r) = u(r) - u(rc) - (r - rc) u'(rc) for r <= rc, else 0. */
double or_lj_pair_energy(const or_potential* p, double r)
{
    if (r > p->rc) return 0.0;
    return lj_u(p, r) - lj_u(p, p->rc) - (r - p->rc) * lj_du(p, p->rc);
}

/* U'(r) = u'(r) - u'(rc) inside the cutoff. */
double or_lj_pair_dU(const or_potential* p, double r)
{
    if (r > p->rc) return 0.0;
    return lj_du(p, r) - lj_du(p, p->rc);
}

/* U''(r) = u''(r) inside the cutoff. */
double or_lj_pair_d2U(const or_potential* p, double r)
{
    if (r > p->rc) return 0.0;
    return lj_d2u(p, r);
}

/* Minimum-image separation component (periodic cubic box). */
static double min_image(const or_potential* p, double dx)
{
    if (p->box > 0.0) dx -= p->box * nearbyint(dx / p->box);
    return dx;
}

/* ---------------------------------------------------------------- */
/* Potential energy V(x) of one slice x[c][n]. */
double or_potential_energy(const or_potential* p, int N, int d, const double* x)
{
    double V = 0.0;
    if (p->kind == OR_HARMONIC) {
        for (int m = 0; m < d * N; ++m) V += 0.5 * p->k * x[m] * x[m];
        return V;
    }
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = 0.0;
            for (int c = 0; c < d; ++c) {
                double dx = min_image(p, x[c * N + i] - x[c * N + j]);
                r2 += dx * dx;
            }
            if (r2 <= p->rc * p->rc) V += or_lj_pair_energy(p, sqrt(r2));
        }
    return V;
}

/* F = -grad V at one slice.  LJ: all pairs, minimum image, r <= rc included. */
void or_force(const or_potential* p, int N, int d, const double* x, double* F)
{
    int M = d * N;
    if (p->kind == OR_HARMONIC) {
        for (int m = 0; m < M; ++m) F[m] = -p->k * x[m];
        return;
    }
    for (int m = 0; m < M; ++m) F[m] = 0.0;
    double rij[8];
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = 0.0;
            for (int c = 0; c < d; ++c) {
                rij[c] = min_image(p, x[c * N + i] - x[c * N + j]);
                r2 += rij[c] * rij[c];
            }
            if (r2 > p->rc * p->rc) continue;
            double r = sqrt(r2);
            /* F_i = -U'(r) r_ij / r, F_j = -F_i */
            double s = -or_lj_pair_dU(p, r) / r;
            for (int c = 0; c < d; ++c) {
                F[c * N + i] += s * rij[c];
                F[c * N + j] -= s * rij[c];
            }
        }
}

/* Hessian-vector product H(x) v of V at one slice.
 * LJ pair block: K_ij = U''(r) rhat rhat^T + (U'(r)/r)(I - rhat rhat^T),
 * (Hv)_i = sum_j K_ij (v_i - v_j). */
void or_hvp(const or_potential* p, int N, int d, const double* x, const double* v, double* Hv)
{
    int M = d * N;
    if (p->kind == OR_HARMONIC) {
        for (int m = 0; m < M; ++m) Hv[m] = p->k * v[m];
        return;
    }
    for (int m = 0; m < M; ++m) Hv[m] = 0.0;
    double rij[8], rhat[8], vij[8];
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = 0.0;
            for (int c = 0; c < d; ++c) {
                rij[c] = min_image(p, x[c * N + i] - x[c * N + j]);
                r2 += rij[c] * rij[c];
            }
            if (r2 > p->rc * p->rc) continue;
            double r = sqrt(r2);
            double proj = 0.0;
            for (int c = 0; c < d; ++c) {
                rhat[c] = rij[c] / r;
                vij[c] = v[c * N + i] - v[c * N + j];
                proj += rhat[c] * vij[c];
            }
            double d2U = or_lj_pair_d2U(p, r);
            double dUr = or_lj_pair_dU(p, r) / r;
            for (int c = 0; c < d; ++c) {
                double w = d2U * proj * rhat[c] + dUr * (vij[c] - proj * rhat[c]);
                Hv[c * N + i] += w;
                Hv[c * N + j] -= w;
            }
        }
}

/* ---------------------------------------------------------------- */
/* Residual of one step, Eq. (3): r = x1 - x0 - a F(x0), a = beta D dt. */
static void step_residual(const or_potential* p, int N, int d, double a,
                          const double* x0, const double* x1, double* r, double* F)
{
    int M = d * N;
    or_force(p, N, d, x0, F);
    for (int m = 0; m < M; ++m) r[m] = x1[m] - x0[m] - a * F[m];
}

/* All residuals r[t][m], t = 0..T-1. */
int or_residuals(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                 const double* pos, double* r)
{
    int M = d * N;
    double a = beta * D * dt;
    double* F = (double*)malloc(sizeof(double) * (size_t)M);
    if (!F) return -1;
    for (int t = 0; t < T; ++t)
        step_residual(p, N, d, a, pos + (size_t)t * M, pos + (size_t)(t + 1) * M,
                      r + (size_t)t * M, F);
    free(F);
    return 0;
}

/* Action S (Eq. (4) without normalisation) and, if grad != NULL, its
 * gradient with respect to every slice x_0..x_T (grad[t][m]).
 * The sum is taken in a fixed order (slice, then component, then particle)
 * so that the result does not depend on nthreads. */
int or_action_grad(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                   const double* pos, double* S, double* grad, int nthreads)
{
    int M = d * N;
    double a = beta * D * dt;
    double* r = (double*)malloc(sizeof(double) * (size_t)T * M);
    double* sq = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    if (!r || !sq) { free(r); free(sq); return -1; }
    int fail = 0;
    if (nthreads < 1) nthreads = 1;

#pragma omp parallel num_threads(nthreads)
    {
        double* F = (double*)malloc(sizeof(double) * (size_t)M);
        double* Hr = (double*)malloc(sizeof(double) * (size_t)M);
        if (!F || !Hr) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (int t = 0; t < T; ++t) {
                double* rt = r + (size_t)t * M;
                step_residual(p, N, d, a, pos + (size_t)t * M, pos + (size_t)(t + 1) * M, rt, F);
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += rt[m] * rt[m];
                sq[t] = s;
            }
            if (grad) {
                double g0 = 1.0 / (2.0 * D * dt);
#pragma omp for schedule(static)
                for (int t = 0; t <= T; ++t) {
                    double* g = grad + (size_t)t * M;
                    for (int m = 0; m < M; ++m) g[m] = 0.0;
                    if (t >= 1) {
                        const double* rp = r + (size_t)(t - 1) * M;
                        for (int m = 0; m < M; ++m) g[m] += rp[m];
                    }
                    if (t <= T - 1) {
                        const double* rt = r + (size_t)t * M;
                        or_hvp(p, N, d, pos + (size_t)t * M, rt, Hr);
                        for (int m = 0; m < M; ++m) g[m] += -rt[m] + a * Hr[m];
                    }
                    for (int m = 0; m < M; ++m) g[m] *= g0;
                }
            }
        }
        free(F);
        free(Hr);
    }
    if (!fail) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += sq[t];
        *S = s / (4.0 * D * dt);
    }
    free(r);
    free(sq);
    return fail ? -1 : 0;
}

/* Per-slice partial actions s[t] = |r_t|^2 / (4 D dt) for a list of steps. */
int or_step_actions(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                    const double* pos, int nt, const int* t_list, double* s_out)
{
    int M = d * N;
    double a = beta * D * dt;
    double* F = (double*)malloc(sizeof(double) * (size_t)M);
    double* r = (double*)malloc(sizeof(double) * (size_t)M);
    if (!F || !r) { free(F); free(r); return -1; }
    for (int q = 0; q < nt; ++q) {
        int t = t_list[q];
        if (t < 0 || t >= T) { s_out[q] = NAN; continue; }
        step_residual(p, N, d, a, pos + (size_t)t * M, pos + (size_t)(t + 1) * M, r, F);
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += r[m] * r[m];
        s_out[q] = s / (4.0 * D * dt);
    }
    free(F);
    free(r);
    return 0;
}

/* Gradient at a list of slices only (each one from x_{t-1}, x_t, x_{t+1}),
 * for spot checks of paths too long for the full oracle. g_out[q][m]. */
int or_grad_slices(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                   const double* pos, int nt, const int* t_list, double* g_out)
{
    int M = d * N;
    double a = beta * D * dt;
    double g0 = 1.0 / (2.0 * D * dt);
    double* F = (double*)malloc(sizeof(double) * (size_t)M);
    double* r = (double*)malloc(sizeof(double) * (size_t)M);
    double* Hr = (double*)malloc(sizeof(double) * (size_t)M);
    if (!F || !r || !Hr) { free(F); free(r); free(Hr); return -1; }
    for (int q = 0; q < nt; ++q) {
        int t = t_list[q];
        double* g = g_out + (size_t)q * M;
        for (int m = 0; m < M; ++m) g[m] = 0.0;
        if (t < 0 || t > T) continue;
        if (t >= 1) {
            step_residual(p, N, d, a, pos + (size_t)(t - 1) * M, pos + (size_t)t * M, r, F);
            for (int m = 0; m < M; ++m) g[m] += r[m];
        }
        if (t <= T - 1) {
            step_residual(p, N, d, a, pos + (size_t)t * M, pos + (size_t)(t + 1) * M, r, F);
            or_hvp(p, N, d, pos + (size_t)t * M, r, Hr);
            for (int m = 0; m < M; ++m) g[m] += -r[m] + a * Hr[m];
        }
        for (int m = 0; m < M; ++m) g[m] *= g0;
    }
    free(F);
    free(r);
    free(Hr);
    return 0;
}

/* ---------------------------------------------------------------- */
/* Forward Euler-Maruyama, Eq. (2), sequential in time:
 *   x_{t+1} = x_t + a F(x_t) + sqrt(2 D dt) xi_t.
 * pos[0] holds x_0 on entry; xi[t][m] are standard normals.
 * store_f32 != 0 rounds every new slice to single precision before it is
 * used, so that the stored single-precision path is its own state. */
int or_euler(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
             const double* xi, int store_f32, double* pos)
{
    int M = d * N;
    double a = beta * D * dt;
    double sig = sqrt(2.0 * D * dt);
    double* F = (double*)malloc(sizeof(double) * (size_t)M);
    if (!F) return -1;
    if (store_f32)
        for (int m = 0; m < M; ++m) pos[m] = (double)(float)pos[m];
    for (int t = 0; t < T; ++t) {
        const double* x = pos + (size_t)t * M;
        double* y = pos + (size_t)(t + 1) * M;
        const double* z = xi + (size_t)t * M;
        or_force(p, N, d, x, F);
        for (int m = 0; m < M; ++m) {
            double v = x[m] + a * F[m] + sig * z[m];
            y[m] = store_f32 ? (double)(float)v : v;
        }
    }
    free(F);
    return 0;
}

/* Independent chains of or_euler in parallel (one chain per thread). */
int or_euler_batch(const or_potential* p, int B, int N, int d, int T, double D, double beta,
                   double dt, const double* xi, int store_f32, double* pos, int nthreads)
{
    size_t per_pos = (size_t)(T + 1) * d * N, per_xi = (size_t)T * d * N;
    int fail = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
    for (int b = 0; b < B; ++b)
        if (or_euler(p, N, d, T, D, beta, dt, xi + b * per_xi, store_f32, pos + b * per_pos))
#pragma omp atomic write
            fail = 1;
    return fail ? -1 : 0;
}

/* ---------------------------------------------------------------- */
/* One whole-path Metropolis-adjusted Langevin step on the path
 * distribution exp(-S[X]) with the tail slice x_0 held fixed (the paper
 * holds the tail endpoint fixed during path updates, Sec. III, and accepts
 * by Metropolis-Hastings).  Proposal, for t >= 1:
 *     x'_t = x_t - h g_t + sqrt(2h) eta_t,     x'_0 = x_0,
 * with g = dS/dx at x.  Acceptance:
 *     log alpha = S(x) - S(x') - q(x | x') + q(x' | x),
 *     q(y | x) = sum_{t>=1} |y_t - x_t + h g_t(x)|^2 / (4h),
 * accept iff log_u < log alpha.
 * Inputs: pos, S, grad at the current path; eta[t][m] (slice 0 ignored).
 * Outputs: prop (x'), S_prop, grad_prop, *log_alpha, *accepted.
 * store_f32 != 0 rounds x' to single precision (the GPU stores FP32). */
int or_mala_step(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                 double h, const double* pos, double S, const double* grad, const double* eta,
                 double log_u, int store_f32, double* prop, double* S_prop, double* grad_prop,
                 double* log_alpha, int* accepted, int nthreads)
{
    int M = d * N;
    size_t n = (size_t)(T + 1) * M;
    double s2h = sqrt(2.0 * h);
    for (size_t e = 0; e < (size_t)M; ++e) prop[e] = pos[e];
    for (size_t e = M; e < n; ++e) {
        double v = pos[e] - h * grad[e] + s2h * eta[e];
        prop[e] = store_f32 ? (double)(float)v : v;
    }
    if (or_action_grad(p, N, d, T, D, beta, dt, prop, S_prop, grad_prop, nthreads)) return -1;
    double q_fwd = 0.0, q_rev = 0.0;
    for (size_t e = M; e < n; ++e) {
        double f = prop[e] - pos[e] + h * grad[e];
        double b = pos[e] - prop[e] + h * grad_prop[e];
        q_fwd += f * f;
        q_rev += b * b;
    }
    double la = S - *S_prop - q_rev / (4.0 * h) + q_fwd / (4.0 * h);
    *log_alpha = la;
    *accepted = (log_u < la) ? 1 : 0;
    return 0;
}

/* ---------------------------------------------------------------- */
/* One multilevel sliding-and-sampling Monte Carlo step (paper Sec. III,
 * Fig. 5) at level `level` with fragmentation offset `offset` in [0, 2^level).
 * Shared fragment endpoints sit at 0 and at offset + k 2^level (0 < . < T); the
 * tail x_0 and every shared endpoint stay fixed, the nose fragment
 * [last endpoint, T] moves its end x_T.  Each fragment is updated
 * independently by Metropolis-Hastings with a trial path of the free particle
 * (V = 0) with the same D and dt: a Brownian bridge between the fixed ends of
 * an interior fragment, a free random walk for the nose.  The trial density is
 * exp(-S0) with S0 = sum |x_{t+1} - x_t|^2 / (4 D dt) (up to factors that do not
 * depend on the interior points), so
 *     log alpha = -(S(X') - S(X)) + (S0(X') - S0(X)),
 * both differences over the fragment's own steps.  The trial starts from the
 * free random walk W_t = sig (z_{a+1} + ... + z_t), t in (a, b], with z[t][m]
 * standard normals and sig = sqrt(2 D dt):
 *     nose:    x'_t = x_a + W_t
 *     bridge:  x'_t = x_a + s (x_b - x_a) + (W_t - s W_b),   s = (t - a)/(b - a),
 * the textbook Brownian bridge: a walk with its end pulled back to x_b by a
 * linear correction (x'_b = x_b exactly).
 * log_u[f] decides fragment f (in order from the tail).  Returns the number of
 * fragments; *n_acc counts accepted fragments with interior points.
 *
 * exact_ho = 1 (harmonic potential only) replaces the short-time propagator of
 * Eq. (3) in S by the exact transition density of the overdamped oscillator
 * (the marginal of Sec. II for V = k x^2 / 2, with gamma^-1 = beta D):
 *     K(x'|x) ~ exp(-(beta k / 2) |x' - phi x|^2 / (1 - phi^2)),  phi = exp(-beta D k dt),
 * so each step contributes |x' - phi x|^2 beta k / (2 (1 - phi^2)).  The trial
 * distribution and S0 are unchanged. */
int or_fragment_step(const or_potential* p, int N, int d, int T, double D, double beta, double dt,
                     int level, int offset, const double* z, const double* log_u, double* pos,
                     int* n_acc, int* n_prop, int exact_ho)
{
    int M = d * N;
    double a = beta * D * dt, sig = sqrt(2.0 * D * dt), c4 = 1.0 / (4.0 * D * dt);
    if (exact_ho && p->kind != OR_HARMONIC) return -2;
    double phi = exp(-beta * D * p->k * dt);
    double cx = beta * p->k / (2.0 * (1.0 - phi * phi));
    int len = 1 << level;
    double* trial = (double*)malloc(sizeof(double) * (size_t)(T + 1) * M);
    double* F = (double*)malloc(sizeof(double) * (size_t)M);
    double* Ft = (double*)malloc(sizeof(double) * (size_t)M);
    if (!trial || !F || !Ft) { free(trial); free(F); free(Ft); return -1; }
    /* fragment boundaries */
    int nb = 0;
    int* bnd = (int*)malloc(sizeof(int) * (size_t)(T / len + 3));
    bnd[nb++] = 0;
    for (int e = offset; e < T; e += len)
        if (e > 0) bnd[nb++] = e;
    bnd[nb++] = T;
    int nfrag = nb - 1;
    *n_acc = 0;
    *n_prop = 0;
    for (int f = 0; f < nfrag; ++f) {
        int fa = bnd[f], fb = bnd[f + 1];
        int nose = (f == nfrag - 1);
        if (!nose && fb - fa < 2) continue; /* no interior point */
        ++*n_prop;
        /* trial path on [fa, fb]: the walk W first (held in `trial`), then the
         * bridge or nose built from it in place */
        for (int m = 0; m < M; ++m) {
            double xa = pos[(size_t)fa * M + m], xb = pos[(size_t)fb * M + m];
            double W = 0.0;
            for (int t = fa + 1; t <= fb; ++t) {
                W += sig * z[(size_t)t * M + m];
                trial[(size_t)t * M + m] = W;
            }
            double Wb = W;
            trial[(size_t)fa * M + m] = xa;
            for (int t = fa + 1; t <= fb; ++t) {
                double y;
                if (nose) {
                    y = xa + trial[(size_t)t * M + m];
                } else if (t == fb) {
                    y = xb;
                } else {
                    double sf = (double)(t - fa) / (double)(fb - fa);
                    y = xa + sf * (xb - xa) + (trial[(size_t)t * M + m] - sf * Wb);
                }
                trial[(size_t)t * M + m] = y;
            }
        }
        /* action differences over the fragment's steps */
        double dS = 0.0, dS0 = 0.0;
        for (int t = fa; t < fb; ++t) {
            or_force(p, N, d, pos + (size_t)t * M, F);
            or_force(p, N, d, trial + (size_t)t * M, Ft);
            for (int m = 0; m < M; ++m) {
                double x0 = pos[(size_t)t * M + m], x1 = pos[(size_t)(t + 1) * M + m];
                double y0 = trial[(size_t)t * M + m], y1 = trial[(size_t)(t + 1) * M + m];
                if (exact_ho) {
                    double r = x1 - phi * x0, rt = y1 - phi * y0;
                    dS += (rt * rt - r * r) * cx;
                } else {
                    double r = x1 - x0 - a * F[m], rt = y1 - y0 - a * Ft[m];
                    dS += (rt * rt - r * r) * c4;
                }
                dS0 += ((y1 - y0) * (y1 - y0) - (x1 - x0) * (x1 - x0)) * c4;
            }
        }
        double la = -dS + dS0;
        if (log_u[f] < la) {
            ++*n_acc;
            for (int t = fa + 1; t <= fb; ++t)
                for (int m = 0; m < M; ++m) pos[(size_t)t * M + m] = trial[(size_t)t * M + m];
        }
    }
    free(bnd);
    free(trial);
    free(F);
    free(Ft);
    return nfrag;
}

/* ---------------------------------------------------------------- */
/* Shift and regenerate (paper Fig. 2, Sec. II.A): the trajectory advances by
 * n_shift steps -- traj[k] = x_{k+1}, k < n_shift -- the path drops its first
 * n_shift steps, and n_shift new slices are grown from the nose with the
 * trial distribution of the sampler (free particle):
 *     out[t] = pos[t + n_shift]                      (t <= T - n_shift)
 *     out[T - n_shift + k] = out[T - n_shift + k - 1] + sqrt(2 D dt) z[k-1]   (k = 1..n_shift)
 * z is [n_shift][M] standard normals. */
void or_shift_regenerate(int N, int d, int T, double D, double dt, int n_shift, const double* pos,
                         const double* z, double* out, double* traj)
{
    int M = d * N;
    double sig = sqrt(2.0 * D * dt);
    for (int k = 0; k < n_shift; ++k)
        for (int m = 0; m < M; ++m) traj[(size_t)k * M + m] = pos[(size_t)(k + 1) * M + m];
    for (int t = 0; t <= T - n_shift; ++t)
        for (int m = 0; m < M; ++m) out[(size_t)t * M + m] = pos[(size_t)(t + n_shift) * M + m];
    for (int k = 1; k <= n_shift; ++k)
        for (int m = 0; m < M; ++m)
            out[(size_t)(T - n_shift + k) * M + m] =
                out[(size_t)(T - n_shift + k - 1) * M + m] + sig * z[(size_t)(k - 1) * M + m];
}

/* ---------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with
 * the round keys bumped by the two Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normals for element e of one chain's noise stream.
 * Counter = (e/4, chain, counter_lo, counter_hi16 | stream<<16),
 * key = (seed_lo, seed_hi).  Each of the four words gives a 24-bit
 * uniform: u = ((w >> 8) + 1) 2^-24 in (0,1] for words 0 and 2,
 * v = (w >> 8) 2^-24 in [0,1) for words 1 and 3.  Box-Muller, evaluated
 * here in double precision:
 *   z0 = sqrt(-2 ln u0) cos(2 pi v1), z1 = sqrt(-2 ln u0) sin(2 pi v1),
 *   z2 = sqrt(-2 ln u2) cos(2 pi v3), z3 = sqrt(-2 ln u2) sin(2 pi v3);
 * element e takes z_(e mod 4). */
void or_normals(uint64_t seed, uint64_t counter, uint32_t stream, uint32_t chain,
                int64_t e0, int64_t n, double* out)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t q = 0; q < n; ++q) {
        int64_t e = e0 + q;
        uint32_t ctr[4] = {(uint32_t)(e >> 2), chain, (uint32_t)counter,
                           (uint32_t)((counter >> 32) & 0xFFFFu) | (stream << 16)};
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        int lane = (int)(e & 3);
        uint32_t wu = (lane < 2) ? w[0] : w[2];
        uint32_t wv = (lane < 2) ? w[1] : w[3];
        double u = ((double)(wu >> 8) + 1.0) * 0x1p-24;
        double v = (double)(wv >> 8) * 0x1p-24;
        double rad = sqrt(-2.0 * log(u));
        out[q] = (lane & 1) ? rad * sin(two_pi * v) : rad * cos(two_pi * v);
    }
}

/* Uniform in (0,1] for a chain's accept test (53 bits from words 0,1). */
double or_uniform(uint64_t seed, uint64_t counter, uint32_t stream, uint32_t chain)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {0u, chain, (uint32_t)counter,
                       (uint32_t)((counter >> 32) & 0xFFFFu) | (stream << 16)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    return ((double)((uint64_t)(w[0] >> 5) * 67108864u + (w[1] >> 6)) + 1.0) * 0x1p-53;
}

/* ---------------------------------------------------------------- */
/* Number of ordered pairs (i != j) within the cutoff at one slice, with
 * the inclusion decision taken in single precision by the documented rule
 * shared with the GPU (an integer decided by floating point is compared
 * bit for bit, so both sides decide in the kernel's precision):
 *   Lf = (float)box, iLf = 1.0f / Lf, rc2f = (float)rc * (float)rc,
 *   dx = xi - xj;  k = fmaf(dx, iLf, 1.5*2^23) - 1.5*2^23  (nearest integer
 *   to the exact product);  dx = fmaf(-Lf, k, dx)            (per component)
 *   r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));   include iff r2 <= rc2f.
 * x is one slice [3][N] in single precision. */
long long or_pair_count_f32(int N, double box, double rc, const float* x)
{
    float Lf = (float)box;
    float iLf = 1.0f / Lf;
    float rcf = (float)rc;
    float rc2f = rcf * rcf;
    long long count = 0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (i == j) continue;
            float dxyz[3];
            for (int c = 0; c < 3; ++c) {
                float dx = x[c * N + i] - x[c * N + j];
                float sh = fmaf(dx, iLf, 12582912.0f) - 12582912.0f;
                dxyz[c] = fmaf(-Lf, sh, dx);
            }
            float xx = dxyz[0] * dxyz[0];
            float r2 = fmaf(dxyz[2], dxyz[2], fmaf(dxyz[1], dxyz[1], xx));
            if (r2 <= rc2f) ++count;
        }
    return count;
}

/* ---------------------------------------------------------------- */
/* Hard-sphere path bias of the paper's Lennard-Jones runs (Sec. IV.B): slice t
 * of the path carries, besides the pair potential U of Eq. (11), the pair
 * potential U_HS(r; sigma_t) = +inf for r <= sigma_t and 0 beyond, sigma_t the
 * schedule's value at that slice.  Only pairs within the cutoff rc are tested
 * (a sigma_t at or above rc acts as rc).  The hard-sphere term adds no force
 * where it is finite, so it changes the action only through the +inf of a path
 * with such a pair at any slice t = 0..T.  Returns the first such slice, or -1.
 * All pairs, minimum image, double precision. */
int or_hs_first_overlap(const or_potential* p, int N, int d, int T, const double* pos,
                        const double* sigma_hs)
{
    int M = d * N;
    for (int t = 0; t <= T; ++t) {
        double lim = sigma_hs[t] < p->rc ? sigma_hs[t] : p->rc;
        if (!(lim > 0.0)) continue;
        const double* x = pos + (size_t)t * M;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                double r2 = 0.0;
                for (int c = 0; c < d; ++c) {
                    double dx = min_image(p, x[c * N + i] - x[c * N + j]);
                    r2 += dx * dx;
                }
                if (r2 <= lim * lim) return t;
            }
    }
    return -1;
}

/* The same decision at one slice in the kernels' single precision (an integer
 * outcome decided in floating point, compared bit for bit): the pair vector by
 * the rule of or_pair_count_f32, included iff r2 <= rc2f (the cutoff) and
 * r2 <= (float)(sigma * sigma).  Returns 1 if some pair i < j is included. */
int or_hs_overlap_f32(int N, double box, double rc, double sigma, const float* x)
{
    float Lf = (float)box;
    float iLf = 1.0f / Lf;
    float rcf = (float)rc;
    float rc2f = rcf * rcf;
    float hs2 = (float)(sigma * sigma);
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            float dxyz[3];
            for (int c = 0; c < 3; ++c) {
                float dx = x[c * N + i] - x[c * N + j];
                float sh = fmaf(dx, iLf, 12582912.0f) - 12582912.0f;
                dxyz[c] = fmaf(-Lf, sh, dx);
            }
            float xx = dxyz[0] * dxyz[0];
            float r2 = fmaf(dxyz[2], dxyz[2], fmaf(dxyz[1], dxyz[1], xx));
            if (r2 <= rc2f && r2 <= hs2) return 1;
        }
    return 0;
}

int or_num_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
