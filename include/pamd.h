/*
 * pamd.h -- C ABI of libpamd, the GB300 (sm_103a) path-action library for
 * path-accelerated molecular dynamics (Rosa-Raices, Zhang & Miller,
 * arXiv:1907.09529).
 *
 * The library evaluates, for every timeslice of whole Brownian-dynamics
 * paths at once, the force F(x_t), the Euler-Maruyama residual
 *     r_t = x_{t+1} - x_t - beta D dt F(x_t)                   (Sec. II.A, Eq. (3))
 * the action
 *     S = sum_{t=0}^{T-1} |r_t|^2 / (4 D dt)                    (Eq. (4), unnormalised)
 * and its path gradient
 *     dS/dx_t = [r_{t-1} - r_t + beta D dt H(x_t) r_t] / (2 D dt),  r_{-1} = r_T = 0,
 * with H the Hessian of the potential (Eq. (1): drift -gamma^-1 V',
 * D = 1/(beta gamma)).  The normalisation of the short-time propagator of
 * Eq. (3) is dropped; it does not depend on the path.
 *
 * Data layout.  A chain's path is T+1 slices, each slice [dim][N] (all
 * x coordinates of the particles, then all y, then all z):
 *     pos[t][c][n],  element index (t*dim + c)*N + n.
 * A system's chains follow one another contiguously starting at element
 * `pos_offset` of the buffer; gradients use exactly the same layout.
 * Chains are numbered globally in system order; per-chain arrays (S,
 * acceptance counters, ...) are indexed by that number.
 *
 * Precision.  PAMD_FP32: positions, forces, residuals and gradients are
 * float; every action, acceptance term and Metropolis comparison is
 * accumulated and taken in double.  PAMD_FP64: everything is double
 * ("plain" form).  The position/gradient buffers hold the element type of
 * the chosen precision.
 *
 * Pointers.  Unless stated otherwise a pointer argument may be a device
 * pointer or a host pointer.  Device pointers must be allocated by the
 * caller (the library never frees them).  If ANY buffer argument of a call
 * is a host pointer, the library copies inputs to its own device workspace,
 * runs, copies results back, and synchronises `stream` before returning.
 * With device pointers every call is asynchronous on `stream`.  Device
 * buffers must be 16-byte aligned, and are read in whole 16-byte units: a
 * buffer must stay readable up to its end rounded up to 16 bytes (any
 * cudaMalloc'd buffer is).  A device path, gradient, noise or trajectory
 * buffer that is not 16-byte aligned (a view at an odd element offset) is
 * refused with PAMD_ERR_ARG before any other check and before anything runs.
 *
 * Errors.  Every entry point returns PAMD_OK (0) or a negative status; no
 * C++ exception crosses this boundary.  On error nothing is guaranteed
 * about the output buffers.
 *
 * First use.  The first call for a given problem shape builds a plan and
 * allocates its device workspace (cudaMalloc); make that first call before
 * any stream capture.  pamd_release_cache() frees all of it.
 *
 * Fault injection (tests of the error paths; nothing faults on the device).
 * With the environment variable PAMD_FAULT_INJECT set to "alloc", every
 * workspace allocation fails (PAMD_ERR_ALLOC; a plan that could not be built is
 * not cached); "launch": every CUDA call the library checks reports failure
 * (PAMD_ERR_CUDA; a graph whose capture failed is not cached); "nonfinite":
 * every action computed is flagged non-finite (pamd_device_status then returns
 * PAMD_ERR_NONFINITE).  The variable is read at each call.
 */
#ifndef PAMD_H
#define PAMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PAMD_OK 0
#define PAMD_ERR_ARG (-1)          /* invalid argument or shape */
#define PAMD_ERR_UNSUPPORTED (-2)  /* valid, but outside what the kernels handle */
#define PAMD_ERR_CUDA (-3)         /* a CUDA runtime call or launch failed */
#define PAMD_ERR_TIMEOUT (-4)      /* a bounded device wait ran out (reserved: no kernel of
                                      this library waits on another, so no call returns it) */
#define PAMD_ERR_NONFINITE (-5)    /* a non-finite action was produced */
#define PAMD_ERR_ALLOC (-6)        /* workspace allocation failed */

/* Potential kinds. */
#define PAMD_HARMONIC 0  /* V = k/2 |x|^2 per coordinate (Sec. IV.A, isotropic in dim) */
#define PAMD_LJ 1        /* cut-and-force-shifted Lennard-Jones, Eq. (11), periodic cube */

/* Precisions. */
#define PAMD_FP32 0      /* float data, double accumulation of S and acceptance terms */
#define PAMD_FP64 1      /* double everywhere */

/* Potential parameters (Eq. (11): U(r) = u(r) - u(rc) - (r - rc) u'(rc) for r <= rc,
 * u(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6]).  For PAMD_LJ, 0 < rc <= box/2 is
 * required (only the nearest periodic image can then interact) and dim must be 3.
 * For PAMD_HARMONIC only k is read. */
typedef struct {
    int kind;
    double k;
    double eps, sigma, rc, box;
} pamd_potential;

/* One system: n_chains independent paths of n_steps steps (n_steps+1 slices)
 * of n_particles particles in dim dimensions.  Supported: 1 <= dim <= 3,
 * n_steps >= 1; PAMD_LJ: 2 <= n_particles <= 1024.
 *
 * Time slabs.  The forces of different timesteps are independent (Sec. II.B),
 * so one long path can be split in time over several processes: rank k of K
 * owns steps [s_k, s_{k+1}) and slices [s_k, s_{k+1}) of every chain (the last
 * rank also slice T).  Its buffer holds, per chain, the whole path's slices
 * [s_k - halo_lo, s_{k+1}], so n_steps = s_{k+1} - s_k + halo_lo, and
 *   first_slice : global index of local slice 0 (s_k - halo_lo);
 *   halo_lo     : 1 when local slice 0 is the previous rank's last slice
 *                 x_{s_k - 1}: its step only supplies the residual r_{s_k - 1}
 *                 that the gradient at x_{s_k} needs (its force is evaluated
 *                 here again, so ranks exchange positions only); 0 for rank 0
 *                 (then first_slice = 0);
 *   halo_hi     : 1 when the last local slice is the next rank's first slice
 *                 x_{s_{k+1}} (its gradient belongs to that rank); 0 for the
 *                 last rank.
 * pamd_action and pamd_action_grad then return this rank's part of S (its
 * owned steps; the caller sums the parts) and the whole path's gradient at the
 * owned slices; the halo slices of grad are left unchanged.  The MALA pieces
 * below work on the owned slices and draw the whole path's noise (elements
 * counted from global slice 0).  Every other entry point requires
 * first_slice = halo_lo = halo_hi = 0 (whole paths), PAMD_ERR_UNSUPPORTED
 * otherwise. */
typedef struct {
    int n_particles;
    int n_steps;
    int dim;
    int n_chains;
    long long pos_offset;  /* element offset of chain 0, slice 0 in pos/grad buffers */
    pamd_potential pot;
    long long first_slice; /* time slab: global index of local slice 0 (0: whole path) */
    int halo_lo, halo_hi;  /* time slab: halo slice below / above the owned slices */
} pamd_system;

/* A batch of systems sharing D, beta, dt (paper notation; dt is the path
 * discretisation step, beta the inverse temperature, D the diffusion
 * coefficient).  `systems` is a host array of n_systems entries. */
typedef struct {
    double D, beta, dt;
    int n_systems;
    const pamd_system* systems;
    int precision;  /* PAMD_FP32 or PAMD_FP64 */
    int flags;      /* 0, or PAMD_FLAG_* below */
} pamd_problem;

/* Run one chain per launch (the "plain" single-path form). */
#define PAMD_FLAG_ONE_CHAIN_PER_LAUNCH 1
/* Multilevel sampler and PAMD loop only (pamd_fragment_mc, pamd_event): the
 * harmonic systems' path action uses the oscillator's exact transition
 * density (the marginal of Sec. II for V = k|x|^2/2, gamma^-1 = beta D),
 *     S = sum_t |x_{t+1} - phi x_t|^2 beta k / (2 (1 - phi^2)),  phi = exp(-beta D k dt),
 * in place of Eq. (3); trials and regeneration are unchanged.  The action,
 * gradient, update and Euler entry points reject it (PAMD_ERR_UNSUPPORTED). */
#define PAMD_FLAG_HO_EXACT_PROPAGATOR 2
/* Shift and regeneration (pamd_shift_regenerate, pamd_event): continue the
 * path past the nose as the horizontal straight line x_T (Fig. 2B's
 * straight-line regeneration, zero slope) instead of free-particle steps. */
#define PAMD_FLAG_REGENERATE_FLAT 4

/* Action S of every chain (Eqs. (3)-(4)).
 *   pos : path buffer (precision's element type), layout above.
 *   S   : double[n_chains_total], written.
 * Returns PAMD_OK or an error status. */
int pamd_action(const pamd_problem* prob, const void* pos, double* S, void* stream);

/* Action and path gradient of every chain (Eqs. (3)-(4) differentiated).
 *   pos  : path buffer, read.
 *   S    : double[n_chains_total], written.
 *   grad : same layout and type as pos, written for all T+1 slices (x_0
 *          included; masking the fixed tail is the caller's business). */
int pamd_action_grad(const pamd_problem* prob, const void* pos, double* S, void* grad,
                     void* stream);

/* Action and path gradient with the hard-sphere path bias of the paper's
 * Lennard-Jones runs (Sec. IV.B): at slice t the pair potential is
 *     V(r; sigma_HS(t)) = U(r) + U_HS(r; sigma_HS(t)),
 *     U_HS = +inf for r <= sigma_HS(t), 0 beyond,
 * U the cut-and-force-shifted Lennard-Jones potential of Eq. (11) and sigma_HS(t)
 * a schedule along the path supplied by the caller.  U_HS adds no force where it
 * is finite, so:
 *   S[c]  = the Lennard-Jones action of chain c (as pamd_action_grad), or +inf if
 *           at some slice t = 0..T a pair within the cutoff lies at
 *           r <= sigma_HS(t) (minimum image, decided in the path's precision by
 *           the rule of pamd_lj_pair_counts, with the squared radius rounded to
 *           the element type; a radius <= 0 tests nothing, one >= rc acts as rc);
 *   grad  = the Lennard-Jones gradient (written as by pamd_action_grad), or NULL
 *           for the action only.
 *   sigma_hs : device double array: for every PAMD_LJ system in order, its T+1
 *           radii sigma_HS(0..T) (harmonic systems take none).
 * Harmonic systems get their plain action.  Device pointers only
 * (PAMD_ERR_ARG otherwise); whole paths only (PAMD_ERR_UNSUPPORTED for a time
 * slab).  Combined with the pamd_mala_* pieces, a proposal
 * with an overlapping pair has S' = +inf and is rejected.  The trial paths the
 * paper draws from a hard-sphere propagator are not part of this library. */
int pamd_action_grad_hs(const pamd_problem* prob, const void* pos, const double* sigma_hs,
                        double* S, void* grad, void* stream);

/* n_updates successive whole-path Metropolis-adjusted Langevin updates of
 * every chain, consuming the path gradient; the tail slice x_0 is held
 * fixed and the update is accepted by the Metropolis-Hastings test (the
 * paper's path-sampling move, Sec. III, with a gradient-informed trial):
 *     x'_t = x_t - h g_t + sqrt(2h) eta_t  (t >= 1),   x'_0 = x_0,
 *     log alpha = S(x) - S(x') - |x - x' + h g(x')|^2/(4h) + |x' - x + h g(x)|^2/(4h)
 * (sums over t >= 1), accepted iff log u < log alpha, all in double.
 *   pos, grad, S : in/out.  On entry grad and S must hold the gradient and
 *                  action of pos (from pamd_action_grad); on return they
 *                  hold those of the updated path.
 *   h            : step size (> 0).
 *   seed,counter : Philox4x32-10 key and counter; update u uses counter+u.
 *   noise        : NULL (normals drawn from Philox, stream 1) or, only with
 *                  n_updates == 1, standard normals eta in the layout of pos
 *                  (slice-0 entries ignored), element type of the precision.
 *   log_u        : NULL (uniforms from Philox, stream 2) or, only with
 *                  n_updates == 1, double[n_chains_total] of log uniforms.
 *   n_accepted   : int[n_chains_total], incremented by accepted updates (may be NULL).
 *   log_alpha    : double[n_chains_total], log alpha of the last update (may be NULL).
 * With device pointers and n_updates > 1 the updates are captured once into
 * a CUDA graph (cached per shape) and replayed.  With host buffers, no noise
 * and no log_u, and at least two chains, the call is pipelined over up to 8
 * chunks of chains: one chunk's buffers are copied in while earlier chunks
 * are updated (on up to three compute streams, so that several chunks' kernels
 * share the GPU) and copied back (the library's own streams, ordered after the
 * work already queued on `stream`); the results are bitwise those of the
 * device-pointer call, and the call returns once every result is on the host. */
int pamd_path_update(const pamd_problem* prob, void* pos, void* grad, double* S, double h,
                     int n_updates, uint64_t seed, uint64_t counter, const void* noise,
                     const double* log_u, int* n_accepted, double* log_alpha, void* stream);

/* The update of pamd_path_update in pieces, for callers that split paths in
 * time over several processes (time slabs, see pamd_system) and must sum each
 * piece's per-chain terms over the processes before the next piece.  On whole
 * paths the sequence
 *     pamd_mala_propose -> pamd_action_grad(prop) -> pamd_mala_reverse
 *     -> pamd_mala_accept -> pamd_mala_commit
 * gives bitwise the result of pamd_path_update with n_updates = 1 and the same
 * seed, counter, noise and log_u.  Device pointers only (PAMD_ERR_ARG
 * otherwise); asynchronous on `stream`.
 *
 * pamd_mala_propose: prop = x - h g + sqrt(2h) eta on the owned slices other
 *   than the fixed tail (global slice 0); the other slices of prop are copied
 *   from pos.  q_fwd : double[n_chains_total], written, this slab's part of
 *   sum |x' - x + h g|^2 over those slices.  noise: NULL (Philox stream 1, the
 *   element index counted from global slice 0) or normals in the layout of pos. */
int pamd_mala_propose(const pamd_problem* prob, const void* pos, const void* grad, void* prop,
                      double h, uint64_t seed, uint64_t counter, const void* noise, double* q_fwd,
                      void* stream);

/* pamd_mala_reverse: q_rev : double[n_chains_total], written, this slab's part of
 *   sum |x - x' + h g(x')|^2 over the proposed slices. */
int pamd_mala_reverse(const pamd_problem* prob, const void* pos, const void* prop,
                      const void* grad_prop, double h, double* q_rev, void* stream);

/* pamd_mala_accept: per chain, from whole-path sums (device double[n_chains_total]
 *   each: S = S(x), S_prop = S(x'), q_fwd, q_rev),
 *       log alpha = S - S_prop - q_rev/(4h) + q_fwd/(4h),
 *   accepted iff log u < log alpha, in double; log_u NULL (Philox stream 2,
 *   counter) or double[n_chains_total].  accept : int[n_chains_total], written
 *   (1 or 0); n_accepted (incremented) and log_alpha (written) may be NULL.  The
 *   same inputs give the same decisions on every process. */
int pamd_mala_accept(const pamd_problem* prob, const double* S, const double* S_prop,
                     const double* q_fwd, const double* q_rev, double h, uint64_t seed,
                     uint64_t counter, const double* log_u, int* accept, int* n_accepted,
                     double* log_alpha, void* stream);

/* pamd_mala_commit: for every chain with accept[c] != 0, pos <- prop and
 *   grad <- grad_prop over all its slices (halos included) and S[c] <- S_prop[c]. */
int pamd_mala_commit(const pamd_problem* prob, void* pos, void* grad, double* S, const void* prop,
                     const void* grad_prop, const double* S_prop, const int* accept,
                     void* stream);

/* Forward Euler-Maruyama paths (Eq. (2)), sequential in time:
 *     x_{t+1} = x_t + beta D dt F(x_t) + sqrt(2 D dt) xi_t,
 * each new slice stored in the precision's element type and used as stored.
 *   pos   : in/out; slice 0 of every chain holds x_0 on entry, slices 1..T
 *           are written.
 *   noise : NULL (normals from Philox, stream 0, seed/counter) or standard
 *           normals in the layout of pos, slice t+1 holding xi_t (slice-0
 *           entries ignored). */
int pamd_euler_reference(const pamd_problem* prob, void* pos, uint64_t seed, uint64_t counter,
                         const void* noise, void* stream);

/* n_steps multilevel sliding-and-sampling Monte Carlo steps (paper Sec. III,
 * Fig. 5) of every chain of harmonic systems, with free-particle trial paths.
 * A step of a chain draws a level l in [l_min, l_max] and an offset o in
 * [0, 2^l); the fragments' shared endpoints are 0 and o + k 2^l (0 < . < T),
 * the tail x_0 and the shared endpoints stay fixed and the nose fragment moves
 * x_T.  Each fragment is accepted or rejected on its own by Metropolis-Hastings
 * with a Brownian-bridge trial (random walk for the nose):
 *     log alpha = -(S(X') - S(X)) + (S0(X') - S0(X)),  S0 = free-particle action,
 * both over the fragment's steps: per-step terms (r'-r)(r'+r) in the path's
 * precision, fragment sums and the accept test in double.
 *   pos         : in/out, device buffer (precision's element type).
 *   l_min,l_max : 1 <= l_min <= l_max, 2^l_max <= T of every system.
 *   seed,counter: Philox key and counter (step u uses counter+u; streams 3-5:
 *                 level/offset from words 0/1 modulo the range, trial normals,
 *                 per-fragment 53-bit uniforms).
 *   levels, offsets : NULL, or (only with n_steps == 1) int[n_chains_total]
 *                 each, the fragmentation of every chain; a chain whose level
 *                 lies outside [l_min, l_max] or whose offset lies outside
 *                 [0, 2^level) is left unchanged and proposes nothing.
 *   noise       : NULL, or (n_steps == 1) standard normals in the layout of pos;
 *                 slice t+1's entries drive the trial step t -> t+1.
 *   log_u       : NULL, or (n_steps == 1) double[n_chains_total * F] with
 *                 F = max over systems of (T >> l_min) + 2; fragment f (counted
 *                 from the tail) of chain c uses log_u[c*F + f].
 *   n_accepted, n_proposed : int[n_chains_total], incremented (fragments with
 *                 interior points are proposed).
 * The trial of a fragment [a, b] is built from the walk
 * W_t = sqrt(2 D dt) (z_{a+1} + ... + z_t): x_a + W_t for the nose, and
 * x_a + s (x_b - x_a) + W_t - s W_b with s = (t-a)/(b-a) for a bridge.  A chain
 * whose path (two copies) fits in shared memory is handled by one CTA.
 * Device pointers only (host pointers: PAMD_ERR_ARG); Lennard-Jones systems:
 * PAMD_ERR_UNSUPPORTED (their trial needs a hard-sphere pair propagator). */
int pamd_fragment_mc(const pamd_problem* prob, void* pos, int l_min, int l_max, int n_steps,
                     uint64_t seed, uint64_t counter, const int* levels, const int* offsets,
                     const void* noise, const double* log_u, int* n_accepted, int* n_proposed,
                     void* stream);

/* Shift and regenerate (paper Fig. 2): every chain's trajectory advances by
 * n_shift steps and its path is grown back to n_steps at the nose.
 *   pos     : path buffer, read (device).
 *   pos_out : another path buffer of the same layout, written: slices
 *             0..T-n_shift are pos's slices n_shift..T; the last n_shift slices
 *             continue from the nose by free-particle steps x + sqrt(2 D dt) z
 *             (the sampler's trial distribution), or hold x_T with
 *             PAMD_FLAG_REGENERATE_FLAT.
 *   traj    : written, the trajectory points x_1..x_{n_shift} of every chain:
 *             [chains][n_shift][dim][N] per system, systems one after another.
 *   noise   : NULL (Philox stream 6, seed/counter) or standard normals
 *             [n_chains_total][n_shift][dim][N] (every system uses its dim*N).
 * Device pointers only; pos and pos_out must differ. */
int pamd_shift_regenerate(const pamd_problem* prob, const void* pos, void* pos_out, int n_shift,
                          void* traj, uint64_t seed, uint64_t counter, const void* noise,
                          void* stream);

/* One shifting event of the path-accelerated MD loop (paper Fig. 2) for every
 * chain of harmonic systems: n_sample multilevel MC steps (as pamd_fragment_mc
 * with counters event*n_sample + u, u = 0..n_sample-1), then the shift and
 * regeneration (as pamd_shift_regenerate with counter `event`).  The results
 * are bit-identical to that sequence of calls.  For one-line systems (dim*N
 * == 1) whose path fits in shared memory the last MC step writes the shifted
 * path, the trajectory points and the regrown nose itself, so the event reads
 * and writes every path once.
 *   pos      : in/out, the paths; on return the paths after the MC steps.
 *   pos_out  : written, the shifted and regrown paths (another buffer).
 *   traj     : written, x_1..x_{n_shift} of every chain (layout as in
 *              pamd_shift_regenerate).
 *   n_accepted, n_proposed : int[n_chains_total], incremented.
 * Device pointers only; l_min, l_max and n_shift as in pamd_fragment_mc and
 * pamd_shift_regenerate; Lennard-Jones systems: PAMD_ERR_UNSUPPORTED. */
int pamd_event(const pamd_problem* prob, void* pos, void* pos_out, int n_sample, int n_shift,
               int l_min, int l_max, void* traj, uint64_t seed, uint64_t event, int* n_accepted,
               int* n_proposed, void* stream);

/* Diagnostics for bit-exact index parity: number of ordered in-cutoff pairs
 * (i != j) of every slice of every LJ chain, decided in single precision by
 * the kernels' rule (dx = xi - xj; k = fmaf(dx, 1/L, 1.5*2^23) - 1.5*2^23;
 * dx = fmaf(-L, k, dx); r2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx)); in iff
 * r2 <= rc*rc), with L, 1/L, rc*rc rounded to float.  PAMD_FP32 only.
 *   counts : long long[sum over LJ chains of (T+1)], chain-major, written.
 * A Lennard-Jones system with more than 65535 chains: PAMD_ERR_UNSUPPORTED. */
int pamd_lj_pair_counts(const pamd_problem* prob, const void* pos, long long* counts,
                        void* stream);

/* Raw Philox4x32-10 output (Salmon et al., SC'11) for n consecutive
 * counters: block q uses counter (ctr0 + q, ctr1, ctr2, ctr3), key (key0, key1);
 * out: uint32[4 n], written (device or host). */
int pamd_philox(uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, uint32_t key0,
                uint32_t key1, long long n, uint32_t* out, void* stream);

/* Standard normals of the library's noise streams for elements e0..e0+n-1
 * of one chain (the same values pamd_path_update / pamd_euler_reference
 * draw): Philox4x32-10 with counter (e/4, chain, counter_lo,
 * counter_hi16 | stream<<16) and key (seed_lo, seed_hi); the four words
 * give 24-bit uniforms u = ((w>>8)+1)/2^24 (words 0, 2) and v = (w>>8)/2^24
 * (words 1, 3); z = sqrt(-2 ln u) (cos, sin)(2 pi v) in single precision.
 *   out : float[n], written. */
int pamd_normals(uint64_t seed, uint64_t counter, uint32_t stream_id, uint32_t chain,
                 long long e0, long long n, float* out, void* stream);

/* Status left on the device by earlier asynchronous calls: synchronises
 * `stream`, then returns PAMD_ERR_NONFINITE (and clears it) if an action
 * computed since the last check was not finite (overlapping particles, an
 * exploding path), else PAMD_OK. */
int pamd_device_status(void* stream);

/* Launch-shape override for the Lennard-Jones kernels (0 or a negative skin
 * keeps the automatic choice): steps per CTA tile, threads per particle
 * (1, 2 or 4), neighbour-list capacity per particle, Verlet skin (sigma
 * units; double precision), steps per neighbour-list window (single
 * precision; >= 2).  Affects plans built afterwards.  Results do not depend
 * on the tile, capacity, skin or window (candidate order is fixed); the
 * number of threads per particle changes how a particle's force and
 * Hessian sums are split, so results differ by rounding only.  PAMD_ERR_ARG
 * for a negative size, an unsupported thread count or a window of 1.
 * Host-side setting, not thread-safe against concurrent calls.
 *
 * Environment switches read when a plan is built (part of the plan's key, so
 * a change takes effect at the next call):
 *   PAMD_LJ_NO_PIPE=1        single precision: the two-pass gradient form
 *                            instead of the pipelined one (bitwise equal);
 *   PAMD_LJ_PER_STEP_SHIFT=1 single precision: the minimum image rounded at
 *                            every slice (bitwise equal);
 *   PAMD_LJ_ONE_CLASS=1      single precision: one launch for all LJ systems
 *                            instead of one per block-size class;
 *   PAMD_LJ_ONE_STEP=1       single precision through the one-step kernel;
 *   PAMD_PIPE_LANES=n        compute lanes of the host-buffer update pipeline
 *                            (1..4, default 3). */
int pamd_tune(int tile_steps, int threads_per_particle, int max_neighbours, double skin,
              int window_steps);

/* Harmonic action and gradient that allocates nothing (no counterpart in the
 * paper; it exists for callers, not for the method).
 *
 * Some callers cannot allocate device memory once they are running: a
 * process whose allocator has already reserved the GPU's memory for itself,
 * or a service that forbids cudaMalloc/cudaFree after start-up because they
 * synchronise the device and can fail under memory pressure.  This entry
 * point computes exactly what pamd_action_grad computes for harmonic systems,
 * using only the caller's buffers plus a fixed scratch array compiled into
 * the library: PAMD_NOALLOC_MAX_BLOCKS doubles (512 KiB) of block sums, one
 * per 4096 elements of every chain.  Every GPU that loads the library holds
 * that array until the process exits.
 *   prob : harmonic systems only (PAMD_FP32 or PAMD_FP64), whole paths; otherwise
 *          PAMD_ERR_ARG (time slabs: PAMD_ERR_UNSUPPORTED).  A problem needing more than PAMD_NOALLOC_MAX_BLOCKS
 *          blocks (sum over chains of ceil((T+1)*dim*N / 4096)), or with a
 *          system of more than 65535 chains, is rejected with
 *          PAMD_ERR_UNSUPPORTED before anything is enqueued.
 *   pos, S, grad : device pointers on the current device (host pointers, or
 *          another device's memory: PAMD_ERR_ARG), as in pamd_action_grad.
 * No cudaMalloc, cudaFree or allocating library call is made.  Every call made
 * outside stream capture looks up the scratch array's device address
 * (cudaGetSymbolAddress) on the current device, so the address stays right
 * after a device reset; a call made while `stream` is capturing uses the
 * address found by an earlier uncaptured call on that device, so make one
 * call on each device before any stream capture (otherwise PAMD_ERR_CUDA).
 * All calls share the one array and it keeps the
 * last call's contents (every block sum is written before it is read, so
 * nothing needs clearing); calls whose kernels overlap on the GPU -- on two
 * streams, or from two threads -- race on it and must be serialised by the
 * caller. */
#define PAMD_NOALLOC_MAX_BLOCKS 65536
int pamd_ho_action_grad_noalloc(const pamd_problem* prob, const void* pos, double* S, void* grad,
                                void* stream);

/* Measured FP32 fused multiply-add throughput, the denominator of the
 * single-precision roofline (a diagnostic; the paper has no counterpart).
 * Launches `blocks` CTAs of `threads` threads on `stream`; every thread runs 8
 * independent chains of `iters` dependent FMAs, scalar (packed == 0) or packed
 * two-wide f32x2 instructions (packed != 0).  The caller times the launch (CUDA
 * events on `stream`) and divides *flops (FMA = 2 flops, written on return) by
 * the duration.
 *   out   : float[blocks * threads], device memory, written (keeps the chains live).
 *   flops : host double, written; may be NULL.
 * PAMD_ERR_ARG for a non-device `out`, threads not a multiple of 32 in
 * [32, 1024], or blocks / iters < 1. */
int pamd_fp32_fma_probe(int packed, int blocks, int threads, int iters, float* out,
                        double* flops, void* stream);

/* Measured FP64 fused multiply-add throughput, the rate that bounds the plain
 * double-precision form (a diagnostic, as above): 8 independent chains of
 * `iters` dependent fma.rn.f64 per thread.
 *   out   : double[blocks * threads], device memory, written.
 *   flops : host double, written (FMA = 2 flops); may be NULL.
 * PAMD_ERR_ARG as for pamd_fp32_fma_probe. */
int pamd_fp64_fma_probe(int blocks, int threads, int iters, double* out, double* flops,
                        void* stream);

/* Bounds checks of the debug build (a diagnostic; the paper has no counterpart).
 * libpamd_debug.so is this library compiled with -DPAMD_DEBUG: every array
 * index of the Lennard-Jones, oscillator, update and multilevel-sampler kernels
 * is checked, and an index outside its array is recorded on the device and the
 * access sent to a scratch sink instead (nothing traps, nothing outside the
 * arrays is touched).  This call synchronises the device, then reports
 *   *checked : 1 in the debug build, 0 in the normal library (no checks);
 *   *count   : out-of-bounds accesses recorded since the last call;
 *   *site, *index, *bound : the first of them: file * 100000 + source line
 *              (files 1..5: ho_kernels, lj_kernels, lj_paired, update_kernels,
 *              fragment_kernels), the index and the array's extent,
 * and clears the records.  Any pointer may be NULL. */
int pamd_debug_status(int* checked, int* count, int* site, long long* index, long long* bound);

/* Human-readable name of a status code (static string). */
const char* pamd_status_string(int status);

/* Numbers of cached plans (one per problem shape and launch-shape override)
 * and of captured update graphs (one per plan, buffer set and update count):
 * a loop that repeats a call on the same buffers must leave both unchanged.
 * Either pointer may be NULL.  Host-side; no device work. */
int pamd_cache_stats(int* n_plans, int* n_graphs);

/* Timeline of the last pamd_path_update call that was pipelined over chunks of
 * chains (host buffers; a diagnostic, not part of the method): ms[0] is the
 * call's device time from its start to the last copy back, then for each chunk
 * k three times since the start: its inputs on the device, its update done,
 * its results on the host (ms[1 + 3k + 0..2]).  Writes min(max_entries,
 * 1 + 3 n_chunks) floats; *n_chunks (may be NULL) gets the number of chunks
 * (0 if no pipelined call was made).  Host-side; no device work. */
int pamd_pipeline_timeline(float* ms, int max_entries, int* n_chunks);

/* Free every cached plan, workspace and graph (synchronises the device). */
int pamd_release_cache(void);

/* Library version, for the bindings. */
int pamd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAMD_H */
