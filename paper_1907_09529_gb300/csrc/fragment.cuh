// fragment.cuh -- launchers of the multilevel sampler and of the PAMD loop's
// shift (paper Sec. III, Fig. 2), defined in fragment_kernels.cu.
#pragma once

#include "pamd_internal.cuh"

namespace pamd {

// Shift every chain of one system by n_shift steps into `out`, emit the
// trajectory points, regrow the nose with free-particle steps.
template <typename R>
cudaError_t launch_shift_regenerate(const R* pos, R* out, R* traj, long long off, long long traj_off,
                                    int T, int M, int n_shift, int n_chains, int chain0, double sig,
                                    uint64_t seed, uint64_t counter, const R* noise, cudaStream_t st);

// Largest shared-memory footprint of the one-CTA-per-chain fragment kernels;
// larger chains take the one-thread-per-fragment kernel.
constexpr size_t kFragBlockSmemMax = 192 * 1024;

// Whether the last MC step of a shifting event can also shift the path.
template <typename R>
bool fragment_event_fusable(int T, int M, int l_min, int n_shift);

// One multilevel sliding-and-sampling MC step of every chain of one harmonic
// system (free-particle trials).  g, cS: drift factor and action scale of a
// step, S_t = cS |x_{t+1} - x_t + g x_t|^2; c0: scale of the free-particle trial
// action.  shift_out != nullptr: the step also performs the shift of a shifting
// event (one-line systems only, see fragment_event_fusable), regrowing with
// steps of width shift_sig.
template <typename R>
cudaError_t launch_fragment_mc(R* pos, long long off, int T, int M, int n_chains, int chain0,
                               int l_min, int l_max, uint64_t seed, uint64_t counter,
                               const int* levels, const int* offsets, const R* noise,
                               const double* log_u, int fstride, double g, double sig, double cS,
                               double c0, int* n_accepted, int* n_proposed, cudaStream_t st,
                               R* shift_out = nullptr, R* shift_traj = nullptr, int n_shift = 0,
                               uint64_t shift_counter = 0, double shift_sig = 0.0);
}  // namespace pamd
