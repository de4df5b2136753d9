// fragment_kernels.cu -- multilevel sliding-and-sampling Monte Carlo on harmonic
// paths (paper Sec. III, Fig. 5), with free-particle trial paths.
//
// One MC step of a chain: a level l in [l_min, l_max] and an offset o in
// [0, 2^l) cut the path into fragments whose shared endpoints sit at 0 and at
// o + k 2^l (0 < . < T); the nose fragment ends at T and moves its end point.
// Every fragment is updated independently by Metropolis-Hastings with a trial
// from the free particle (V = 0, same D and dt): a Brownian bridge between the
// fixed ends of an interior fragment, a free random walk for the nose.  The
// trial density is exp(-S0), S0 = sum |x_{t+1} - x_t|^2/(4 D dt), so
//     log alpha = -(S(X') - S(X)) + (S0(X') - S0(X))
// over the fragment's own steps (each residual belongs to exactly one fragment,
// hence fragments are independent and run in parallel).  Trial, step by step:
//     bridge:  x'_{t+1} = x'_t + (x_b - x'_t)/(b - t) + sig sqrt((b-t-1)/(b-t)) z_{t+1}
//     nose:    x'_{t+1} = x'_t + sig z_{t+1},          sig = sqrt(2 D dt).
// One thread owns one fragment: it builds the trial on the fly, accumulates both
// action differences in double, draws its own uniform, and on acceptance builds
// the same trial again (same normals) and writes it.  Fragments share only
// fixed endpoints, so the writes never overlap.
#include <algorithm>

#include "pamd_internal.cuh"

namespace pamd {

struct FragSys {
    long long off;   // element offset of chain 0
    int T, M;        // steps, elements per slice
    int chain0;      // global index of chain 0
    double k;        // harmonic constant
};

// Level and offset of one chain's step (Philox stream 3), or given.
__device__ __forceinline__ void frag_cut(uint64_t seed, uint64_t counter, uint32_t chain, int l_min,
                                         int l_max, const int* levels, const int* offsets, int c,
                                         int& l, int& o)
{
    if (levels) {
        l = levels[c];
        o = offsets[c];
        return;
    }
    const uint4 ctr = make_uint4(0u, chain, (uint32_t)counter,
                                 (uint32_t)((counter >> 32) & 0xFFFFu) | (kStreamFragCut << 16));
    const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    l = l_min + (int)(w.x % (uint32_t)(l_max - l_min + 1));
    o = (int)(w.y % (1u << l));
}

template <typename R>
__global__ void __launch_bounds__(128)
    fragment_mc_kernel(R* __restrict__ pos, const FragSys S, int l_min, int l_max, uint64_t seed,
                       uint64_t counter, const int* __restrict__ levels,
                       const int* __restrict__ offsets, const R* __restrict__ noise,
                       const double* __restrict__ log_u, int fstride, R a, R sig, double c4,
                       int* __restrict__ n_accepted, int* __restrict__ n_proposed)
{
    const int b_chain = blockIdx.y;
    const int c = S.chain0 + b_chain;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    int l, o;
    frag_cut(seed, counter, (uint32_t)c, l_min, l_max, levels, offsets, c, l, o);
    const int len = 1 << l, T = S.T, M = S.M;
    const int first = o > 0 ? o : len;  // first interior endpoint
    const int n_in = first < T ? (T - 1 - first) / len + 1 : 0;
    const int nfrag = 1 + n_in;
    if (f >= nfrag) return;
    const int fa = (f == 0) ? 0 : first + (f - 1) * len;
    const int fb = (f == nfrag - 1) ? T : first + f * len;
    const bool nose = (f == nfrag - 1);
    if (!nose && fb - fa < 2) return;  // no interior point
    R* X = pos + S.off + (long long)b_chain * (long long)(T + 1) * M;
    const R* Z = noise ? noise + S.off + (long long)b_chain * (long long)(T + 1) * M : nullptr;
    const R ak = a * (R)S.k;

    auto znorm = [&](int t1, int m) -> R {
        const long long e = (long long)t1 * M + m;
        if (Z) return Z[e];
        const float4 q = philox_normals4(seed, counter, kStreamFragTrial, (uint32_t)c, (uint32_t)(e >> 2));
        return (R)pick4(q, (int)(e & 3));
    };

    // pass 1: action differences of the trial
    double dS = 0.0, dS0 = 0.0;
    for (int m = 0; m < M; ++m) {
        const R xb = X[(long long)fb * M + m];
        R y = X[(long long)fa * M + m];
        R x = y;
        for (int t = fa; t < fb; ++t) {
            const R x1 = X[(long long)(t + 1) * M + m];
            R y1;
            if (nose) {
                y1 = y + sig * znorm(t + 1, m);
            } else if (t + 1 == fb) {
                y1 = xb;
            } else {
                const R rem = (R)(fb - t);
                y1 = y + (xb - y) / rem + sig * sqrt((rem - R(1)) / rem) * znorm(t + 1, m);
            }
            const R r = (x1 - x) + ak * x, rt = (y1 - y) + ak * y;
            dS += ((double)rt * rt - (double)r * r) * c4;
            dS0 += ((double)(y1 - y) * (y1 - y) - (double)(x1 - x) * (x1 - x)) * c4;
            x = x1;
            y = y1;
        }
    }
    const double la = -dS + dS0;
    double lu;
    if (log_u) {
        lu = log_u[(long long)c * fstride + f];
    } else {
        const uint4 ctr = make_uint4((uint32_t)f, (uint32_t)c, (uint32_t)counter,
                                     (uint32_t)((counter >> 32) & 0xFFFFu) | (kStreamFragAccept << 16));
        const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const uint64_t mant = (uint64_t)(w.x >> 5) * 67108864ull + (uint64_t)(w.y >> 6);
        lu = log(((double)mant + 1.0) * 1.1102230246251565e-16);
    }
    atomicAdd(n_proposed + c, 1);
    if (!(lu < la)) return;
    atomicAdd(n_accepted + c, 1);
    // pass 2: the same trial again, written in place
    for (int m = 0; m < M; ++m) {
        const R xb = X[(long long)fb * M + m];
        R y = X[(long long)fa * M + m];
        const int tend = nose ? fb : fb - 1;
        for (int t = fa; t < tend; ++t) {
            R y1;
            if (nose) {
                y1 = y + sig * znorm(t + 1, m);
            } else {
                const R rem = (R)(fb - t);
                y1 = y + (xb - y) / rem + sig * sqrt((rem - R(1)) / rem) * znorm(t + 1, m);
            }
            X[(long long)(t + 1) * M + m] = y1;
            y = y1;
        }
    }
}

template <typename R>
cudaError_t launch_fragment_mc(R* pos, long long off, int T, int M, int n_chains, int chain0,
                               double k, int l_min, int l_max, uint64_t seed, uint64_t counter,
                               const int* levels, const int* offsets, const R* noise,
                               const double* log_u, int fstride, double a, double sig, double c4,
                               int* n_accepted, int* n_proposed, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    FragSys S;
    S.off = off;
    S.T = T;
    S.M = M;
    S.chain0 = chain0;
    S.k = k;
    const int maxfrag = (T >> l_min) + 2;
    const int threads = 128;
    dim3 grid((maxfrag + threads - 1) / threads, n_chains);
    fragment_mc_kernel<R><<<grid, threads, 0, st>>>(pos, S, l_min, l_max, seed, counter, levels,
                                                    offsets, noise, log_u, fstride, (R)a, (R)sig,
                                                    c4, n_accepted, n_proposed);
    return cudaGetLastError();
}

template cudaError_t launch_fragment_mc<float>(float*, long long, int, int, int, int, double, int,
                                               int, uint64_t, uint64_t, const int*, const int*,
                                               const float*, const double*, int, double, double,
                                               double, int*, int*, cudaStream_t);
template cudaError_t launch_fragment_mc<double>(double*, long long, int, int, int, int, double, int,
                                                int, uint64_t, uint64_t, const int*, const int*,
                                                const double*, const double*, int, double, double,
                                                double, int*, int*, cudaStream_t);

// ------------------------------------------------------------------ shift and regenerate
// Trajectory points x_1..x_{n_shift} of every chain are copied out, the path is
// shifted by n_shift steps into `out`, and the last n_shift slices of `out` are
// grown from the nose by free-particle steps x + sqrt(2 D dt) z (paper Fig. 2:
// the regenerated slices come from the sampler's trial distribution).
template <typename R>
__global__ void shift_copy_kernel(const R* __restrict__ pos, R* __restrict__ out,
                                  R* __restrict__ traj, long long off, long long traj_off, int T,
                                  int M, int n_shift, int n_chains)
{
    const long long per = (long long)(T + 1) * M;
    const long long n = (long long)n_chains * per;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / per, le = e - b * per;
        const long long src = le + (long long)n_shift * M;
        if (src < per) out[off + b * per + le] = pos[off + b * per + src];
        if (le >= M && le < (long long)(n_shift + 1) * M)
            traj[traj_off + b * (long long)n_shift * M + (le - M)] = pos[off + b * per + le];
    }
}

template <typename R>
__global__ void regenerate_kernel(R* __restrict__ out, long long off, int T, int M, int n_shift,
                                  int n_chains, int chain0, R sig, uint64_t seed, uint64_t counter,
                                  const R* __restrict__ noise)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)n_chains * M) return;
    const int b = (int)(g / M), m = (int)(g % M);
    const long long per = (long long)(T + 1) * M;
    R* X = out + off + b * per;
    R x = X[(long long)(T - n_shift) * M + m];
    for (int k = 1; k <= n_shift; ++k) {
        const long long e = (long long)(k - 1) * M + m;  // index into this chain's [n_shift][M] noise
        R z;
        if (noise) {
            z = noise[((long long)(chain0 + b)) * n_shift * M + e];
        } else {
            const float4 q = philox_normals4(seed, counter, kStreamRegenerate, (uint32_t)(chain0 + b),
                                             (uint32_t)(e >> 2));
            z = (R)pick4(q, (int)(e & 3));
        }
        x = x + sig * z;
        X[(long long)(T - n_shift + k) * M + m] = x;
    }
}

template <typename R>
cudaError_t launch_shift_regenerate(const R* pos, R* out, R* traj, long long off, long long traj_off,
                                    int T, int M, int n_shift, int n_chains, int chain0, double sig,
                                    uint64_t seed, uint64_t counter, const R* noise, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    const long long n = (long long)n_chains * (T + 1) * M;
    const int threads = 256;
    const int blocks = (int)std::min<long long>((n + threads - 1) / threads, 152LL * 16);
    shift_copy_kernel<R><<<blocks, threads, 0, st>>>(pos, out, traj, off, traj_off, T, M, n_shift,
                                                     n_chains);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nr = (long long)n_chains * M;
    regenerate_kernel<R><<<(unsigned)((nr + 127) / 128), 128, 0, st>>>(
        out, off, T, M, n_shift, n_chains, chain0, (R)sig, seed, counter, noise);
    return cudaGetLastError();
}

template cudaError_t launch_shift_regenerate<float>(const float*, float*, float*, long long, long long,
                                                    int, int, int, int, int, double, uint64_t,
                                                    uint64_t, const float*, cudaStream_t);
template cudaError_t launch_shift_regenerate<double>(const double*, double*, double*, long long,
                                                     long long, int, int, int, int, int, double,
                                                     uint64_t, uint64_t, const double*, cudaStream_t);

}  // namespace pamd
