// ho_kernels.cu -- harmonic-oscillator path action and gradient (memory bound),
// and the sequential Euler-Maruyama reference for the oscillator.
//
// Potential V = k/2 |x|^2 per coordinate (paper Sec. IV.A, isotropic in dim),
// so F = -k x and H = k I.  With a = beta D dt the residual of step t is
//   r_t = x_{t+1} - x_t - a F(x_t) = (x_{t+1} - x_t) + a k x_t        (Eq. (3))
// and the gradient of S = sum |r_t|^2 / (4 D dt) with respect to x_t is
//   g_t = [r_{t-1} - r_t + a k r_t] / (2 D dt),   r_{-1} = r_T = 0.
// Every coordinate is an independent time series; in the slice-major layout
// pos[t][c][n] the time neighbours of element e are e - s and e + s, s = dim*N.
// One pass reads each position once and writes each gradient once.
#include "pamd_internal.cuh"

namespace pamd {

template <typename R, bool GRAD>
__global__ void __launch_bounds__(kElemThreads)
    ho_action_kernel(const ElemBlock* __restrict__ blocks, const R* __restrict__ pos,
                     R* __restrict__ grad, double* __restrict__ partials, int slot0, R a, R ginv)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* xs = reinterpret_cast<R*>(smem_raw);
    __shared__ double red[kElemThreads / 32];

    const ElemBlock B = blocks[blockIdx.x];
    const R ak = a * (R)B.k;
    const R* __restrict__ X = pos + B.chain_base;
    const int s = B.s;
    const int lo = B.e0 - s;  // first staged element (may be negative: zero-filled)
    const int cnt = B.n + 2 * s;

    // Stage x[e0 - s, e0 + n + s) of this chain: coalesced, many loads in flight.
#pragma unroll 8
    for (int q = threadIdx.x; q < cnt; q += kElemThreads) {
        const int e = lo + q;
        xs[q] = (e >= 0 && e < B.chain_len) ? __ldg(X + e) : R(0);
    }
    __syncthreads();

    const int rend = B.chain_len - s;  // residuals exist for chain-local e < rend (t < T)
    R acc = R(0);
#pragma unroll 4
    for (int q = threadIdx.x; q < B.n; q += kElemThreads) {
        const int e = B.e0 + q;
        const R xm = xs[q], x0 = xs[q + s], xp = xs[q + 2 * s];
        const R rp = (e >= s) ? fma_r(ak, xm, x0 - xm) : R(0);
        const R r = (e < rend) ? fma_r(ak, x0, xp - x0) : R(0);
        if (GRAD) grad[B.chain_base + e] = fma_r(ak, r, rp - r) * ginv;
        acc = fma_r(r, r, acc);
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) partials[slot0 + blockIdx.x] = tot;
}

template <typename R>
cudaError_t launch_ho_action(const ElemBlock* blocks, int n_blocks, int max_s, const R* pos, R* grad,
                             double* partials, int slot0, double a, double ginv, bool with_grad,
                             cudaStream_t st)
{
    if (n_blocks <= 0) return cudaSuccess;
    const size_t smem = sizeof(R) * (size_t)(kElemChunk + 2 * max_s);
    if (with_grad) {
        auto k = ho_action_kernel<R, true>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_blocks, kElemThreads, smem, st>>>(blocks, pos, grad, partials, slot0, (R)a, (R)ginv);
    } else {
        auto k = ho_action_kernel<R, false>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_blocks, kElemThreads, smem, st>>>(blocks, pos, grad, partials, slot0, (R)a, (R)ginv);
    }
    return cudaGetLastError();
}

template cudaError_t launch_ho_action<float>(const ElemBlock*, int, int, const float*, float*,
                                             double*, int, double, double, bool, cudaStream_t);
template cudaError_t launch_ho_action<double>(const ElemBlock*, int, int, const double*, double*,
                                              double*, int, double, double, bool, cudaStream_t);

// ------------------------------------------------------------------ Euler-Maruyama (Eq. (2))
// One thread per (chain, coordinate), sequential in time:
//   x_{t+1} = x_t - a k x_t + sqrt(2 D dt) xi_t, stored in R and reused as stored.
template <typename R>
__global__ void ho_euler_kernel(R* __restrict__ pos, const R* __restrict__ noise, int s, int T,
                                int n_chains, long long sys_offset, int chain0, R ak, R sig,
                                uint64_t seed, uint64_t counter)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)n_chains * s) return;
    const int b = (int)(gid / s), kk = (int)(gid % s);
    const long long chain_len = (long long)(T + 1) * s;
    R* X = pos + sys_offset + b * chain_len;
    const R* Z = noise ? noise + sys_offset + b * chain_len : nullptr;
    R x = X[kk];
    for (int t = 0; t < T; ++t) {
        const long long e = (long long)(t + 1) * s + kk;
        R z;
        if (Z) {
            z = Z[e];
        } else {
            const float4 q = philox_normals4(seed, counter, kStreamEuler, (uint32_t)(chain0 + b),
                                             (uint32_t)(e >> 2));
            z = (R)pick4(q, (int)(e & 3));
        }
        x = x + fma_r(-ak, x, sig * z);
        X[e] = x;
    }
}

template <typename R>
cudaError_t launch_ho_euler(R* pos, const R* noise, int s, int T, int n_chains, long long sys_offset,
                            int chain0, double k, double a, double sig, uint64_t seed,
                            uint64_t counter, cudaStream_t st)
{
    const long long n = (long long)n_chains * s;
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const unsigned grid = (unsigned)((n + threads - 1) / threads);
    ho_euler_kernel<R><<<grid, threads, 0, st>>>(pos, noise, s, T, n_chains, sys_offset, chain0,
                                                 (R)(a * k), (R)sig, seed, counter);
    return cudaGetLastError();
}

template cudaError_t launch_ho_euler<float>(float*, const float*, int, int, int, long long, int,
                                            double, double, double, uint64_t, uint64_t,
                                            cudaStream_t);
template cudaError_t launch_ho_euler<double>(double*, const double*, int, int, int, long long, int,
                                             double, double, double, uint64_t, uint64_t,
                                             cudaStream_t);

}  // namespace pamd
