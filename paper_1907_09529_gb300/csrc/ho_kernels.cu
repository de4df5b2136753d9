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
// One pass reads each position once and writes each gradient once.  On a time
// slab (see pamd_system) the halo step's residual is formed but not summed, and
// the halo slices' gradients are not written (ElemBlock::sum_lo, own_lo/own_hi).
#include "pamd_internal.cuh"

namespace pamd {

// SLAB: the blocks belong to a time slab (owned elements and the summed steps
// masked); whole paths take the form without the masks.
template <typename R, bool GRAD, bool SLAB>
__global__ void __launch_bounds__(kElemThreads)
    ho_action_kernel(const ElemBlock* __restrict__ blocks, const R* __restrict__ pos,
                     R* __restrict__ grad, double* __restrict__ partials, int slot0, R a, R ginv)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[kElemThreads / 32];

    const ElemBlock B = blocks[blockIdx.x];
    PAMD_ARR(R, xs, reinterpret_cast<R*>(smem_raw), B.n + 2 * B.s);
    const R ak = a * (R)B.k;
    const R* __restrict__ X = pos + B.chain_base;
    const int s = B.s;
    const int lo = B.e0 - s;  // first staged element (may be negative: zero-filled)
    const int cnt = B.n + 2 * s;

    // Stage x[e0 - s, e0 + n + s) of this chain: coalesced, many loads in flight.
#pragma unroll 8
    for (int q = threadIdx.x; q < cnt; q += kElemThreads) {
        const int e = lo + q;
        xs[q] = (e >= 0 && e < B.chain_len && PAMD_OK_IDX(e, B.chain_len)) ? __ldg(X + e) : R(0);
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
        if (GRAD && (!SLAB || (e >= B.own_lo && e < B.own_hi)) && PAMD_OK_IDX(e, B.chain_len))
            grad[B.chain_base + e] = fma_r(ak, r, rp - r) * ginv;
        if (!SLAB || e >= B.sum_lo) acc = fma_r(r, r, acc);
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) partials[slot0 + blockIdx.x] = tot;
}

template <typename R>
cudaError_t launch_ho_action(const ElemBlock* blocks, int n_blocks, int max_s, const R* pos, R* grad,
                             double* partials, int slot0, double a, double ginv, bool with_grad,
                             cudaStream_t st, bool slab)
{
    if (n_blocks <= 0) return cudaSuccess;
    const size_t smem = sizeof(R) * (size_t)(kElemChunk + 2 * max_s);
    auto k = with_grad ? (slab ? ho_action_kernel<R, true, true> : ho_action_kernel<R, true, false>)
                       : (slab ? ho_action_kernel<R, false, true> : ho_action_kernel<R, false, false>);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<n_blocks, kElemThreads, smem, st>>>(blocks, pos, grad, partials, slot0, (R)a, (R)ginv);
    return cudaGetLastError();
}

template cudaError_t launch_ho_action<float>(const ElemBlock*, int, int, const float*, float*,
                                             double*, int, double, double, bool, cudaStream_t, bool);
template cudaError_t launch_ho_action<double>(const ElemBlock*, int, int, const double*, double*,
                                              double*, int, double, double, bool, cudaStream_t, bool);

// ------------------------------------------------------------------ vectorised form (s <= 4)
// When a slice holds at most 4 elements (one particle in 1-3D, or a few in 1D),
// the time neighbours e - s and e + s of the 4 elements in an aligned float4
// all lie in the float4s just before and after it.  Each thread loads those
// three 16-byte vectors (the neighbours' loads hit L1), forms 4 gradients in
// registers and stores one float4: no shared-memory staging and no barrier
// before the final block sum.  The unaligned ends of a block (< 4 elements
// each) are done element by element.
template <int S, bool GRAD, bool SLAB>
__global__ void __launch_bounds__(kElemThreads)
    ho_vec_kernel(const ElemBlock* __restrict__ blocks, const float* __restrict__ pos,
                  float* __restrict__ grad, double* __restrict__ partials, int slot0, float a,
                  float ginv, long long sys_lo, long long sys_hi)
{
    __shared__ double red[kElemThreads / 32];
    const ElemBlock B = blocks[blockIdx.x];
    const float ak = a * (float)B.k;
    const long long base = B.chain_base;
    const long long glo = base + B.e0, ghi = glo + B.n;
    const long long gal = (glo + 3) & ~3LL, gah = ghi & ~3LL;
    const int rend = B.chain_len - S;
    float acc = 0.f;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long g = gal + 4LL * threadIdx.x; g < gah; g += 4LL * kElemThreads) {
        if (!PAMD_OK_IDX(g - base + 3, B.chain_len) || !PAMD_OK_IDX(g - base, B.chain_len)) continue;
        const float4 c = __ldg(reinterpret_cast<const float4*>(pos + g));
        const float4 p = (g - 4 >= sys_lo) ? __ldg(reinterpret_cast<const float4*>(pos + g - 4)) : z4;
        const float4 n = (g + 4 < sys_hi) ? __ldg(reinterpret_cast<const float4*>(pos + g + 4)) : z4;
        const float xx[12] = {p.x, p.y, p.z, p.w, c.x, c.y, c.z, c.w, n.x, n.y, n.z, n.w};
        float out[4];
        const int le0 = (int)(g - base);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int le = le0 + l;
            const float xm = xx[4 + l - S], x0 = xx[4 + l], xp = xx[4 + l + S];
            const float rp = (le >= S) ? fma_r(ak, xm, x0 - xm) : 0.f;
            const float r = (le < rend) ? fma_r(ak, x0, xp - x0) : 0.f;
            out[l] = fma_r(ak, r, rp - r) * ginv;
            if (!SLAB || le >= B.sum_lo) acc = fma_r(r, r, acc);
        }
        if (GRAD) {
            if (!SLAB || (le0 >= B.own_lo && le0 + 3 < B.own_hi)) {
                *reinterpret_cast<float4*>(grad + g) = make_float4(out[0], out[1], out[2], out[3]);
            } else {  // a vector holding time-slab halo elements
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (le0 + l >= B.own_lo && le0 + l < B.own_hi) grad[g + l] = out[l];
            }
        }
    }
    // unaligned ends: [glo, gal) and [gah, ghi) (at most 3 + 3 elements), or the
    // whole block (fewer than 8 elements) when it holds no aligned float4
    const bool body = gal < gah;
    const int nhead = (int)((body ? gal : ghi) - glo);
    const int ntail = body ? (int)(ghi - gah) : 0;
    if ((int)threadIdx.x < nhead + ntail) {
        const long long g = (int)threadIdx.x < nhead ? glo + threadIdx.x : gah + (threadIdx.x - nhead);
        const int le = (int)(g - base);
        const bool ok = PAMD_OK_IDX(le, B.chain_len);
        const float x0 = ok ? pos[g] : 0.f;
        const float xm = (le >= S && ok) ? pos[g - S] : 0.f;
        const float xp = (le < rend && ok) ? pos[g + S] : 0.f;
        const float rp = (le >= S) ? fma_r(ak, xm, x0 - xm) : 0.f;
        const float r = (le < rend) ? fma_r(ak, x0, xp - x0) : 0.f;
        if (GRAD && (!SLAB || (le >= B.own_lo && le < B.own_hi)) && ok) grad[g] = fma_r(ak, r, rp - r) * ginv;
        if (!SLAB || le >= B.sum_lo) acc = fma_r(r, r, acc);
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) partials[slot0 + blockIdx.x] = tot;
}

template <int S>
static cudaError_t launch_vec_s(const ElemBlock* blocks, int n_blocks, const float* pos, float* grad,
                                double* partials, int slot0, double a, double ginv, bool with_grad,
                                long long sys_lo, long long sys_hi, cudaStream_t st, bool slab)
{
    auto kern = with_grad ? (slab ? ho_vec_kernel<S, true, true> : ho_vec_kernel<S, true, false>)
                          : (slab ? ho_vec_kernel<S, false, true> : ho_vec_kernel<S, false, false>);
    kern<<<n_blocks, kElemThreads, 0, st>>>(blocks, pos, grad, partials, slot0, (float)a, (float)ginv,
                                            sys_lo, sys_hi);
    return cudaGetLastError();
}

cudaError_t launch_ho_action_vec(const ElemBlock* blocks, int n_blocks, int s, const float* pos,
                                 float* grad, double* partials, int slot0, double a, double ginv,
                                 bool with_grad, long long sys_lo, long long sys_hi, cudaStream_t st,
                                 bool slab)
{
    if (n_blocks <= 0) return cudaSuccess;
    switch (s) {
        case 1: return launch_vec_s<1>(blocks, n_blocks, pos, grad, partials, slot0, a, ginv, with_grad, sys_lo, sys_hi, st, slab);
        case 2: return launch_vec_s<2>(blocks, n_blocks, pos, grad, partials, slot0, a, ginv, with_grad, sys_lo, sys_hi, st, slab);
        case 3: return launch_vec_s<3>(blocks, n_blocks, pos, grad, partials, slot0, a, ginv, with_grad, sys_lo, sys_hi, st, slab);
        case 4: return launch_vec_s<4>(blocks, n_blocks, pos, grad, partials, slot0, a, ginv, with_grad, sys_lo, sys_hi, st, slab);
        default: return cudaErrorInvalidValue;
    }
}

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

PAMD_DEBUG_FETCHER(ho)

}  // namespace pamd
