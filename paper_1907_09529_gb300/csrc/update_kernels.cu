// update_kernels.cu -- deterministic per-chain reductions, the whole-path
// Metropolis-adjusted Langevin update that consumes the path gradient, and
// the random-number fill kernels.
//
// Update (tail slice x_0 fixed, Metropolis-Hastings acceptance as in the
// paper's path sampling, Sec. III; the trial moves along -grad S):
//   x'_t = x_t - h g_t + sqrt(2h) eta_t            (t >= 1),  x'_0 = x_0
//   log alpha = S(x) - S(x') - q_rev/(4h) + q_fwd/(4h)
//   q_fwd = sum_{t>=1} |x'_t - x_t + h g_t(x)|^2,  q_rev = sum_{t>=1} |x_t - x'_t + h g_t(x')|^2
// accepted iff log u < log alpha.  Element-wise terms are formed in the data
// precision from the stored values; every sum and the comparison are double.
#include <type_traits>

#include "pamd_internal.cuh"

namespace pamd {

// ------------------------------------------------------------------ finalize
// One warp per chain: fixed lane assignment and a fixed shuffle tree, so the
// result is bitwise reproducible.
__global__ void finalize_kernel(const double* __restrict__ partials, const ChainSlots* __restrict__ slots,
                                int n_chains, double scale, double* __restrict__ out,
                                int* __restrict__ err)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_chains) return;
    const ChainSlots cs = slots[warp];
    double s = 0.0;
    for (int q = cs.begin + lane; q < cs.end; q += 32) s += partials[q];
    s = warp_sum(s);
    if (lane == 0) {
        out[warp] = s * scale;
        if (err && !isfinite(s)) atomicExch(err, PAMD_ERR_NONFINITE);
    }
}

cudaError_t launch_finalize(const double* partials, const ChainSlots* slots, int n_chains,
                            double scale, double* out, cudaStream_t st, int* err)
{
    if (n_chains <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (n_chains * 32 + threads - 1) / threads;
    finalize_kernel<<<blocks, threads, 0, st>>>(partials, slots, n_chains, scale, out, err);
    return cudaGetLastError();
}

__global__ void set_status_kernel(int* err, int v) { *err = v; }

cudaError_t launch_set_status(int* err, int v, cudaStream_t st)
{
    set_status_kernel<<<1, 1, 0, st>>>(err, v);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ MALA pieces
__global__ void set_mala_params_kernel(MalaDev* md, uint64_t seed, uint64_t counter, double h)
{
    md->seed = seed;
    md->counter = counter;
    md->h = h;
}

cudaError_t launch_set_mala_params(MalaDev* md, uint64_t seed, uint64_t counter, double h,
                                   cudaStream_t st)
{
    set_mala_params_kernel<<<1, 1, 0, st>>>(md, seed, counter, h);
    return cudaGetLastError();
}

// Each thread owns groups of 4 consecutive chain-local elements.  The normal of
// element e is component (g & 3) of the Philox call for group g >> 2, g = e_glob + e
// its whole-path index (one call per group on whole paths).  Elements outside
// [s, own_hi) -- the fixed tail x_0 or a time slab's halo slices -- are copied.
// A group of four free elements of a single-precision whole path on a 16-byte
// aligned block moves as float4 loads and one float4 store, with the arithmetic of
// the elements in the same order as the element-wise loop (bitwise the same).
template <typename R, bool SLAB>
__global__ void __launch_bounds__(kElemThreads)
    mala_propose_kernel(const ElemBlock* __restrict__ blocks, const R* __restrict__ pos,
                        const R* __restrict__ grad, const R* __restrict__ noise, R* __restrict__ prop,
                        double* __restrict__ part_qf, const MalaDev* __restrict__ md, int update_index)
{
    __shared__ double red[kElemThreads / 32];
    const ElemBlock B = blocks[blockIdx.x];
    const double hd = md->h;
    const R h = (R)hd, s2h = (R)sqrt(2.0 * hd);
    const uint64_t seed = md->seed, counter = md->counter + (uint64_t)update_index;
    const long long base = B.chain_base;
    R acc = R(0);
    const int ng = (B.n + 3) >> 2;             // e0 is a multiple of 4
    const bool vec = std::is_same<R, float>::value && !SLAB && ((base + B.e0) & 3) == 0;
    for (int gq = threadIdx.x; gq < ng; gq += kElemThreads) {
        float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        long long zg = -1;                     // Philox group held in z4 (time slabs)
        if (!SLAB && !noise)                   // whole paths: the group of the 4 elements
            z4 = philox_normals4(seed, counter, kStreamMala, (uint32_t)B.chain,
                                 (uint32_t)((B.e0 >> 2) + gq));
        if constexpr (std::is_same<R, float>::value) {
            const int e4 = B.e0 + 4 * gq;
            if (vec && e4 + 3 < B.e0 + B.n && e4 >= B.s && PAMD_OK_IDX(e4 + 3, B.chain_len)) {
                const float4 x4 = __ldg(reinterpret_cast<const float4*>(pos + base + e4));
                const float4 g4 = __ldg(reinterpret_cast<const float4*>(grad + base + e4));
                if (noise) z4 = __ldg(reinterpret_cast<const float4*>(noise + base + e4));
                const float xs[4] = {x4.x, x4.y, x4.z, x4.w}, gs[4] = {g4.x, g4.y, g4.z, g4.w},
                            zs[4] = {z4.x, z4.y, z4.z, z4.w};
                float ps[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    ps[l] = xs[l] + fma_r(-h, gs[l], s2h * zs[l]);
                    const float f = fma_r(h, gs[l], ps[l] - xs[l]);
                    acc = fma_r(f, f, acc);
                }
                *reinterpret_cast<float4*>(prop + base + e4) = make_float4(ps[0], ps[1], ps[2], ps[3]);
                continue;
            }
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = B.e0 + 4 * gq + l;
            if (e >= B.e0 + B.n) break;
            if (!PAMD_OK_IDX(e, B.chain_len)) continue;
            const R x = pos[base + e];
            if (e < B.s || (SLAB && e >= B.own_hi)) {  // fixed tail x_0, or a time-slab halo
                prop[base + e] = x;
                continue;
            }
            const R g = grad[base + e];
            long long ge = e;
            if (SLAB) {
                ge = B.e_glob + e;
                if (!noise && (ge >> 2) != zg) {
                    zg = ge >> 2;
                    z4 = philox_normals4(seed, counter, kStreamMala, (uint32_t)B.chain, (uint32_t)zg);
                }
            }
            const R z = noise ? noise[base + e] : (R)pick4(z4, (int)(ge & 3));
            const R xp = x + fma_r(-h, g, s2h * z);
            prop[base + e] = xp;
            const R f = fma_r(h, g, xp - x);
            acc = fma_r(f, f, acc);
        }
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) part_qf[blockIdx.x] = tot;
}

template <typename R, bool SLAB>
__global__ void __launch_bounds__(kElemThreads)
    mala_reverse_kernel(const ElemBlock* __restrict__ blocks, const R* __restrict__ pos,
                        const R* __restrict__ prop, const R* __restrict__ grad_prop,
                        double* __restrict__ part_qr, const MalaDev* __restrict__ md)
{
    __shared__ double red[kElemThreads / 32];
    const ElemBlock B = blocks[blockIdx.x];
    const R h = (R)md->h;
    const long long base = B.chain_base;
    R acc = R(0);
#pragma unroll 4
    for (int q = threadIdx.x; q < B.n; q += kElemThreads) {
        const int e = B.e0 + q;
        if (e < B.s || (SLAB && e >= B.own_hi) || !PAMD_OK_IDX(e, B.chain_len)) continue;
        const R x = pos[base + e], xp = prop[base + e], gp = grad_prop[base + e];
        const R b = fma_r(h, gp, x - xp);
        acc = fma_r(b, b, acc);
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) part_qr[blockIdx.x] = tot;
}

// Chains [chain0, chain0 + n_chains); every array is indexed by the global chain.
__global__ void mala_accept_kernel(int chain0, int n_chains, const double* __restrict__ S,
                                   const double* __restrict__ S_prop, const double* __restrict__ qf,
                                   const double* __restrict__ qr, const double* __restrict__ log_u,
                                   const MalaDev* __restrict__ md, int update_index,
                                   int* __restrict__ accept_flag, int* __restrict__ n_accepted,
                                   double* __restrict__ log_alpha)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_chains) return;
    const int c = chain0 + q;
    const double h4 = 4.0 * md->h;
    const double la = (S[c] - S_prop[c]) - qr[c] / h4 + qf[c] / h4;
    double lu;
    if (log_u) {
        lu = log_u[c];
    } else {
        lu = log(philox_uniform53(md->seed, md->counter + (uint64_t)update_index, kStreamAccept,
                                  (uint32_t)c));
    }
    const int acc = (lu < la) ? 1 : 0;  // NaN log alpha never accepts
    accept_flag[c] = acc;
    if (n_accepted) n_accepted[c] += acc;
    if (log_alpha) log_alpha[c] = la;
}

template <typename R>
__global__ void __launch_bounds__(kElemThreads)
    mala_commit_kernel(const ElemBlock* __restrict__ blocks, R* __restrict__ pos, R* __restrict__ grad,
                       const R* __restrict__ prop, const R* __restrict__ grad_prop,
                       const int* __restrict__ accept_flag, double* __restrict__ S,
                       const double* __restrict__ S_prop)
{
    const ElemBlock B = blocks[blockIdx.x];
    if (!accept_flag[B.chain]) return;
    const long long base = B.chain_base;
#pragma unroll 4
    for (int q = threadIdx.x; q < B.n; q += kElemThreads) {
        const long long e = base + B.e0 + q;
        if (!PAMD_OK_IDX(B.e0 + q, B.chain_len)) continue;
        pos[e] = prop[e];
        grad[e] = grad_prop[e];
    }
    if (B.e0 == 0 && threadIdx.x == 0) S[B.chain] = S_prop[B.chain];
}

template <typename R>
cudaError_t launch_mala_propose(const ElemBlock* blocks, int n_blocks, const R* pos, const R* grad,
                                const R* noise, R* prop, double* part_qf, const MalaDev* md,
                                int update_index, cudaStream_t st, bool slab)
{
    if (n_blocks <= 0) return cudaSuccess;
    auto k = slab ? mala_propose_kernel<R, true> : mala_propose_kernel<R, false>;
    k<<<n_blocks, kElemThreads, 0, st>>>(blocks, pos, grad, noise, prop, part_qf, md, update_index);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mala_reverse(const ElemBlock* blocks, int n_blocks, const R* pos, const R* prop,
                                const R* grad_prop, double* part_qr, const MalaDev* md,
                                cudaStream_t st, bool slab)
{
    if (n_blocks <= 0) return cudaSuccess;
    auto k = slab ? mala_reverse_kernel<R, true> : mala_reverse_kernel<R, false>;
    k<<<n_blocks, kElemThreads, 0, st>>>(blocks, pos, prop, grad_prop, part_qr, md);
    return cudaGetLastError();
}

cudaError_t launch_mala_accept(int chain0, int n_chains, const double* S, const double* S_prop,
                               const double* qf, const double* qr, const double* log_u,
                               const MalaDev* md, int update_index, int* accept_flag,
                               int* n_accepted, double* log_alpha, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    const int threads = 128;
    mala_accept_kernel<<<(n_chains + threads - 1) / threads, threads, 0, st>>>(
        chain0, n_chains, S, S_prop, qf, qr, log_u, md, update_index, accept_flag, n_accepted,
        log_alpha);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mala_commit(const ElemBlock* blocks, int n_blocks, R* pos, R* grad, const R* prop,
                               const R* grad_prop, const int* accept_flag, double* S,
                               const double* S_prop, cudaStream_t st)
{
    if (n_blocks <= 0) return cudaSuccess;
    mala_commit_kernel<R><<<n_blocks, kElemThreads, 0, st>>>(blocks, pos, grad, prop, grad_prop,
                                                             accept_flag, S, S_prop);
    return cudaGetLastError();
}

#define PAMD_INST(R)                                                                               \
    template cudaError_t launch_mala_propose<R>(const ElemBlock*, int, const R*, const R*,         \
                                                const R*, R*, double*, const MalaDev*, int,        \
                                                cudaStream_t, bool);                               \
    template cudaError_t launch_mala_reverse<R>(const ElemBlock*, int, const R*, const R*,         \
                                                const R*, double*, const MalaDev*, cudaStream_t,   \
                                                bool);                                             \
    template cudaError_t launch_mala_commit<R>(const ElemBlock*, int, R*, R*, const R*, const R*,  \
                                               const int*, double*, const double*, cudaStream_t);
PAMD_INST(float)
PAMD_INST(double)
#undef PAMD_INST

// ------------------------------------------------------------------ RNG fills
__global__ void philox_fill_kernel(uint4 ctr, uint2 key, long long n, uint32_t* __restrict__ out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint4 c = ctr;
    const unsigned long long lo = (unsigned long long)c.x + (unsigned long long)q;
    c.x = (uint32_t)lo;
    const uint4 w = philox4x32_10(c, key);
    out[4 * q + 0] = w.x;
    out[4 * q + 1] = w.y;
    out[4 * q + 2] = w.z;
    out[4 * q + 3] = w.w;
}

cudaError_t launch_philox(uint4 ctr, uint2 key, long long n, uint32_t* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    philox_fill_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(ctr, key, n, out);
    return cudaGetLastError();
}

__global__ void normals_fill_kernel(uint64_t seed, uint64_t counter, uint32_t stream_id,
                                    uint32_t chain, long long e0, long long n, float* __restrict__ out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long e = e0 + q;
    const float4 z = philox_normals4(seed, counter, stream_id, chain, (uint32_t)(e >> 2));
    out[q] = pick4(z, (int)(e & 3));
}

cudaError_t launch_normals(uint64_t seed, uint64_t counter, uint32_t stream_id, uint32_t chain,
                           long long e0, long long n, float* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    normals_fill_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        seed, counter, stream_id, chain, e0, n, out);
    return cudaGetLastError();
}

PAMD_DEBUG_FETCHER(update)

}  // namespace pamd
