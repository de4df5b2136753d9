// noalloc.cu -- pamd_ho_action_grad_noalloc: the harmonic action + gradient
// without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a process
// whose allocator has already reserved the GPU's memory for itself (so a
// cudaMalloc outside it fails or fragments that pool), or a long-running
// service that forbids allocation after start-up because cudaMalloc and
// cudaFree synchronise the device and can fail under memory pressure.  This
// entry point needs nothing but the caller's buffers: the only scratch it uses
// -- one double per 4096-element block for the block sums of |r|^2 -- lives in
// the file-scope array below, which every GPU that loads the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "pamd_internal.cuh"

namespace {

constexpr int kNoallocMaxBlocks = PAMD_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (host code may not
// use the symbol itself as an address).  Outside stream capture the address is
// looked up on every call, so a device reset (which unloads the module) is
// followed by the new address; while `st` is capturing, the address cached by
// an earlier uncaptured call on this device is used.
int noalloc_scratch(cudaStream_t st, double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PAMD_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return PAMD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return PAMD_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    if (!g_noalloc_ptr[dev]) return PAMD_ERR_CUDA;  // first call on this device inside a capture
    *out = g_noalloc_ptr[dev];
    return PAMD_OK;
}

// Same arithmetic as the planned harmonic kernel; the block's chain and chunk
// come from the grid (x: chunk of 4096 elements, y: chain) instead of a
// descriptor table, and its |r|^2 partial goes to partials[slot0 + y*gridDim.x + x].
template <typename R>
__global__ void __launch_bounds__(pamd::kElemThreads)
    ho_noalloc_kernel(const R* __restrict__ pos, R* __restrict__ grad, double* __restrict__ partials,
                      int slot0, long long sys_off, int s, int chain_len, R ak, R ginv)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* xs = reinterpret_cast<R*>(smem_raw);
    __shared__ double red[pamd::kElemThreads / 32];
    const long long base = sys_off + (long long)blockIdx.y * chain_len;
    const int e0 = blockIdx.x * pamd::kElemChunk;
    const int n = min(pamd::kElemChunk, chain_len - e0);
    const R* __restrict__ X = pos + base;
    const int lo = e0 - s, cnt = n + 2 * s;
#pragma unroll 8
    for (int q = threadIdx.x; q < cnt; q += pamd::kElemThreads) {
        const int e = lo + q;
        xs[q] = (e >= 0 && e < chain_len) ? __ldg(X + e) : R(0);
    }
    __syncthreads();
    const int rend = chain_len - s;
    R acc = R(0);
#pragma unroll 4
    for (int q = threadIdx.x; q < n; q += pamd::kElemThreads) {
        const int e = e0 + q;
        const R xm = xs[q], x0 = xs[q + s], xp = xs[q + 2 * s];
        const R rp = (e >= s) ? pamd::fma_r(ak, xm, x0 - xm) : R(0);
        const R r = (e < rend) ? pamd::fma_r(ak, x0, xp - x0) : R(0);
        grad[base + e] = pamd::fma_r(ak, r, rp - r) * ginv;
        acc = pamd::fma_r(r, r, acc);
    }
    const double tot = pamd::block_sum((double)acc, red);
    if (threadIdx.x == 0) partials[slot0 + blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// One warp per chain sums its chunks' partials in a fixed order.
__global__ void ho_noalloc_finalize(const double* __restrict__ partials, int slot0, int chunks,
                                    int n_chains, int chain0, double scale, double* __restrict__ S)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n_chains) return;
    double v = 0.0;
    for (int q = lane; q < chunks; q += 32) v += partials[slot0 + c * chunks + q];
    v = pamd::warp_sum(v);
    if (lane == 0) S[chain0 + c] = v * scale;
}

// Device (or managed) memory of the current device.
bool device_ptr(const void* p)
{
    cudaPointerAttributes a;
    int dev = -1;
    if (!p || cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <typename R>
int run_noalloc(const pamd_problem* p, const R* pos, double* S, R* grad, double* scratch,
                cudaStream_t st)
{
    const double a = p->beta * p->D * p->dt, ginv = 1.0 / (2.0 * p->D * p->dt);
    // Shared-memory attribute for the largest system, set before anything is
    // enqueued, so that a failure leaves every output untouched.
    size_t smem_max = 0;
    for (int q = 0; q < p->n_systems; ++q)
        smem_max = std::max(smem_max, sizeof(R) * (size_t)(pamd::kElemChunk +
                                                           2 * p->systems[q].dim * p->systems[q].n_particles));
    auto kern = ho_noalloc_kernel<R>;
    if (smem_max > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) !=
            cudaSuccess)
        return PAMD_ERR_CUDA;
    int slot = 0, chain0 = 0;
    for (int q = 0; q < p->n_systems; ++q) {
        const pamd_system& s = p->systems[q];
        const int sz = s.dim * s.n_particles;
        const int chain_len = (s.n_steps + 1) * sz;
        const int chunks = (chain_len + pamd::kElemChunk - 1) / pamd::kElemChunk;
        const size_t smem = sizeof(R) * (size_t)(pamd::kElemChunk + 2 * sz);
        kern<<<dim3(chunks, s.n_chains), pamd::kElemThreads, smem, st>>>(
            pos, grad, scratch, slot, s.pos_offset, sz, chain_len, (R)(a * s.pot.k), (R)ginv);
        if (cudaGetLastError() != cudaSuccess) return PAMD_ERR_CUDA;
        const int threads = 256, blocks = (s.n_chains * 32 + threads - 1) / threads;
        ho_noalloc_finalize<<<blocks, threads, 0, st>>>(scratch, slot, chunks, s.n_chains, chain0,
                                                        1.0 / (4.0 * p->D * p->dt), S);
        if (cudaGetLastError() != cudaSuccess) return PAMD_ERR_CUDA;
        slot += chunks * s.n_chains;
        chain0 += s.n_chains;
    }
    return PAMD_OK;
}

}  // namespace

extern "C" int pamd_ho_action_grad_noalloc(const pamd_problem* prob, const void* pos, double* S,
                                           void* grad, void* stream)
{
    if (pamd::any_misaligned({pos, grad})) return PAMD_ERR_ARG;
    if (!prob || !prob->systems || prob->n_systems <= 0 || !pos || !S || !grad) return PAMD_ERR_ARG;
    if (prob->precision != PAMD_FP32 && prob->precision != PAMD_FP64) return PAMD_ERR_ARG;
    if (!(prob->D > 0) || !(prob->dt > 0) || !(prob->beta > 0)) return PAMD_ERR_ARG;
    if (prob->flags & ~PAMD_FLAG_ONE_CHAIN_PER_LAUNCH) return PAMD_ERR_UNSUPPORTED;  // Eq. (3) only
    long long blocks = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        if (s.pot.kind != PAMD_HARMONIC || s.n_particles < 1 || s.n_steps < 1 || s.dim < 1 ||
            s.dim > 3 || s.n_chains < 1 || s.pos_offset < 0)
            return PAMD_ERR_ARG;
        if (s.dim * s.n_particles > 8192) return PAMD_ERR_UNSUPPORTED;
        if (s.n_chains > 65535) return PAMD_ERR_UNSUPPORTED;  // one grid row per chain
        if (s.first_slice || s.halo_lo || s.halo_hi) return PAMD_ERR_UNSUPPORTED;  // whole paths
        const long long chain_len = (long long)(s.n_steps + 1) * s.dim * s.n_particles;
        if (chain_len >= (1LL << 31)) return PAMD_ERR_UNSUPPORTED;
        blocks += (long long)s.n_chains * ((chain_len + pamd::kElemChunk - 1) / pamd::kElemChunk);
    }
    if (blocks > kNoallocMaxBlocks) return PAMD_ERR_UNSUPPORTED;  // scratch array too small
    if (!device_ptr(pos) || !device_ptr(S) || !device_ptr(grad)) return PAMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* scratch = nullptr;
    int rc = noalloc_scratch(st, &scratch);
    if (rc) return rc;
    if (prob->precision == PAMD_FP64)
        return run_noalloc<double>(prob, (const double*)pos, S, (double*)grad, scratch, st);
    return run_noalloc<float>(prob, (const float*)pos, S, (float*)grad, scratch, st);
}
