// probe.cu -- FP32 fused multiply-add throughput of this GPU, the denominator of
// the single-precision roofline of the Lennard-Jones kernels, and the FP64 rate
// that bounds the plain double-precision form.
//
// Every thread runs kChains independent dependent chains a <- a * b + c for
// `iters` iterations (scalar fma.rn.f32, or packed fma.rn.f32x2 where each
// instruction performs two).  With enough resident warps the chains keep the
// FMA pipes busy; the result is summed and stored so nothing is eliminated.
#include <cuda_runtime.h>

#include "pamd_internal.cuh"

namespace {

constexpr int kChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(1024) fma_probe_kernel(float* __restrict__ out, int iters, float b,
                                                         float c)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (PACKED) {
        float2 a[kChains];
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = make_float2(tid * 1e-7f + q, q * 0.5f);
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int q = 0; q < kChains; ++q) a[q] = __ffma2_rn(a[q], b2, c2);
        }
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kChains; ++q) s += a[q].x + a[q].y;
        out[tid] = s;
    } else {
        float a[kChains];
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = tid * 1e-7f + q;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int q = 0; q < kChains; ++q) a[q] = __fmaf_rn(a[q], b, c);
        }
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kChains; ++q) s += a[q];
        out[tid] = s;
    }
}

// The same in double precision (fma.rn.f64), for the plain FP64 form.
__global__ void __launch_bounds__(1024) fma64_probe_kernel(double* __restrict__ out, int iters,
                                                           double b, double c)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = tid * 1e-9 + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = __fma_rn(a[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    out[tid] = s;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int pamd_fp64_fma_probe(int blocks, int threads, int iters, double* out, double* flops,
                                   void* stream)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !out)
        return PAMD_ERR_ARG;
    if (!is_device_ptr(out)) return PAMD_ERR_ARG;
    fma64_probe_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, 0.999999999, 1e-9);
    if (cudaGetLastError() != cudaSuccess) return PAMD_ERR_CUDA;
    if (flops) *flops = 2.0 * kChains * (double)iters * (double)blocks * threads;
    return PAMD_OK;
}

extern "C" int pamd_fp32_fma_probe(int packed, int blocks, int threads, int iters, float* out,
                                   double* flops, void* stream)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !out)
        return PAMD_ERR_ARG;
    if (!is_device_ptr(out)) return PAMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // b slightly below 1 and c small keep every chain finite for any iteration count.
    if (packed)
        fma_probe_kernel<true><<<blocks, threads, 0, st>>>(out, iters, 0.999999f, 1e-6f);
    else
        fma_probe_kernel<false><<<blocks, threads, 0, st>>>(out, iters, 0.999999f, 1e-6f);
    if (cudaGetLastError() != cudaSuccess) return PAMD_ERR_CUDA;
    if (flops)
        *flops = 2.0 * (packed ? 2.0 : 1.0) * kChains * (double)iters * (double)blocks * threads;
    return PAMD_OK;
}
