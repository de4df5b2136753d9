// pamd_internal.cuh -- device helpers and kernel argument blocks shared by the
// libpamd translation units.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdint>
#include <initializer_list>

#include "pamd.h"

namespace pamd {

// ------------------------------------------------------------------ debug bounds checks
// In a build with -DPAMD_DEBUG (libpamd_debug.so) the kernels' array accesses
// made through PAMD_ARR arrays, pamd::at() and the shared-memory accessors are
// bounds-checked: an index outside [0, n) records (source line, index, bound) in
// this translation unit's device record -- the first one wins -- and the access
// goes to a sink instead (a load then reads garbage, nothing outside the arrays
// is touched, nothing traps).  pamd_debug_status() collects and clears the
// records.  Without PAMD_DEBUG every check compiles away.
struct DebugRecord {
    int count;        // out-of-bounds accesses seen
    int site;         // source line of the first
    long long index;  // its index
    long long bound;  // the array's extent
};
#ifdef PAMD_DEBUG
static __device__ DebugRecord g_pamd_debug;
static __device__ __align__(32) unsigned char g_pamd_sink[64];

__device__ __forceinline__ bool debug_in_bounds(long long i, long long n, int site)
{
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_pamd_debug.count, 1) == 0) {
        g_pamd_debug.site = site;
        g_pamd_debug.index = i;
        g_pamd_debug.bound = n;
    }
    return false;
}

// An array with its extent: indexing checks the bound.
template <typename T>
struct ChkArr {
    T* p;
    long long n;
    int site;
    __device__ __forceinline__ T& operator[](long long i) const
    {
        return debug_in_bounds(i, n, site) ? p[i] : *reinterpret_cast<T*>(g_pamd_sink);
    }
    __device__ __forceinline__ ChkArr operator+(long long k) const { return ChkArr{p + k, n - k, site}; }
    __device__ __forceinline__ operator T*() const { return p; }
};
#define PAMD_ARR(T, name, ptr, extent) ::pamd::ChkArr<T> name{(ptr), (long long)(extent), __LINE__}
#define PAMD_AT(ptr, i, extent) \
    (*(::pamd::debug_in_bounds((long long)(i), (long long)(extent), __LINE__) ? &(ptr)[i] \
        : reinterpret_cast<decltype(&(ptr)[0])>(::pamd::g_pamd_sink)))

// Guard of one access: true when 0 <= i < n (a failure is recorded).
#define PAMD_OK_IDX(i, n) ::pamd::debug_in_bounds((long long)(i), (long long)(n), __LINE__)

// Host side: this translation unit's record, copied out and cleared.
static inline int debug_fetch_record(DebugRecord* out)
{
    if (cudaMemcpyFromSymbol(out, g_pamd_debug, sizeof(DebugRecord)) != cudaSuccess) return -1;
    const DebugRecord zero{0, 0, 0, 0};
    return cudaMemcpyToSymbol(g_pamd_debug, &zero, sizeof(DebugRecord)) == cudaSuccess ? 0 : -1;
}
#define PAMD_DEBUG_FETCHER(tu) \
    int debug_fetch_##tu(DebugRecord* out) { return debug_fetch_record(out); }
#else
#define PAMD_OK_IDX(i, n) true
#define PAMD_ARR(T, name, ptr, extent) T* name = (ptr)
#define PAMD_AT(ptr, i, extent) ((ptr)[i])
#define PAMD_DEBUG_FETCHER(tu) \
    int debug_fetch_##tu(DebugRecord* out) { *out = DebugRecord{0, 0, 0, 0}; return 0; }
#endif
// Per translation unit: its record (zeros in a build without the checks).
int debug_fetch_ho(DebugRecord* out);
int debug_fetch_lj(DebugRecord* out);
int debug_fetch_lj_paired(DebugRecord* out);
int debug_fetch_update(DebugRecord* out);
int debug_fetch_fragment(DebugRecord* out);

// ------------------------------------------------------------------ vector types
struct alignas(32) double4a {
    double x, y, z, w;
};
template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4a;
};
template <typename R>
using vec4_t = typename Vec4<R>::type;

template <typename R>
__device__ __forceinline__ vec4_t<R> make4(R x, R y, R z)
{
    vec4_t<R> v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = R(0);
    return v;
}

// Round-to-nearest-integer and fused multiply-add in the element type.
__device__ __forceinline__ float rint_r(float v) { return rintf(v); }
__device__ __forceinline__ double rint_r(double v) { return rint(v); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_r(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_r(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_r(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_r(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_r(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_r(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_r(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_r(double v) { return rsqrt(v); }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds; each round multiplies words 0 and 2 by two odd 32-bit
// constants, mixes the high halves with words 1/3 and the round key; the key
// is advanced by two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Four standard normals for element group `group` (elements 4*group..4*group+3)
// of one chain's noise stream: 24-bit uniforms, Box-Muller in single precision.
__device__ __forceinline__ float4 philox_normals4(uint64_t seed, uint64_t counter, uint32_t stream,
                                                  uint32_t chain, uint32_t group)
{
    const uint4 ctr = make_uint4(group, chain, (uint32_t)counter,
                                 (uint32_t)((counter >> 32) & 0xFFFFu) | (stream << 16));
    const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float two_m24 = 5.9604644775390625e-8f;  // 2^-24
    const float u0 = (float)((w.x >> 8) + 1u) * two_m24;
    const float v1 = (float)(w.y >> 8) * two_m24;
    const float u2 = (float)((w.z >> 8) + 1u) * two_m24;
    const float v3 = (float)(w.w >> 8) * two_m24;
    const float ra = sqrtf(-2.0f * logf(u0));
    const float rb = sqrtf(-2.0f * logf(u2));
    float sa, ca, sb, cb;
    sincospif(2.0f * v1, &sa, &ca);
    sincospif(2.0f * v3, &sb, &cb);
    return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

__device__ __forceinline__ float pick4(const float4& v, int lane)
{
    return lane == 0 ? v.x : lane == 1 ? v.y : lane == 2 ? v.z : v.w;
}

// Uniform in (0,1] with 53 bits (words 0 and 1), for the per-chain accept test.
__device__ __forceinline__ double philox_uniform53(uint64_t seed, uint64_t counter, uint32_t stream,
                                                   uint32_t chain)
{
    const uint4 ctr = make_uint4(0u, chain, (uint32_t)counter,
                                 (uint32_t)((counter >> 32) & 0xFFFFu) | (stream << 16));
    const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint64_t m = (uint64_t)(w.x >> 5) * 67108864ull + (uint64_t)(w.y >> 6);
    return ((double)m + 1.0) * 1.1102230246251565e-16;  // 2^-53
}

enum : uint32_t {
    kStreamEuler = 0,
    kStreamMala = 1,
    kStreamAccept = 2,
    kStreamFragCut = 3,
    kStreamFragTrial = 4,
    kStreamFragAccept = 5,
    kStreamRegenerate = 6
};

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree); result valid in thread 0.
// `scratch` needs blockDim.x/32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* scratch)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        for (int q = lane; q < nw; q += 32) s += scratch[q];
        s = warp_sum(s);
    }
    return s;
}

// A device buffer whose address is not 16-byte aligned: the element kernels read
// and write whole 16-byte units, so such a buffer is refused (PAMD_ERR_ARG) before
// anything is launched.  Host buffers are staged into the library's own aligned
// workspace and pass.  Asks the driver only about a misaligned address.
inline bool misaligned_device_buffer(const void* p)
{
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u) == 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline bool any_misaligned(std::initializer_list<const void*> ps)
{
    for (const void* p : ps)
        if (misaligned_device_buffer(p)) return true;
    return false;
}

// ------------------------------------------------------------------ work descriptors
// A contiguous run of elements of one chain (element-wise passes).
struct ElemBlock {
    long long chain_base;  // element offset of the chain's slice 0 in the buffer
    long long e_glob;      // whole-path index of chain-local element 0 (time slabs; else 0)
    int e0;                // first chain-local element handled by this block
    int n;                 // number of elements
    int s;                 // elements per slice (dim * N)
    int chain_len;         // (T+1) * s
    int chain;             // global chain index
    int sys;               // system index
    int own_lo, own_hi;    // owned chain-local elements (gradient written, proposed)
    int sum_lo;            // first element whose step counts in S (halo step excluded)
    double k;              // harmonic constant (harmonic systems)
};

constexpr int kElemThreads = 256;
constexpr int kElemChunk = 4096;  // elements per ElemBlock

// Slot ranges of one chain in a partial-sum array.
struct ChainSlots {
    int begin, end;
};

// ------------------------------------------------------------------ launchers
// Harmonic action (+ gradient) over element blocks.  Writes one partial
// sum of |r|^2 per block into partials[slot0 + block].
// slab: the blocks belong to a time slab (ElemBlock's owned range and summed
// steps applied); false for whole paths.
template <typename R>
cudaError_t launch_ho_action(const ElemBlock* blocks, int n_blocks, int max_s, const R* pos, R* grad,
                             double* partials, int slot0, double a, double ginv, bool with_grad,
                             cudaStream_t st, bool slab);

// Single-precision form for slices of s <= 4 elements: aligned float4 loads and
// stores, neighbours from registers.  The blocks must all belong to one system
// whose elements span [sys_lo, sys_hi) of the buffer (reads stay inside it).
cudaError_t launch_ho_action_vec(const ElemBlock* blocks, int n_blocks, int s, const float* pos,
                                 float* grad, double* partials, int slot0, double a, double ginv,
                                 bool with_grad, long long sys_lo, long long sys_hi, cudaStream_t st,
                                 bool slab);

struct LJConst {
    double L, rc, eps, sigma, a, ginv, skin;
};

// Per-system constants of the LJ kernels in the element type.
template <typename R>
struct LJK {
    R L, iL, rc2, rl2, hs2;  // box, 1/box, rc^2, list radius^2, (skin/2)^2
    R rcm;                   // rc plus a margin that covers rounding in window lists
    R c1, c2, c3, duc;       // 24 eps sigma^6, 2 sigma^6, 26 sigma^6, u'(rc)
    R a, ginv, sig_em;       // beta D dt, 1/(2 D dt), sqrt(2 D dt)
    // Folded coefficients of the paired kernel, with ir8 = r^-8, ir6 = r^-6:
    //   -U'(r)/r               = ir8 (c12 ir6 + nc1) + duc / r
    //   -(U''(r) - U'(r)/r)/r^2 = [ir8 (c8 + nc23 ir6) - duc / r] / r^2
    R c12, nc1, c8, nc23;    // c1 c2, -c1, 8 c1, -c1 (c2 + c3)
    R hb;                    // half the box less a rounding allowance: one image shift
                             // serves a window when rc + 4 max(delta) <= hb
};

template <typename R>
inline LJK<R> make_lj_consts(const LJConst& c, double sig_em)
{
    LJK<R> k;
    const double rl = c.rc + c.skin;
    const double s6 = c.sigma * c.sigma * c.sigma * c.sigma * c.sigma * c.sigma;
    const double src = c.sigma / c.rc;
    const double q6 = src * src * src * src * src * src;
    // u'(rc) = 4 eps (-12 (s/rc)^12 + 6 (s/rc)^6) / rc
    const double duc = 4.0 * c.eps * (-12.0 * q6 * q6 + 6.0 * q6) / c.rc;
    if (sizeof(R) == sizeof(float)) {
        // The single-precision cutoff rule: L, 1/L and rc^2 rounded to float.
        const float Lf = (float)c.L;
        const float rcf = (float)c.rc;
        k.L = (R)Lf;
        k.iL = (R)(1.0f / Lf);
        k.rc2 = (R)(rcf * rcf);
    } else {
        k.L = (R)c.L;
        k.iL = (R)(1.0 / c.L);
        k.rc2 = (R)(c.rc * c.rc);
    }
    k.rl2 = (R)(rl * rl);
    k.rcm = (R)(c.rc * (1.0 + 1.0e-6) + 1.0e-5);
    k.hs2 = (R)(0.25 * c.skin * c.skin);
    k.c1 = (R)(24.0 * c.eps * s6);
    k.c2 = (R)(2.0 * s6);
    k.c3 = (R)(26.0 * s6);
    k.duc = (R)duc;
    k.c12 = (R)(24.0 * c.eps * s6 * 2.0 * s6);
    k.nc1 = (R)(-24.0 * c.eps * s6);
    k.c8 = (R)(8.0 * 24.0 * c.eps * s6);
    k.nc23 = (R)(-24.0 * c.eps * s6 * 28.0 * s6);
    k.hb = (R)(0.5 * c.L * (1.0 - 1.0e-5) - 1.0e-5);
    k.a = (R)c.a;
    k.ginv = (R)c.ginv;
    k.sig_em = (R)sig_em;
    return k;
}

// One LJ system as the kernels see it.
template <typename R>
struct LJSysDev {
    long long off;        // element offset of chain 0
    long long chain_len;  // (T+1) * 3N
    int N, T;
    int tpp, lg_tpp;      // threads per particle (power of two) and its log2
    int cap;              // neighbour-list capacity per thread
    int window;           // steps per neighbour-list window (paired kernel)
    int outer_cap;        // outer-list capacity per thread (paired kernel, global memory)
    int shared_shift;     // paired kernel: windows may use one image shift per list entry
    int write_nose;       // the last slice is owned (not a time-slab halo): write its gradient
    int chain0;           // global index of chain 0
    long long hs_off;     // hard-sphere path bias: this system's slices in the radii array
    LJK<R> k;
};

// A work item: steps [t0, t1) of one chain of one system; its |r|^2 sum goes
// to partials[slot].
struct LJItem {
    int sys, chain, t0, t1, slot;
};

// Shared memory of the LJ action kernel: three slices of nmax particles and a
// list of cap_lane entries for each of NT threads.
size_t lj_smem_bytes(int nmax, int NT, int cap_lane, bool fp64);

template <typename R>
int lj_blocks_per_sm(int NT, size_t smem, bool with_grad);

template <typename R>
cudaError_t launch_lj_items(const LJItem* items, int n_items, const void* sys_table, int nmax,
                            const R* pos, R* grad, double* partials, int* counter, int NT,
                            size_t smem, int grid, bool with_grad, cudaStream_t st,
                            const R* hs2 = nullptr, int* overlap = nullptr);

// Hard-sphere path bias: squared radii from the caller's radii (<= 0: none, -1);
// the all-pairs check of slice t of every chain of one system (host copy of its
// LJSysDev row); S = +inf where a chain's overlap flag is set.
template <typename R>
cudaError_t launch_hs_square(const double* sigma, R* hs2, long long n, cudaStream_t st);
template <typename R>
cudaError_t launch_lj_hs_slice(const R* pos, const void* sys_entry_host, int n_chains, int t,
                               const R* hs2t, int* overlap, cudaStream_t st);
cudaError_t launch_hs_fixup(double* S, const int* overlap, int n, cudaStream_t st);

// Single-precision action (+ adjoint) with two consecutive steps per thread and
// packed f32x2 pair arithmetic (lj_paired.cu), for systems of N <= NT <= 1024.
// Shared memory: positions and residuals of two slices (48 bytes per particle
// slot, 512 or 1024 slots) and cap_lane list entries per thread, two to a word.
// pipe: the gradient launch uses the pipelined form (blocks of <= 512 threads).
size_t lj_paired_smem_bytes(int NT, int cap_lane, bool pipe);
int lj_paired_blocks_per_sm(int NT, size_t smem, bool with_grad, bool pipe);
// outer: per-CTA outer lists, outer_words 32-bit words for each of grid CTAs.
// hs2 (NULL: no bias): squared hard-sphere radii per slice of every LJ system
// (LJSysDev::hs_off); overlap: per global chain, set to 1 where a pair lies within
// its slice's radius at a slice whose force the launch evaluates.
cudaError_t launch_lj_paired(const LJItem* items, int n_items, const void* sys_table,
                             const float* pos, float* grad, double* partials, int* counter, int NT,
                             size_t smem, int grid, bool with_grad, bool pipe, uint32_t* outer,
                             long long outer_words, cudaStream_t st, const float* hs2 = nullptr,
                             int* overlap = nullptr);

cudaError_t launch_lj_pair_counts(const float* pos, long long* counts, int N, int T, int n_chains,
                                  long long sys_offset, double L, double rc, cudaStream_t st);

// Euler-Maruyama reference paths.
template <typename R>
cudaError_t launch_ho_euler(R* pos, const R* noise, int s, int T, int n_chains, long long sys_offset,
                            int chain0, double k, double a, double sig, uint64_t seed,
                            uint64_t counter, cudaStream_t st);
template <typename R>
cudaError_t launch_lj_euler(R* pos, const R* noise, const void* sys_entry_host, int NT, size_t smem,
                            int n_chains, int chain0, uint64_t seed, uint64_t counter,
                            cudaStream_t st);

// Deterministic per-chain sums of partials: out[c] = scale * sum(partials[slots[c]]);
// a non-finite sum sets *err (if given) to PAMD_ERR_NONFINITE.
cudaError_t launch_finalize(const double* partials, const ChainSlots* slots, int n_chains,
                            double scale, double* out, cudaStream_t st, int* err = nullptr);

// Sets a device status word (host-side fault injection of non-finite actions).
cudaError_t launch_set_status(int* err, int v, cudaStream_t st);

// MALA update pieces (element-wise over all systems' blocks).
struct MalaDev {
    uint64_t seed;
    uint64_t counter;
    double h;
};
// slab: some block belongs to a time slab (halo elements copied / skipped, noise
// indexed from the whole path's slice 0); false for whole paths.
template <typename R>
cudaError_t launch_mala_propose(const ElemBlock* blocks, int n_blocks, const R* pos, const R* grad,
                                const R* noise, R* prop, double* part_qf, const MalaDev* md,
                                int update_index, cudaStream_t st, bool slab);
template <typename R>
cudaError_t launch_mala_reverse(const ElemBlock* blocks, int n_blocks, const R* pos, const R* prop,
                                const R* grad_prop, double* part_qr, const MalaDev* md,
                                cudaStream_t st, bool slab);
// Accept test for chains [chain0, chain0 + n_chains) (arrays indexed by global chain).
cudaError_t launch_mala_accept(int chain0, int n_chains, const double* S, const double* S_prop,
                               const double* qf, const double* qr, const double* log_u,
                               const MalaDev* md, int update_index, int* accept_flag,
                               int* n_accepted, double* log_alpha, cudaStream_t st);
template <typename R>
cudaError_t launch_mala_commit(const ElemBlock* blocks, int n_blocks, R* pos, R* grad, const R* prop,
                               const R* grad_prop, const int* accept_flag, double* S,
                               const double* S_prop, cudaStream_t st);
cudaError_t launch_set_mala_params(MalaDev* md, uint64_t seed, uint64_t counter, double h,
                                   cudaStream_t st);

cudaError_t launch_philox(uint4 ctr, uint2 key, long long n, uint32_t* out, cudaStream_t st);

cudaError_t launch_normals(uint64_t seed, uint64_t counter, uint32_t stream_id, uint32_t chain,
                           long long e0, long long n, float* out, cudaStream_t st);

}  // namespace pamd
