// fragment_kernels.cu -- multilevel sliding-and-sampling Monte Carlo on harmonic
// paths (paper Sec. III, Fig. 5), with free-particle trial paths.
//
// One MC step of a chain: a level l in [l_min, l_max] and an offset o in
// [0, 2^l) cut the path into fragments whose shared endpoints sit at 0 and at
// o + k 2^l (0 < . < T); the nose fragment ends at T and moves its end point.
// Every fragment [a, b] is updated independently by Metropolis-Hastings with a
// trial from the free particle (V = 0, same D and dt).  From the walk
// W_t = sig (z_{a+1} + ... + z_t), sig = sqrt(2 D dt):
//     nose:    x'_t = x_a + W_t
//     bridge:  x'_t = x_a + s (x_b - x_a) + (W_t - s W_b),  s = (t - a)/(b - a).
// The trial density is exp(-S0), S0 = sum |x_{t+1} - x_t|^2/(4 D dt), so
//     log alpha = -(S(X') - S(X)) + (S0(X') - S0(X))
// over the fragment's own steps; each residual belongs to exactly one fragment,
// so all fragments of all chains are decided in parallel.
//
// The harmonic step action is S_t = cS |x_{t+1} - x_t + g x_t|^2 (g, cS from the
// host: Eq. (3), or the oscillator's exact transition density), and the trial
// action S0 has its own scale c0 = 1/(4 D dt).
//
// fragment_line_kernel (one-line paths, M = 1) and fragment_block_kernel (any
// M <= 32): one CTA per chain with the chain's path X and the walk W staged in
// shared memory.  The walks are a segmented prefix sum (warp shuffles along the
// lines, carries across warp pieces), the per-fragment action differences a
// segmented scan with one segment per fragment, and accepted fragments are
// written back with coalesced stores.  HBM traffic: the path is read once and
// accepted interiors written once.
//
// fragment_thread_kernel: the fallback for chains too large for shared memory,
// one thread per fragment walking it three times (W_b; trial and action
// differences; write-back on acceptance).
//
// Precision.  GB300 runs FP64 at a small fraction of the FP32 rate and spends a
// whole warp slot per FP64 instruction however few lanes are active, so FP32
// paths do no per-element work in double.  A fragment's log alpha is summed as
// per-step differences (r'-r)(r'+r) and (dy-dx)(dy+dx) -- never as S' - S of
// two large sums, so nothing cancels -- over at most 2^l_max steps, in FP32 in a
// fixed order (the rounding of the FP32 terms themselves is the larger error);
// the accept test is decided in double whenever the FP32 margin cannot.
#include <algorithm>

#include "fragment.cuh"

namespace pamd {

struct FragSys {
    long long off;   // element offset of chain 0
    int T, M;        // steps, elements per slice
    int chain0;      // global index of chain 0
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

// Fragments of one chain at level l, offset o: f = 0 is [0, first], then
// [first + (f-1) len, first + f len], the last (the nose) ends at T.
struct FragGeom {
    int T, l, first, nfrag;
    __device__ __forceinline__ FragGeom(int T_, int l_, int o) : T(T_), l(l_)
    {
        const int len = 1 << l;
        first = o > 0 ? o : len;
        nfrag = 1 + (first < T ? ((T - 1 - first) >> l) + 1 : 0);
    }
    // fragment holding the step t-1 -> t (1 <= t <= T)
    __device__ __forceinline__ int of_step(int t) const
    {
        return (t - 1 < first) ? 0 : 1 + ((t - 1 - first) >> l);
    }
    __device__ __forceinline__ int a(int f) const { return f == 0 ? 0 : first + ((f - 1) << l); }
    __device__ __forceinline__ int b(int f) const { return f == nfrag - 1 ? T : first + (f << l); }
};

// Metropolis-Hastings test of fragment f with the fragment sums s = sum r'^2 - r^2
// and s0 = sum dy^2 - dx^2:  log u < log alpha = s0 c0 - s cS, with u given as
// log u or the 53-bit uniform (mant + 1) 2^-53 of Philox stream 5.  For FP32
// paths the test is first made in FP32 with the top 24 bits of u; only when
// the two sides lie within a bound of the FP32 errors (|log u - log u24| <=
// 2^-23/u24, rounding of la and of logf) is it repeated in double.  The
// decision always equals the double one.
template <typename R>
__device__ __forceinline__ bool frag_accept(R s, R s0, double cS, float cSf, double c0, float c0f,
                                            const double* log_u, int fstride, int c, int f,
                                            uint64_t seed, uint64_t counter)
{
    if (log_u) return log_u[(long long)c * fstride + f] < (double)s0 * c0 - (double)s * cS;
    const uint4 ctr = make_uint4((uint32_t)f, (uint32_t)c, (uint32_t)counter,
                                 (uint32_t)((counter >> 32) & 0xFFFFu) | (kStreamFragAccept << 16));
    const uint4 w = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    if (sizeof(R) == 4 && (w.x >> 8) != 0u) {
        const float sh = (float)s, s0h = (float)s0;
        const float laf = s0h * c0f - sh * cSf;
        const float u24 = (float)((w.x >> 8) + 1u) * 5.9604644775390625e-8f;
        const float lf = logf(u24);
        const float margin = 1e-5f * (1.0f + fabsf(sh) * cSf + fabsf(s0h) * c0f + fabsf(lf)) +
                             2.384185791015625e-7f / u24;  // 2^-22 / u24
        if (fabsf(laf - lf) > margin) return lf < laf;
    }
    const uint64_t mant = (uint64_t)(w.x >> 5) * 67108864ull + (uint64_t)(w.y >> 6);
    const double u = ((double)mant + 1.0) * 1.1102230246251565e-16;
    return log(u) < (double)s0 * c0 - (double)s * cS;
}

constexpr int kFragMaxThreads = 256;

// Exact float of a small non-negative int (n < 2^23) without a conversion
// instruction: 2^23 + n has n in its mantissa.
__device__ __forceinline__ float small_int_to_float(int n)
{
    return __int_as_float(0x4B000000 | n) - 8388608.0f;
}
template <typename R>
__device__ __forceinline__ R small_int_to_r(int n)
{
    return (R)small_int_to_float(n);
}

// Slice index and line of element e of a chain ([T+1][M] layout): M == 1 at
// compile time, else floor(e / M) = umulhi(e, ceil(2^32 / M)), exact for
// e < 2^32 / M (a chain in shared memory holds far fewer elements).
template <bool M1>
struct LineDiv {
    uint32_t inv;
    int M;
    __device__ __forceinline__ explicit LineDiv(int M_) : M(M_)
    {
        inv = M1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)M_ - 1) / (uint64_t)M_);
    }
    __device__ __forceinline__ int slice(int e) const
    {
        return M1 ? e : (int)__umulhi((uint32_t)e, inv);
    }
};

// Shared memory of fragment_block_kernel, in bytes.
template <typename R>
__host__ __device__ inline size_t frag_block_smem(int T, int M, int nfrag_max, int nwarps)
{
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t E = (size_t)(T + 1) * M;
    return up16(2 * sizeof(R) * nfrag_max)            // fragment sums s, s0
           + 2 * up16(sizeof(R) * E)                   // X, W
           + up16(sizeof(R) * (size_t)nfrag_max * M)   // W_b per fragment and line
           + up16(sizeof(R) * (size_t)nwarps * (M + 2))  // piece tails
           + up16(sizeof(int) * ((size_t)nfrag_max + 2));  // accept flags, counts
}

template <typename R, bool M1>
__global__ void __launch_bounds__(kFragMaxThreads)
    fragment_block_kernel(R* __restrict__ pos, const FragSys S, int l_min, int l_max, uint64_t seed,
                          uint64_t counter, const int* __restrict__ levels,
                          const int* __restrict__ offsets, const R* __restrict__ noise,
                          const double* __restrict__ log_u, int fstride, int nfrag_max, R ak, R sig,
                          double cS, float cSf, double c0, float c0f, int* __restrict__ n_accepted,
                          int* __restrict__ n_proposed)
{
    extern __shared__ __align__(16) unsigned char frag_smem[];
    const int tid = threadIdx.x, nt = blockDim.x, NW = nt >> 5, warp = tid >> 5, lane = tid & 31;
    const int b_chain = blockIdx.x;
    const int c = S.chain0 + b_chain;
    const int T = S.T, M = M1 ? 1 : S.M, E = (T + 1) * M;
    const LineDiv<M1> D(M);
    int l, o;
    frag_cut(seed, counter, (uint32_t)c, l_min, l_max, levels, offsets, c, l, o);
    if (l < l_min || l > l_max || o < 0 || o >= (1 << l)) return;  // invalid cut: chain untouched
    const FragGeom G(T, l, o);
    const R inv_len = R(1) / (R)(1 << l);  // exact: a power of two

    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    unsigned char* p = frag_smem;
    PAMD_ARR(R, FS, (R*)p, nfrag_max);
    PAMD_ARR(R, FS0, (R*)p + nfrag_max, nfrag_max);
    p += up16(2 * sizeof(R) * nfrag_max);
    PAMD_ARR(R, X, (R*)p, E);
    p += up16(sizeof(R) * (size_t)E);
    PAMD_ARR(R, W, (R*)p, E);
    p += up16(sizeof(R) * (size_t)E);
    PAMD_ARR(R, WB, (R*)p, (long long)nfrag_max * M);
    p += up16(sizeof(R) * (size_t)nfrag_max * M);
    PAMD_ARR(R, tail, (R*)p, NW * M);
    PAMD_ARR(R, tS, (R*)p + NW * M, NW);
    PAMD_ARR(R, tS0, (R*)p + NW * M + NW, NW);
    p += up16(sizeof(R) * (size_t)NW * (M + 2));
    PAMD_ARR(int, accf, (int*)p, nfrag_max);
    PAMD_ARR(int, cnt, (int*)p + nfrag_max, 2);

    PAMD_ARR(R, gX, pos + S.off + (long long)b_chain * E, E);
    // 1. stage the path, draw sig z into W (slices 1..T), clear the sums
#pragma unroll 4
    for (int e = tid; e < E; e += nt) X[e] = gX[e];
    if (noise) {
        PAMD_ARR(const R, gZ, noise + S.off + (long long)b_chain * E, E);
#pragma unroll 4
        for (int e = M + tid; e < E; e += nt) W[e] = sig * gZ[e];
    } else {
        for (int g = (M >> 2) + tid; g <= ((E - 1) >> 2); g += nt) {
            const float4 q = philox_normals4(seed, counter, kStreamFragTrial, (uint32_t)c, (uint32_t)g);
            const float zq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * g + j;
                if (e >= M && e < E) W[e] = sig * (R)zq[j];
            }
        }
    }
    if (tid == 0) cnt[0] = cnt[1] = 0;
    __syncthreads();

    // 2. segmented prefix sum of W along each line over slices 1..T, one
    //    segment per fragment (slices a+1..b).  Warp w scans slices [t_lo, t_hi)
    //    in chunks of Lw lanes (whole slices), lane k on line k % M; lanes whose
    //    steps share a fragment combine.
    const int per = (T + NW - 1) / NW;
    const int t_lo = 1 + warp * per, t_hi = min(T + 1, t_lo + per);
    const int Lw = M1 ? 32 : (32 / M) * M;
    const int m_lane = M1 ? 0 : lane % M;
    {
        R carry = R(0);
        for (int e0 = t_lo * M; e0 < t_hi * M; e0 += Lw) {
            const int e = e0 + lane;
            const int n_act = min(Lw, t_hi * M - e0);
            const bool act = lane < n_act;
            const int t = D.slice(e);
            const int f = G.of_step(act ? t : t_lo);
            R v = act ? W[e] : R(0);
#pragma unroll
            for (int i = 0; (M1 ? 1 : M) << i < 32; ++i) {
                const int d = M << i;
                if (d >= Lw) break;
                const R vu = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d && G.of_step(t - (1 << i)) == f) v += vu;
            }
            const int t0 = D.slice(e0);
            if (act && f == G.of_step(t0 - 1)) v += carry;  // carry is 0 in the first chunk
            if (act) W[e] = v;
            carry = __shfl_sync(0xffffffffu, v, n_act - M + m_lane);
        }
        if (lane < M) tail[warp * M + lane] = (t_lo < t_hi) ? carry : R(0);
    }
    __syncthreads();
    // carry into the piece's first fragment from the pieces it began in
    if (warp > 0 && t_lo < t_hi) {
        const int f0 = G.of_step(t_lo), a0 = G.a(f0);
        if (a0 < t_lo - 1) {
            const int t_end = min(G.b(f0) + 1, t_hi);  // slices t_lo..t_end-1 are in f0
            for (int e = t_lo * M + lane; e < t_end * M; e += 32) {
                const int m = M1 ? 0 : e - D.slice(e) * M;
                R cin = R(0);
                for (int q = warp - 1; q >= 0; --q) {
                    cin += tail[q * M + m];
                    if (1 + q * per - 1 <= a0) break;  // fragment f0 starts in piece q
                }
                W[e] += cin;
            }
        }
    }
    __syncthreads();

    // 3. W_b of every fragment and line, then the trial in place of W
    for (int i = tid; i < G.nfrag * M; i += nt) {
        const int f = D.slice(i), m = i - f * M;
        WB[i] = W[G.b(f) * M + m];
    }
    __syncthreads();
    for (int e = M + tid; e < E; e += nt) {
        const int t = D.slice(e), m = M1 ? 0 : e - t * M;
        const int f = G.of_step(t), fa = G.a(f), fb = G.b(f);
        const R xa = X[fa * M + m];
        R y;
        if (f == G.nfrag - 1) {
            y = xa + W[e];
        } else if (t == fb) {
            y = X[e];
        } else {
            const R tf = small_int_to_r<R>(t - fa);
            const R sf = (f == 0) ? tf / small_int_to_r<R>(fb) : tf * inv_len;
            y = xa + sf * (X[fb * M + m] - xa) + (W[e] - sf * WB[f * M + m]);
        }
        W[e] = y;
    }
    __syncthreads();

    // 4. action differences of the step t-1 -> t, summed per fragment.  The
    //    per-step terms r'^2 - r^2 = (r' - r)(r' + r) (no cancellation) and
    //    dy^2 - dx^2 are in the path's precision and summed over all lines and
    //    steps of a fragment by a segmented scan of each warp's piece (elements
    //    in order, one segment per fragment); the lane holding a fragment's last
    //    element stores the piece's share, and shares of fragments that began in
    //    earlier pieces are added below in a fixed order (deterministic sums).
    {
        R carry = R(0), carry0 = R(0);
        int carry_key = -1;
        const int e_hi = t_hi * M;
        for (int e0 = t_lo * M; e0 < e_hi; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < e_hi;
            const int t = D.slice(act ? e : e0);
            const int f = G.of_step(t);
            R cs = R(0), cs0 = R(0);
            if (act) {
                const R x1 = X[e], x0 = X[e - M];
                const R y1 = W[e], y0 = (t - 1 == G.a(f)) ? x0 : W[e - M];
                const R r = (x1 - x0) + ak * x0, rt = (y1 - y0) + ak * y0;
                const R dx = x1 - x0, dy = y1 - y0;
                cs = (rt - r) * (rt + r);
                cs0 = (dy - dx) * (dy + dx);
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const R u1 = __shfl_up_sync(0xffffffffu, cs, d);
                const R u2 = __shfl_up_sync(0xffffffffu, cs0, d);
                const int fk = __shfl_up_sync(0xffffffffu, f, d);
                if (lane >= d && fk == f) {
                    cs += u1;
                    cs0 += u2;
                }
            }
            if (f == carry_key) {
                cs += carry;
                cs0 += carry0;
            }
            if (act && t == G.b(f) && (M1 || e - t * M == M - 1)) {
                FS[f] = cs;
                FS0[f] = cs0;
            }
            const int src = min(31, e_hi - 1 - e0);
            carry = __shfl_sync(0xffffffffu, cs, src);
            carry0 = __shfl_sync(0xffffffffu, cs0, src);
            carry_key = __shfl_sync(0xffffffffu, f, src);
        }
        if (lane == 0) {
            tS[warp] = (t_lo < t_hi) ? carry : R(0);
            tS0[warp] = (t_lo < t_hi) ? carry0 : R(0);
        }
    }
    __syncthreads();
    if (tid > 0 && tid < NW) {
        const int w_lo = 1 + tid * per, w_hi = min(T + 1, w_lo + per);
        if (w_lo < w_hi) {
            const int f0 = G.of_step(w_lo), a0 = G.a(f0);
            if (a0 < w_lo - 1 && G.b(f0) < w_hi) {
                R c1 = R(0), c2 = R(0);
                for (int q = tid - 1; q >= 0; --q) {
                    c1 += tS[q];
                    c2 += tS0[q];
                    if (q * per <= a0) break;  // f0 starts in piece q
                }
                FS[f0] += c1;
                FS0[f0] += c2;
            }
        }
    }
    __syncthreads();

    // 5. Metropolis-Hastings decision of every fragment with an interior point
    for (int f = tid; f < G.nfrag; f += nt) {
        int acc = 0;
        const int fa = G.a(f), fb = G.b(f);
        if (f == G.nfrag - 1 || fb - fa >= 2) {
            acc = frag_accept<R>(FS[f], FS0[f], cS, cSf, c0, c0f, log_u, fstride, c, f, seed, counter);
            atomicAdd(cnt, 1);
            if (acc) atomicAdd(cnt + 1, 1);
        }
        accf[f] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(n_proposed + c, cnt[0]);
        atomicAdd(n_accepted + c, cnt[1]);
    }

    // 6. accepted interiors (and the nose end) back to the path
#pragma unroll 4
    for (int e = M + tid; e < E; e += nt) {
        const int t = D.slice(e);
        const int f = G.of_step(t);
        if (accf[f] && (t < G.b(f) || f == G.nfrag - 1)) gX[e] = W[e];
    }
}

// Asynchronous global -> shared copy of one element (LDGSTS), so that staging
// the path overlaps the normal generation and the walk scan.
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* smem, const R* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One-line paths (M = 1, e.g. the 1D oscillator): as fragment_block_kernel, but
// every lane holds four consecutive slices (one Philox group, one 16-byte
// shared-memory word), so the scans are a local scan of four plus one warp scan
// per 128 slices.
template <typename R>
__host__ __device__ inline size_t frag_line_smem(int T, int nfrag_max, int nwarps, int n_shift)
{
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t E4 = ((size_t)T + 4) & ~(size_t)3;  // slices 0..T, rounded up to quads
    return up16(2 * sizeof(R) * nfrag_max)           // fragment sums s, s0
           + 2 * up16(sizeof(R) * E4)                 // X, W
           + up16(sizeof(R) * (size_t)nfrag_max)      // W_b
           + up16(sizeof(R) * (size_t)nwarps * 3)     // piece tails (W, s, s0)
           + up16(sizeof(R) * (size_t)n_shift)        // regeneration normals
           + up16(sizeof(int) * (2 * (size_t)nfrag_max + 2));  // accepted list and flags, counts
}

template <typename R>
struct Quad {
    R v[4];
};

template <typename R>
__device__ __forceinline__ Quad<R> load_quad(const R* p)
{
    Quad<R> q;
    if (sizeof(R) == 4) {
        const float4 f = *reinterpret_cast<const float4*>(p);
        q.v[0] = (R)f.x;
        q.v[1] = (R)f.y;
        q.v[2] = (R)f.z;
        q.v[3] = (R)f.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) q.v[j] = p[j];
    }
    return q;
}

template <typename R>
__device__ __forceinline__ void store_quad(R* p, const R (&v)[4])
{
    if (sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = v[j];
    }
}

// Segmented inclusive scan of one quad per lane in lane order: v[j] (and w[j])
// of the elements with fragment keys k[j] (non-decreasing along the warp).
// Adds the earlier lanes' part of each element's segment and the carry from
// the previous chunk (carry_key), and returns the new carry from lane `src`.
template <typename R, int NV>
__device__ __forceinline__ void quad_scan(R (&v)[NV][4], const int (&k)[4], int lane, R (&carry)[NV],
                                          int& carry_key, int src)
{
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (k[j] == k[j - 1])
#pragma unroll
            for (int n = 0; n < NV; ++n) v[n][j] += v[n][j - 1];
    R agg[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) agg[n] = v[n][3];
    const int akey = k[3];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        R up[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) up[n] = __shfl_up_sync(0xffffffffu, agg[n], d);
        const int uk = __shfl_up_sync(0xffffffffu, akey, d);
        if (lane >= d && uk == akey)
#pragma unroll
            for (int n = 0; n < NV; ++n) agg[n] += up[n];
    }
    R pre[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) pre[n] = __shfl_up_sync(0xffffffffu, agg[n], 1);
    int pkey = __shfl_up_sync(0xffffffffu, akey, 1);
    if (lane == 0) pkey = -1;
    R add[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n)
        add[n] = (pkey == k[0] ? pre[n] : R(0)) + (carry_key == k[0] ? carry[n] : R(0));
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (k[j] == k[0])
#pragma unroll
            for (int n = 0; n < NV; ++n) v[n][j] += add[n];
#pragma unroll
    for (int n = 0; n < NV; ++n) carry[n] = __shfl_sync(0xffffffffu, v[n][3], src);
    carry_key = __shfl_sync(0xffffffffu, k[3], src);
}

// Optional epilogue of the last MC step of a shifting event (paper Fig. 2): the
// final path of each chain also goes, shifted by n_shift steps, to `out`, its
// points x_1..x_{n_shift} to `traj`, and the last n_shift slices of `out` are
// regrown from the nose exactly as launch_shift_regenerate does (Philox stream
// 6 at `counter`, sequential x <- fma(sig, z, x)).
template <typename R>
struct ShiftOut {
    R* out;           // path buffer in the layout of pos; nullptr: no epilogue
    R* traj;          // this system's [chains][n_shift] block of the trajectory
    int n_shift;
    uint64_t counter;
    double sig;       // width of a regeneration step (0: the line x_T continues)
};

template <typename R>
__global__ void __launch_bounds__(kFragMaxThreads)
    fragment_line_kernel(R* __restrict__ pos, const FragSys S, int l_min, int l_max, uint64_t seed,
                         uint64_t counter, const int* __restrict__ levels,
                         const int* __restrict__ offsets, const R* __restrict__ noise,
                         const double* __restrict__ log_u, int fstride, int nfrag_max, R ak, R sig,
                         double cS, float cSf, double c0, float c0f, int* __restrict__ n_accepted,
                         int* __restrict__ n_proposed, const ShiftOut<R> sh)
{
    extern __shared__ __align__(16) unsigned char frag_smem[];
    const int tid = threadIdx.x, nt = blockDim.x, NW = nt >> 5, warp = tid >> 5, lane = tid & 31;
    if (nt & 31) return;  // the launcher uses whole warps
    const int b_chain = blockIdx.x;
    const int c = S.chain0 + b_chain;
    const int T = S.T, E = T + 1, Q = (T + 4) >> 2;  // quads of slices 0..T
    int l, o;
    frag_cut(seed, counter, (uint32_t)c, l_min, l_max, levels, offsets, c, l, o);
    if (l < l_min || l > l_max || o < 0 || o >= (1 << l)) return;  // invalid cut: chain untouched
    const FragGeom G(T, l, o);
    const R inv_len = R(1) / (R)(1 << l);  // exact: a power of two

    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    unsigned char* p = frag_smem;
    PAMD_ARR(R, FS, (R*)p, nfrag_max);
    PAMD_ARR(R, FS0, (R*)p + nfrag_max, nfrag_max);
    p += up16(2 * sizeof(R) * nfrag_max);
    PAMD_ARR(R, X, (R*)p, Q * 4);
    p += up16(sizeof(R) * (size_t)Q * 4);
    PAMD_ARR(R, W, (R*)p, Q * 4);
    p += up16(sizeof(R) * (size_t)Q * 4);
    PAMD_ARR(R, WB, (R*)p, nfrag_max);
    p += up16(sizeof(R) * (size_t)nfrag_max);
    PAMD_ARR(R, tW, (R*)p, NW);
    PAMD_ARR(R, tS, (R*)p + NW, NW);
    PAMD_ARR(R, tS0, (R*)p + 2 * NW, NW);
    p += up16(sizeof(R) * (size_t)NW * 3);
    PAMD_ARR(R, Zs, (R*)p, sh.out ? sh.n_shift : 0);
    p += up16(sizeof(R) * (size_t)(sh.out ? sh.n_shift : 0));
    PAMD_ARR(int, accf, (int*)p, nfrag_max);
    PAMD_ARR(int, aflag, (int*)p + nfrag_max, nfrag_max);
    PAMD_ARR(int, cnt, (int*)p + 2 * nfrag_max, 2);

    PAMD_ARR(R, gX, pos + S.off + (long long)b_chain * E, E);
    PAMD_ARR(const R, gZ, noise ? noise + S.off + (long long)b_chain * E : nullptr, E);
    // 1. stage the path asynchronously (quads padded with zeros); it is first
    //    read in step 4
#pragma unroll 4
    for (int e = tid; e < E; e += nt)
        if (PAMD_OK_IDX(e, Q * 4)) cp_async_elem((R*)X + e, (R*)gX + e);
    cp_async_commit();
    if (tid < Q * 4 - E) X[E + tid] = R(0);
    if (tid == 0) cnt[0] = cnt[1] = 0;
    if (sh.out) {
        for (int f = tid; f < G.nfrag; f += nt) aflag[f] = 0;
        for (int g = tid; 4 * g < sh.n_shift; g += nt) {
            const float4 z = philox_normals4(seed, sh.counter, kStreamRegenerate, (uint32_t)c, (uint32_t)g);
            const float zq[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * g + j < sh.n_shift) Zs[4 * g + j] = (R)zq[j];
        }
    }
    __syncthreads();

    // pieces: warp w owns quads [q_lo, q_hi), i.e. slices [e_lo, e_hi) of 1..T
    const int perq = (Q + NW - 1) / NW;
    const int q_lo = warp * perq, q_hi = min(Q, q_lo + perq);
    const int e_lo = max(1, 4 * q_lo), e_hi = min(E, 4 * q_hi);
    auto piece_lo = [&](int w) { return max(1, 4 * w * perq); };

    // 2. sig z from Philox (one group per lane) or given, and its segmented
    //    prefix sum over each fragment's slices a+1..b, in place in W
    {
        R carry[1] = {R(0)};
        int ckey = -1;
        for (int q0 = q_lo; q0 < q_hi; q0 += 32) {
            const int q = q0 + lane;
            const bool qa = q < q_hi;
            R v[1][4];
            int k[4];
            if (qa && !gZ) {
                const float4 z = philox_normals4(seed, counter, kStreamFragTrial, (uint32_t)c, (uint32_t)q);
                v[0][0] = sig * (R)z.x;
                v[0][1] = sig * (R)z.y;
                v[0][2] = sig * (R)z.z;
                v[0][3] = sig * (R)z.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * q + j;
                const bool act = qa && e >= 1 && e < E;
                if (gZ) v[0][j] = act ? sig * gZ[e] : R(0);
                else if (!act) v[0][j] = R(0);
                k[j] = G.of_step(min(max(e, 1), T));
            }
            quad_scan<R, 1>(v, k, lane, carry, ckey, min(31, q_hi - 1 - q0));
            if (qa && PAMD_OK_IDX(4 * q + 3, Q * 4)) store_quad((R*)W + 4 * q, v[0]);
        }
        if (lane == 0) tW[warp] = (q_lo < q_hi) ? carry[0] : R(0);
    }
    __syncthreads();
    if (warp > 0 && e_lo < e_hi) {  // carry into the piece's first fragment
        const int f0 = G.of_step(e_lo), a0 = G.a(f0);
        if (a0 < e_lo - 1) {
            R cin = R(0);
            for (int q = warp - 1; q >= 0; --q) {
                cin += tW[q];
                if (piece_lo(q) - 1 <= a0) break;
            }
            const int end = min(G.b(f0) + 1, e_hi);
            for (int e = e_lo + lane; e < end; e += 32) W[e] += cin;
        }
    }
    __syncthreads();

    // 3. W_b of every fragment.  The trial point of slice e in fragment f is
    //    computed where it is needed (the action sums, then the write-back of
    //    accepted fragments) with explicitly rounded operations, so both uses
    //    see the same value.
    for (int f = tid; f < G.nfrag; f += nt) WB[f] = W[G.b(f)];
    cp_async_wait_all();
    __syncthreads();
    auto trial = [&](int e, int f, R w) -> R {
        const int fa = G.a(f), fb = G.b(f);
        const R xa = X[fa];
        if (f == G.nfrag - 1) return add_r(xa, w);
        if (e == fb) return X[e];
        const R tf = small_int_to_r<R>(e - fa);
        const R sf = (f == 0) ? div_r(tf, small_int_to_r<R>(fb)) : mul_r(tf, inv_len);
        return add_r(fma_r(sf, sub_r(X[fb], xa), xa), fma_r(-sf, WB[f], w));
    };

    // 4. per-step terms (r'-r)(r'+r) and (dy-dx)(dy+dx) summed per fragment
    {
        R carry[2] = {R(0), R(0)};
        int ckey = -1;
        // slice 4 q_lo - 1 (the piece's left neighbour) for lane 0 of the first chunk
        R xl = R(0), yl = R(0);
        if (lane == 0 && q_lo > 0 && q_lo < q_hi) {
            const int e = 4 * q_lo - 1, f = G.of_step(e);
            xl = X[e];
            yl = trial(e, f, W[e]);
        }
        for (int q0 = q_lo; q0 < q_hi; q0 += 32) {
            const int q = q0 + lane;
            const bool qa = q < q_hi;
            R v[2][4];
            int k[4];
            R y[4];
            const bool qok = PAMD_OK_IDX(4 * min(q, Q - 1) + 3, Q * 4);
            const Quad<R> xq = load_quad((R*)X + 4 * (qok ? min(q, Q - 1) : 0));
            const Quad<R> wq = load_quad((R*)W + 4 * (qok ? min(q, Q - 1) : 0));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ec = min(max(4 * q + j, 1), T);
                k[j] = G.of_step(ec);
                y[j] = trial(ec, k[j], wq.v[j]);
            }
            // slice 4q - 1 from the lane below (lane 0: the previous chunk's lane 31)
            R xp = __shfl_up_sync(0xffffffffu, xq.v[3], 1);
            R yp = __shfl_up_sync(0xffffffffu, y[3], 1);
            if (lane == 0) {
                xp = xl;
                yp = yl;
            }
            xl = __shfl_sync(0xffffffffu, xq.v[3], 31);
            yl = __shfl_sync(0xffffffffu, y[3], 31);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * q + j;
                const bool act = qa && e >= 1 && e < E;
                const int ec = min(max(e, 1), T);
                const int f = k[j];
                const R x1 = xq.v[j], x0 = j ? xq.v[j - 1] : xp;
                const R y1 = y[j];
                const R y0 = (ec - 1 == G.a(f)) ? x0 : (j ? y[j - 1] : yp);
                const R r = (x1 - x0) + ak * x0, rt = (y1 - y0) + ak * y0;
                const R dx = x1 - x0, dy = y1 - y0;
                v[0][j] = act ? (rt - r) * (rt + r) : R(0);
                v[1][j] = act ? (dy - dx) * (dy + dx) : R(0);
            }
            quad_scan<R, 2>(v, k, lane, carry, ckey, min(31, q_hi - 1 - q0));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * q + j;
                if (qa && e >= 1 && e < E && e == G.b(k[j])) {
                    FS[k[j]] = v[0][j];
                    FS0[k[j]] = v[1][j];
                }
            }
        }
        if (lane == 0) {
            tS[warp] = (q_lo < q_hi) ? carry[0] : R(0);
            tS0[warp] = (q_lo < q_hi) ? carry[1] : R(0);
        }
    }
    __syncthreads();
    if (tid > 0 && tid < NW) {
        const int w_lo = piece_lo(tid), w_hi = min(E, 4 * min(Q, (tid + 1) * perq));
        if (w_lo < w_hi) {
            const int f0 = G.of_step(w_lo), a0 = G.a(f0);
            if (a0 < w_lo - 1 && G.b(f0) < w_hi) {
                R c1 = R(0), c2 = R(0);
                for (int q = tid - 1; q >= 0; --q) {
                    c1 += tS[q];
                    c2 += tS0[q];
                    if (piece_lo(q) - 1 <= a0) break;
                }
                FS[f0] += c1;
                FS0[f0] += c2;
            }
        }
    }
    __syncthreads();

    // 5. Metropolis-Hastings decision of every fragment with an interior point;
    //    accepted fragments are listed (in any order: their writes are disjoint)
    for (int f = tid; f < G.nfrag; f += nt) {
        const int fa = G.a(f), fb = G.b(f);
        if (f == G.nfrag - 1 || fb - fa >= 2) {
            atomicAdd(cnt, 1);
            if (frag_accept<R>(FS[f], FS0[f], cS, cSf, c0, c0f, log_u, fstride, c, f, seed, counter)) {
                accf[atomicAdd(cnt + 1, 1)] = f;
                if (sh.out) aflag[f] = 1;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(n_proposed + c, cnt[0]);
        atomicAdd(n_accepted + c, cnt[1]);
    }

    if (!sh.out) {
        // 6. accepted interiors (and the nose end) back to the path, a warp per fragment
        const int n_acc = cnt[1];
        for (int i = warp; i < n_acc; i += NW) {
            const int f = accf[i], fa = G.a(f), fb = G.b(f);
            const int t_end = (f == G.nfrag - 1) ? fb : fb - 1;
            for (int e = fa + 1 + lane; e <= t_end; e += 32) gX[e] = trial(e, f, W[e]);
        }
        return;
    }
    // 6'. final path P: accepted interiors to the path, P shifted to `out`,
    //     P[1..n_shift] to the trajectory, and the nose regrown
    const int ns = sh.n_shift;
    PAMD_ARR(R, gO, sh.out + S.off + (long long)b_chain * E, E);
    PAMD_ARR(R, gT, sh.traj + (long long)b_chain * ns, ns);
    auto final_at = [&](int e) -> R {
        const int f = G.of_step(e);
        if (aflag[f] && (e < G.b(f) || f == G.nfrag - 1)) return trial(e, f, W[e]);
        return X[e];
    };
    for (int e = 1 + tid; e < E; e += nt) {
        const int f = G.of_step(e);
        R pe = X[e];
        if (aflag[f] && (e < G.b(f) || f == G.nfrag - 1)) {
            pe = trial(e, f, W[e]);
            gX[e] = pe;
        }
        if (e >= ns) gO[e - ns] = pe;
        if (e <= ns) gT[e - 1] = pe;
    }
    if (tid == nt - 1) {
        R x = final_at(T);
        const R sr = (R)sh.sig;
        for (int k = 1; k <= ns; ++k) {
            x = fma_r(sr, Zs[k - 1], x);
            gO[T - ns + k] = x;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128)
    fragment_thread_kernel(R* __restrict__ pos, const FragSys S, int l_min, int l_max, uint64_t seed,
                           uint64_t counter, const int* __restrict__ levels,
                           const int* __restrict__ offsets, const R* __restrict__ noise,
                           const double* __restrict__ log_u, int fstride, R ak, R sig, double cS,
                           double c0, int* __restrict__ n_accepted, int* __restrict__ n_proposed)
{
    const int b_chain = blockIdx.y;
    const int c = S.chain0 + b_chain;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    int l, o;
    frag_cut(seed, counter, (uint32_t)c, l_min, l_max, levels, offsets, c, l, o);
    if (l < l_min || l > l_max || o < 0 || o >= (1 << l)) return;  // invalid cut: chain untouched
    const FragGeom G(S.T, l, o);
    if (f >= G.nfrag) return;
    const int T = S.T, M = S.M, fa = G.a(f), fb = G.b(f);
    const bool nose = (f == G.nfrag - 1);
    if (!nose && fb - fa < 2) return;  // no interior point
    PAMD_ARR(R, X, pos + S.off + (long long)b_chain * (long long)(T + 1) * M, (long long)(T + 1) * M);
    PAMD_ARR(const R, Z, noise ? noise + S.off + (long long)b_chain * (long long)(T + 1) * M : nullptr,
             (long long)(T + 1) * M);

    auto znorm = [&](int t, int m) -> R {
        const long long e = (long long)t * M + m;
        if (Z) return Z[e];
        const float4 q = philox_normals4(seed, counter, kStreamFragTrial, (uint32_t)c, (uint32_t)(e >> 2));
        return (R)pick4(q, (int)(e & 3));
    };
    // trial point at t from the running walk value w
    auto trial = [&](int t, R w, R xa, R xb, R wb) -> R {
        if (nose) return xa + w;
        if (t == fb) return xb;
        const R sf = (R)(t - fa) / (R)(fb - fa);
        return xa + sf * (xb - xa) + (w - sf * wb);
    };

    // sums in the path's precision over blocks of 64 steps, blocks added in double
    double dS = 0.0, dS0 = 0.0;
    R bS = R(0), bS0 = R(0);
    int nb = 0;
    for (int m = 0; m < M; ++m) {
        const R xa = X[(long long)fa * M + m], xb = X[(long long)fb * M + m];
        R wb = R(0);
        if (!nose)
            for (int t = fa + 1; t <= fb; ++t) wb += sig * znorm(t, m);
        R w = R(0), y = xa, x = xa;
        for (int t = fa + 1; t <= fb; ++t) {
            w += sig * znorm(t, m);
            const R y1 = trial(t, w, xa, xb, wb);
            const R x1 = X[(long long)t * M + m];
            const R r = (x1 - x) + ak * x, rt = (y1 - y) + ak * y;
            const R dx = x1 - x, dy = y1 - y;
            bS += (rt - r) * (rt + r);
            bS0 += (dy - dx) * (dy + dx);
            if (++nb == 64) {
                dS += (double)bS;
                dS0 += (double)bS0;
                bS = bS0 = R(0);
                nb = 0;
            }
            x = x1;
            y = y1;
        }
    }
    dS += (double)bS;
    dS0 += (double)bS0;
    atomicAdd(n_proposed + c, 1);
    if (!frag_accept<double>(dS, dS0, cS, (float)cS, c0, (float)c0, log_u, fstride, c, f, seed,
                             counter))
        return;
    atomicAdd(n_accepted + c, 1);
    for (int m = 0; m < M; ++m) {
        const R xa = X[(long long)fa * M + m], xb = X[(long long)fb * M + m];
        R wb = R(0);
        if (!nose)
            for (int t = fa + 1; t <= fb; ++t) wb += sig * znorm(t, m);
        R w = R(0);
        const int tend = nose ? fb : fb - 1;
        for (int t = fa + 1; t <= tend; ++t) {
            w += sig * znorm(t, m);
            X[(long long)t * M + m] = trial(t, w, xa, xb, wb);
        }
    }
}

template <typename R>
bool fragment_event_fusable(int T, int M, int l_min, int n_shift)
{
    const int nfrag_max = (T >> l_min) + 2;
    return M == 1 && frag_line_smem<R>(T, nfrag_max, kFragMaxThreads / 32, n_shift) <= kFragBlockSmemMax;
}

template <typename R>
cudaError_t launch_fragment_mc(R* pos, long long off, int T, int M, int n_chains, int chain0,
                               int l_min, int l_max, uint64_t seed, uint64_t counter,
                               const int* levels, const int* offsets, const R* noise,
                               const double* log_u, int fstride, double g, double sig, double cS,
                               double c0, int* n_accepted, int* n_proposed, cudaStream_t st,
                               R* shift_out, R* shift_traj, int n_shift, uint64_t shift_counter,
                               double shift_sig)
{
    if (n_chains <= 0) return cudaSuccess;
    ShiftOut<R> sh;
    sh.out = shift_out ? shift_out : nullptr;
    sh.traj = shift_traj;
    sh.n_shift = shift_out ? n_shift : 0;
    sh.counter = shift_counter;
    sh.sig = shift_sig;
    if (shift_out && !fragment_event_fusable<R>(T, M, l_min, n_shift)) return cudaErrorInvalidValue;
    FragSys S;
    S.off = off;
    S.T = T;
    S.M = M;
    S.chain0 = chain0;
    const int nfrag_max = (T >> l_min) + 2;
    const long long E = (long long)(T + 1) * M;
    int threads = (int)std::min<long long>(kFragMaxThreads, ((E + 15) / 16 + 31) / 32 * 32);
    threads = std::max(threads, 64);
    if (M == 1 && frag_line_smem<R>(T, nfrag_max, kFragMaxThreads / 32, sh.n_shift) <= kFragBlockSmemMax) {
        // whole warps, about four quads per lane: 64..256 threads
        const int quads = (T + 4) / 4;
        const int lthreads = std::min(kFragMaxThreads, std::max(64, (quads + 127) / 128 * 32));
        const size_t lsmem = frag_line_smem<R>(T, nfrag_max, lthreads / 32, sh.n_shift);
        cudaError_t e = cudaFuncSetAttribute(fragment_line_kernel<R>,
                                             cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        if (e == cudaSuccess && lsmem > 48 * 1024)
            e = cudaFuncSetAttribute(fragment_line_kernel<R>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem);
        if (e != cudaSuccess) return e;
        fragment_line_kernel<R><<<n_chains, lthreads, lsmem, st>>>(
            pos, S, l_min, l_max, seed, counter, levels, offsets, noise, log_u, fstride, nfrag_max,
            (R)g, (R)sig, cS, (float)cS, c0, (float)c0, n_accepted, n_proposed, sh);
        return cudaGetLastError();
    }
    const size_t smem = frag_block_smem<R>(T, M, nfrag_max, threads / 32);
    if (M <= 32 && smem <= kFragBlockSmemMax) {
        auto kern = (M == 1) ? fragment_block_kernel<R, true> : fragment_block_kernel<R, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        if (e == cudaSuccess && smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<n_chains, threads, smem, st>>>(pos, S, l_min, l_max, seed, counter, levels, offsets,
                                              noise, log_u, fstride, nfrag_max, (R)g, (R)sig, cS,
                                              (float)cS, c0, (float)c0, n_accepted, n_proposed);
        return cudaGetLastError();
    }
    // grid.y holds at most 65535 chains: launch in batches (chain0 and the offset advance)
    const int tthreads = 128;
    for (int b0 = 0; b0 < n_chains; b0 += 65535) {
        const int nb = std::min(65535, n_chains - b0);
        FragSys Sb = S;
        Sb.off = off + (long long)b0 * (long long)(T + 1) * M;
        Sb.chain0 = chain0 + b0;
        dim3 grid((nfrag_max + tthreads - 1) / tthreads, nb);
        fragment_thread_kernel<R><<<grid, tthreads, 0, st>>>(pos, Sb, l_min, l_max, seed, counter,
                                                             levels, offsets, noise, log_u, fstride,
                                                             (R)g, (R)sig, cS, c0, n_accepted,
                                                             n_proposed);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template bool fragment_event_fusable<float>(int, int, int, int);
template bool fragment_event_fusable<double>(int, int, int, int);
template cudaError_t launch_fragment_mc<float>(float*, long long, int, int, int, int, int, int,
                                               uint64_t, uint64_t, const int*, const int*,
                                               const float*, const double*, int, double, double,
                                               double, double, int*, int*, cudaStream_t, float*,
                                               float*, int, uint64_t, double);
template cudaError_t launch_fragment_mc<double>(double*, long long, int, int, int, int, int, int,
                                                uint64_t, uint64_t, const int*, const int*,
                                                const double*, const double*, int, double, double,
                                                double, double, int*, int*, cudaStream_t, double*,
                                                double*, int, uint64_t, double);

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
    const int per = (T + 1) * M, nmove = (T + 1 - n_shift) * M, ns = n_shift * M;
    for (int b = blockIdx.x; b < n_chains; b += gridDim.x) {
        const R* src = pos + off + (long long)b * per;
        R* dst = out + off + (long long)b * per;
        R* tr = traj + traj_off + (long long)b * ns;
#pragma unroll 4
        for (int i = threadIdx.x; i < nmove; i += blockDim.x) dst[i] = src[i + ns];
        for (int i = threadIdx.x; i < ns; i += blockDim.x) tr[i] = src[M + i];
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
        x = fma_r(sig, z, x);
        X[(long long)(T - n_shift + k) * M + m] = x;
    }
}

template <typename R>
cudaError_t launch_shift_regenerate(const R* pos, R* out, R* traj, long long off, long long traj_off,
                                    int T, int M, int n_shift, int n_chains, int chain0, double sig,
                                    uint64_t seed, uint64_t counter, const R* noise, cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    if ((long long)(T + 1) * M > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    const int threads = 256;
    const int blocks = std::min(n_chains, 152 * 8);
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

PAMD_DEBUG_FETCHER(fragment)

}  // namespace pamd
