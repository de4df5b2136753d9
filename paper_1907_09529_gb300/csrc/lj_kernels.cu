// lj_kernels.cu -- Lennard-Jones path action and adjoint gradient, Euler-Maruyama
// reference paths, and the single-precision pair-count diagnostic.
//
// Pair potential (paper Eq. (11)), cut and force shifted:
//   U(r) = u(r) - u(rc) - (r - rc) u'(rc)  (r <= rc),  u = 4 eps[(s/r)^12 - (s/r)^6].
// With S6 = (sigma/r)^6 and ir2 = 1/r^2:
//   u'(r)/r = 24 eps ir2 S6 (1 - 2 S6),   u''(r) = 24 eps ir2 S6 (26 S6 - 7),
//   U'(r)/r = u'(r)/r - u'(rc)/r,          U''(r) = u''(r).
// Force on i:  F_i = -sum_j (U'(r)/r) r_ij,  r_ij = x_i - x_j (minimum image).
// Hessian-vector product:  (Hv)_i = sum_j [ (U'/r) v_ij + ((U'' - U'/r)/r^2)(r_ij . v_ij) r_ij ],
// v_ij = v_i - v_j.  With a = beta D dt:
//   r_t = x_{t+1} - x_t - a F(x_t)                          (Eq. (3))
//   g_t = [r_{t-1} - r_t + a H(x_t) r_t] / (2 D dt),  r_{-1} = r_T = 0.
//
// Work decomposition.  A persistent grid pulls work items -- (system, chain,
// tile of consecutive steps) -- from an atomic queue, largest first, so that
// chains and systems of different N and T share one launch.  For an item the
// current slice x_t and the next x_{t+1} live in shared memory as 4-vectors, as
// does r_t (the Hessian-vector product needs the residuals of the neighbours).
// Each particle owns TPP adjacent threads (TPP per system, a power of two);
// thread q of particle i handles the candidates j = q (mod TPP).  A Verlet list of radius rc + skin, built from the
// slice at the tile start, is kept in shared memory and reused for the following
// slices: it stays exact while no particle has moved more than skin/2 from the
// position it had when the list was built (then no pair can have crossed from
// outside rc + skin to inside rc); otherwise the CTA rebuilds it.  A particle
// whose list overflows the capacity scans all candidates instead.  Candidates are
// visited in increasing j in either case, so every sum has the same order no
// matter when the list was (re)built: results do not depend on the tiling.
// The residual of the step before the tile (r_{t0-1}) is recomputed locally.
#include "pamd_internal.cuh"

namespace pamd {

// Round-to-nearest-even of the exact product a*b (|a*b| < 2^22), by adding and
// removing 1.5*2^23 (float) or 1.5*2^52 (double): one FMA and one add.
__device__ __forceinline__ float round_prod(float a, float b)
{
    return __fsub_rn(__fmaf_rn(a, b, 12582912.0f), 12582912.0f);
}
__device__ __forceinline__ double round_prod(double a, double b)
{
    return __dsub_rn(__fma_rn(a, b, 6755399441055744.0), 6755399441055744.0);
}

// Minimum-image pair vector and |r_ij|^2 by the documented rule:
//   dx = xi - xj;  dx = fma(-L, round(dx * (1/L)), dx);  r2 = fma(dz,dz,fma(dy,dy,dx*dx)).
template <typename R>
__device__ __forceinline__ R pair_r2(R xi, R yi, R zi, const vec4_t<R>& pj, const LJK<R>& k, R& dx,
                                     R& dy, R& dz)
{
    dx = xi - pj.x;
    dy = yi - pj.y;
    dz = zi - pj.z;
    dx = fma_r(-k.L, round_prod(dx, k.iL), dx);
    dy = fma_r(-k.L, round_prod(dy, k.iL), dy);
    dz = fma_r(-k.L, round_prod(dz, k.iL), dz);
    return fma_r(dz, dz, fma_r(dy, dy, mul_r(dx, dx)));
}

// Reciprocal square root: the hardware approximation in single precision
// (relative error below 2^-22), the library function in double.
__device__ __forceinline__ float rsqrt_fast(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double rsqrt_fast(double v) { return rsqrt(v); }

// Pair scalars from r^2 (inside the cutoff):
//   fs  = -U'(r)/r = ir2 * u * t + u'(rc)/r,  u = c1 ir6, t = c2 ir6 - 1
//   upp = U''(r)   = ir2 * u * (c3 ir6 - 7)
template <typename R>
__device__ __forceinline__ R pair_fs(R r2, const LJK<R>& k, R& ir2, R& u, R& ir6)
{
    const R ri = rsqrt_fast(r2);
    ir2 = ri * ri;
    ir6 = ir2 * ir2 * ir2;
    u = k.c1 * ir6;
    const R t = fma_r(k.c2, ir6, R(-1));
    return fma_r(u * t, ir2, k.duc * ri);
}


template <typename R>
struct LJBlock {
    using V4 = vec4_t<R>;
    int N, NT, tid, i, q, tpp, cap;
    bool active;
    uint16_t* nbr;  // nbr[m * NT + tid], m < cap
    int cnt;
    bool ovf;
    R xr, yr, zr;   // position at the last list build

    __device__ void init(int n, int tpp_, int lg, int cap_, uint16_t* list)
    {
        N = n;
        NT = blockDim.x;
        tid = threadIdx.x;
        tpp = tpp_;
        i = tid >> lg;
        q = tid & (tpp_ - 1);
        active = i < n;
        cap = cap_;
        nbr = list;
        cnt = 0;
        ovf = false;
    }

    __device__ void build(const V4* __restrict__ buf, const LJK<R>& k)
    {
        cnt = 0;
        ovf = false;
        if (!active) return;
        const V4 p = buf[i];
        xr = p.x;
        yr = p.y;
        zr = p.z;
        int c = 0;
        for (int j = q; j < N; j += tpp) {
            if (j == i) continue;
            R dx, dy, dz;
            const R r2 = pair_r2<R>(p.x, p.y, p.z, buf[j], k, dx, dy, dz);
            if (r2 <= k.rl2) {
                if (c < cap && PAMD_OK_IDX(c * NT + tid, cap * NT)) nbr[c * NT + tid] = (uint16_t)j;
                ++c;
            }
        }
        cnt = c;
        ovf = c > cap;
    }

    __device__ bool moved(const V4* __restrict__ buf, const LJK<R>& k) const
    {
        if (!active) return false;
        const V4 p = buf[i];
        const R dx = p.x - xr, dy = p.y - yr, dz = p.z - zr;
        return dx * dx + dy * dy + dz * dz > k.hs2;
    }

    __device__ __forceinline__ void group_sum(R& x, R& y, R& z) const
    {
        for (int o = tpp >> 1; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
    }

    // Candidates of particle i handled by this thread, in increasing j: the
    // Verlet list, or every other particle when the list overflowed.
    template <typename F>
    __device__ __forceinline__ void for_each_candidate(F&& f) const
    {
        if (!active) return;
        if (!ovf) {
            for (int m = 0; m < cnt; ++m) {
                const int j = PAMD_OK_IDX(m * NT + tid, cap * NT) ? (int)nbr[m * NT + tid] : i;
                if (PAMD_OK_IDX(j, N)) f(j);
            }
        } else {
            for (int j = q; j < N; j += tpp)
                if (j != i) f(j);
        }
    }

    // F(x) of particle i (complete in every thread of the group).  Single
    // precision is branch-free (every list entry evaluated, masked by the cutoff
    // test); double precision skips the costly math outside the cutoff.
    // ov (non-null: the hard-sphere path bias is on): raised when a pair within the
    // cutoff lies within the squared hard-sphere radius hs2v of this slice.
    __device__ void force(const V4* __restrict__ buf, const LJK<R>& k, R& fx, R& fy, R& fz,
                          R hs2v = R(-1), bool* ov = nullptr) const
    {
        fx = fy = fz = R(0);
        if (active) {
            const V4 p = buf[i];
            bool o = false;
            for_each_candidate([&](int j) {
                R dx, dy, dz;
                const R r2 = pair_r2<R>(p.x, p.y, p.z, buf[j], k, dx, dy, dz);
                if (ov && r2 <= k.rc2 && r2 <= hs2v) o = true;
                if (sizeof(R) == 8 && !(r2 <= k.rc2)) return;
                R ir2, u, ir6;
                R fs = pair_fs<R>(r2, k, ir2, u, ir6);
                fs = (r2 <= k.rc2) ? fs : R(0);
                fx = fma_r(fs, dx, fx);
                fy = fma_r(fs, dy, fy);
                fz = fma_r(fs, dz, fz);
            });
            if (ov) *ov |= o;
        }
        group_sum(fx, fy, fz);
    }

    // (H(x) v)_i with v given per particle in vbuf (own value vi).
    __device__ void hvp(const V4* __restrict__ buf, const V4* __restrict__ vbuf, R vix, R viy,
                        R viz, const LJK<R>& k, R& hx, R& hy, R& hz) const
    {
        hx = hy = hz = R(0);
        if (active) {
            const V4 p = buf[i];
            for_each_candidate([&](int j) {
                R dx, dy, dz;
                const R r2 = pair_r2<R>(p.x, p.y, p.z, buf[j], k, dx, dy, dz);
                if (sizeof(R) == 8 && !(r2 <= k.rc2)) return;
                R ir2, u, ir6;
                const R fs = pair_fs<R>(r2, k, ir2, u, ir6);      // -U'(r)/r
                const R upp = ir2 * u * fma_r(k.c3, ir6, R(-7));  // U''(r)
                const bool in = r2 <= k.rc2;
                const R mA = in ? fs : R(0);                      // -(U'/r), masked
                const R Bc = in ? (upp + fs) * ir2 : R(0);        // (U'' - U'/r)/r^2, masked
                const V4 vj = vbuf[j];
                const R vx = vix - vj.x, vy = viy - vj.y, vz = viz - vj.z;
                const R bd = Bc * fma_r(dz, vz, fma_r(dy, vy, dx * vx));
                hx = fma_r(-mA, vx, fma_r(bd, dx, hx));
                hy = fma_r(-mA, vy, fma_r(bd, dy, hy));
                hz = fma_r(-mA, vz, fma_r(bd, dz, hz));
            });
        }
        group_sum(hx, hy, hz);
    }
};

template <typename R>
__device__ __forceinline__ void load_slice(vec4_t<R>* buf, const R* __restrict__ Xt, int N)
{
    for (int n = threadIdx.x; n < N; n += blockDim.x)
        buf[n] = make4<R>(__ldg(Xt + n), __ldg(Xt + N + n), __ldg(Xt + 2 * N + n));
}

// One work item: steps [t0, t1) of one chain.  Writes g_t for t0 <= t < t1 (and
// g_T when t1 == T) and the item's sum of |r_t|^2 into partials[slot].
template <typename R, bool GRAD>
__device__ __forceinline__ void lj_item(const LJItem& I, const LJSysDev<R>& S, unsigned char* smem,
                                        int nmax, const R* __restrict__ pos, R* __restrict__ grad,
                                        double* __restrict__ partials, double* red,
                                        const R* __restrict__ hs2, int* __restrict__ overlap)
{
    bool ov = false;  // hard-sphere path bias (hs2 non-null): a pair within its slice's radius
    using V4 = vec4_t<R>;
    const int N = S.N;
    V4* xa = reinterpret_cast<V4*>(smem);
    V4* xb = xa + nmax;
    V4* rv = xb + nmax;
    LJBlock<R> L;
    L.init(N, S.tpp, S.lg_tpp, S.cap, reinterpret_cast<uint16_t*>(rv + nmax));
    const LJK<R>& k = S.k;

    const int t0 = I.t0, t1 = I.t1, T = S.T;
    const int s = 3 * N;
    const R* __restrict__ X = pos + S.off + (long long)I.chain * S.chain_len;
    R* __restrict__ G = GRAD ? grad + S.off + (long long)I.chain * S.chain_len : nullptr;
    const int i = L.i;
    const bool lead = L.active && L.q == 0;

    R rpx = R(0), rpy = R(0), rpz = R(0);  // r_{t-1}
    double acc = 0.0;

    // Prologue: list at the first slice the item touches; r_{t0-1} if t0 > 0.
    const int tf = t0 > 0 ? t0 - 1 : t0;
    load_slice<R>(xa, X + (long long)tf * s, N);
    __syncthreads();
    L.build(xa, k);
    if (t0 > 0) {
        load_slice<R>(xb, X + (long long)t0 * s, N);
        __syncthreads();
        R fx, fy, fz;
        L.force(xa, k, fx, fy, fz);
        if (L.active) {
            const V4 p0 = xa[i], p1 = xb[i];
            rpx = fma_r(-k.a, fx, p1.x - p0.x);
            rpy = fma_r(-k.a, fy, p1.y - p0.y);
            rpz = fma_r(-k.a, fz, p1.z - p0.z);
        }
        __syncthreads();
        V4* tmp = xa;
        xa = xb;
        xb = tmp;
    }
    load_slice<R>(xb, X + (long long)(t0 + 1) * s, N);
    __syncthreads();

    for (int t = t0; t < t1; ++t) {
        // Prefetch x_{t+2} into registers while this slice is processed.
        const bool pf = (t + 1 < t1) && (int)threadIdx.x < N;
        R px = R(0), py = R(0), pz = R(0);
        if (pf) {
            const R* Xn = X + (long long)(t + 2) * s;
            const bool ok = PAMD_OK_IDX((long long)(t + 2) * s + 2 * N + threadIdx.x, (long long)(T + 1) * s);
            px = ok ? __ldg(Xn + threadIdx.x) : R(0);
            py = ok ? __ldg(Xn + N + threadIdx.x) : R(0);
            pz = ok ? __ldg(Xn + 2 * N + threadIdx.x) : R(0);
        }
        if (__syncthreads_or(L.moved(xa, k))) L.build(xa, k);

        R fx, fy, fz;
        if (hs2)
            L.force(xa, k, fx, fy, fz, hs2[S.hs_off + t], &ov);
        else
            L.force(xa, k, fx, fy, fz);
        R rx = R(0), ry = R(0), rz = R(0);
        if (L.active) {
            const V4 p0 = xa[i], p1 = xb[i];
            rx = fma_r(-k.a, fx, p1.x - p0.x);
            ry = fma_r(-k.a, fy, p1.y - p0.y);
            rz = fma_r(-k.a, fz, p1.z - p0.z);
            if (L.q == 0) {
                rv[i] = make4<R>(rx, ry, rz);
                acc += (double)fma_r(rz, rz, fma_r(ry, ry, rx * rx));
            }
        }
        if (GRAD) {
            __syncthreads();
            R hx, hy, hz;
            L.hvp(xa, rv, rx, ry, rz, k, hx, hy, hz);
            if (lead) {
                R* Gt = G + (long long)t * s;
                if (PAMD_OK_IDX((long long)t * s + 2 * N + i, (long long)(T + 1) * s)) {
                    Gt[i] = fma_r(k.a, hx, rpx - rx) * k.ginv;
                    Gt[N + i] = fma_r(k.a, hy, rpy - ry) * k.ginv;
                    Gt[2 * N + i] = fma_r(k.a, hz, rpz - rz) * k.ginv;
                }
            }
        }
        rpx = rx;
        rpy = ry;
        rpz = rz;
        __syncthreads();
        V4* tmp = xa;
        xa = xb;
        xb = tmp;
        if (pf) xb[threadIdx.x] = make4<R>(px, py, pz);
    }
    if (GRAD && t1 == T && S.write_nose && lead) {
        R* Gt = G + (long long)T * s;
        if (PAMD_OK_IDX((long long)T * s + 2 * N + i, (long long)(T + 1) * s)) {
            Gt[i] = rpx * k.ginv;
            Gt[N + i] = rpy * k.ginv;
            Gt[2 * N + i] = rpz * k.ginv;
        }
    }
    if (hs2 && __syncthreads_or(ov) && threadIdx.x == 0) atomicOr(overlap + S.chain0 + I.chain, 1);
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[I.slot] = tot;
}

// Persistent grid: each CTA takes items from *counter until none is left.
template <typename R, bool GRAD, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 512 ? 2 : 1))
    lj_action_kernel(const LJItem* __restrict__ items, int n_items,
                     const LJSysDev<R>* __restrict__ systems, int nmax, const R* __restrict__ pos,
                     R* __restrict__ grad, double* __restrict__ partials, int* __restrict__ counter,
                     const R* __restrict__ hs2, int* __restrict__ overlap)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const LJItem I = items[it];
        const LJSysDev<R> S = systems[I.sys];
        lj_item<R, GRAD>(I, S, smem_raw, nmax, pos, grad, partials, red, hs2, overlap);
    }
}

size_t lj_smem_bytes(int nmax, int NT, int cap_lane, bool fp64)
{
    const size_t v4 = fp64 ? sizeof(double4a) : sizeof(float4);
    return 3 * (size_t)nmax * v4 + (size_t)cap_lane * NT * sizeof(uint16_t);
}

template <typename R, bool GRAD>
static auto lj_kernel_ptr(int NT)
{
    return NT <= 512 ? lj_action_kernel<R, GRAD, 512> : lj_action_kernel<R, GRAD, 1024>;
}

template <typename R>
int lj_blocks_per_sm(int NT, size_t smem, bool with_grad)
{
    auto kern = with_grad ? lj_kernel_ptr<R, true>(NT) : lj_kernel_ptr<R, false>(NT);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename R>
cudaError_t launch_lj_items(const LJItem* items, int n_items, const void* sys_table, int nmax,
                            const R* pos, R* grad, double* partials, int* counter, int NT,
                            size_t smem, int grid, bool with_grad, cudaStream_t st, const R* hs2,
                            int* overlap)
{
    if (n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    auto kern = with_grad ? lj_kernel_ptr<R, true>(NT) : lj_kernel_ptr<R, false>(NT);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, smem, st>>>(items, n_items, static_cast<const LJSysDev<R>*>(sys_table), nmax,
                                 pos, grad, partials, counter, hs2, overlap);
    return cudaGetLastError();
}

template int lj_blocks_per_sm<float>(int, size_t, bool);
template int lj_blocks_per_sm<double>(int, size_t, bool);
template cudaError_t launch_lj_items<float>(const LJItem*, int, const void*, int, const float*,
                                            float*, double*, int*, int, size_t, int, bool,
                                            cudaStream_t, const float*, int*);
template cudaError_t launch_lj_items<double>(const LJItem*, int, const void*, int, const double*,
                                             double*, double*, int*, int, size_t, int, bool,
                                             cudaStream_t, const double*, int*);

// ------------------------------------------------------------------ hard-sphere path bias
// Squared hard-sphere radii in the path's precision (a radius <= 0: no bias at
// that slice, -1).
template <typename R>
__global__ void hs_square_kernel(const double* __restrict__ sigma, R* __restrict__ hs2, long long n)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double v = sigma[q];
    hs2[q] = v > 0.0 ? (R)(v * v) : R(-1);
}

template <typename R>
cudaError_t launch_hs_square(const double* sigma, R* hs2, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    hs_square_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sigma, hs2, n);
    return cudaGetLastError();
}

// The bias at slice t of every chain of one system, all pairs (the force walks
// test the slices whose forces they evaluate, 0..T-1; this covers the nose T):
// a pair i < j within the cutoff and within the squared radius hs2[t] sets the
// chain's overlap flag.  One CTA per chain; the pair vector by pair_r2's rule.
template <typename R>
__global__ void lj_hs_slice_kernel(const R* __restrict__ pos, int N, int T, int t, long long sys_offset,
                                   int chain0, const LJK<R> k, const R* __restrict__ hs2t,
                                   int* __restrict__ overlap)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    vec4_t<R>* xs = reinterpret_cast<vec4_t<R>*>(smem_raw);
    const int chain = blockIdx.x, s = 3 * N;
    const R h2 = *hs2t;
    if (!(h2 >= R(0))) return;  // no bias at this slice (uniform over the block)
    load_slice<R>(xs, pos + sys_offset + (long long)chain * (T + 1) * s + (long long)t * s, N);
    __syncthreads();
    bool o = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const vec4_t<R> p = xs[i];
        for (int j = i + 1; j < N; ++j) {
            R dx, dy, dz;
            const R r2 = pair_r2<R>(p.x, p.y, p.z, xs[j], k, dx, dy, dz);
            o |= (r2 <= k.rc2) & (r2 <= h2);
        }
    }
    if (__syncthreads_or(o) && threadIdx.x == 0) atomicOr(overlap + chain0 + chain, 1);
}

template <typename R>
cudaError_t launch_lj_hs_slice(const R* pos, const void* sys_entry_host, int n_chains, int t,
                               const R* hs2t, int* overlap, cudaStream_t st)
{
    const LJSysDev<R> S = *static_cast<const LJSysDev<R>*>(sys_entry_host);
    if (n_chains <= 0) return cudaSuccess;
    const size_t smem = sizeof(vec4_t<R>) * (size_t)S.N;
    auto kern = lj_hs_slice_kernel<R>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return cudaErrorInvalidValue;
    kern<<<n_chains, 256, smem, st>>>(pos, S.N, S.T, t, S.off, S.chain0, S.k, hs2t, overlap);
    return cudaGetLastError();
}

// A chain whose path has an overlapping pair gets S = +inf.
__global__ void hs_fixup_kernel(double* __restrict__ S, const int* __restrict__ overlap, int n)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n && overlap[c]) S[c] = __longlong_as_double(0x7ff0000000000000LL);
}

cudaError_t launch_hs_fixup(double* S, const int* overlap, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    hs_fixup_kernel<<<(n + 255) / 256, 256, 0, st>>>(S, overlap, n);
    return cudaGetLastError();
}

template cudaError_t launch_hs_square<float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_hs_square<double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_lj_hs_slice<float>(const float*, const void*, int, int, const float*,
                                               int*, cudaStream_t);
template cudaError_t launch_lj_hs_slice<double>(const double*, const void*, int, int, const double*,
                                                int*, cudaStream_t);

// ------------------------------------------------------------------ Euler-Maruyama (Eq. (2))
// One CTA per chain, sequential in time; forces as in the action kernel.
template <typename R>
__global__ void __launch_bounds__(1024)
    lj_euler_kernel(R* __restrict__ pos, const R* __restrict__ noise, const LJSysDev<R> S,
                    int chain0, uint64_t seed, uint64_t counter)
{
    using V4 = vec4_t<R>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int N = S.N, T = S.T;
    V4* xa = reinterpret_cast<V4*>(smem_raw);
    V4* xb = xa + N;
    LJBlock<R> L;
    L.init(N, S.tpp, S.lg_tpp, S.cap, reinterpret_cast<uint16_t*>(xb + 2 * N));
    const LJK<R>& k = S.k;
    const int chain = blockIdx.x, s = 3 * N, i = L.i;
    R* X = pos + S.off + chain * S.chain_len;
    const R* Z = noise ? noise + S.off + chain * S.chain_len : nullptr;
    load_slice<R>(xa, X, N);
    __syncthreads();
    L.build(xa, k);
    for (int t = 0; t < T; ++t) {
        if (__syncthreads_or(L.moved(xa, k))) L.build(xa, k);
        R f[3];
        L.force(xa, k, f[0], f[1], f[2]);
        if (L.active && L.q == 0) {
            const V4 p = xa[i];
            const R xo[3] = {p.x, p.y, p.z};
            R xn[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long e = (long long)(t + 1) * s + c * N + i;
                R z;
                if (Z) {
                    z = Z[e];
                } else {
                    const float4 w = philox_normals4(seed, counter, kStreamEuler,
                                                     (uint32_t)(chain0 + chain), (uint32_t)(e >> 2));
                    z = (R)pick4(w, (int)(e & 3));
                }
                xn[c] = xo[c] + fma_r(k.a, f[c], k.sig_em * z);
                X[e] = xn[c];
            }
            xb[i] = make4<R>(xn[0], xn[1], xn[2]);
        }
        __syncthreads();
        V4* tmp = xa;
        xa = xb;
        xb = tmp;
    }
}

template <typename R>
cudaError_t launch_lj_euler(R* pos, const R* noise, const void* sys_entry_host, int NT, size_t smem,
                            int n_chains, int chain0, uint64_t seed, uint64_t counter,
                            cudaStream_t st)
{
    if (n_chains <= 0) return cudaSuccess;
    const LJSysDev<R> S = *static_cast<const LJSysDev<R>*>(sys_entry_host);
    if (S.T <= 0) return cudaSuccess;
    auto kern = lj_euler_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_chains, NT, smem, st>>>(pos, noise, S, chain0, seed, counter);
    return cudaGetLastError();
}

template cudaError_t launch_lj_euler<float>(float*, const float*, const void*, int, size_t, int, int,
                                            uint64_t, uint64_t, cudaStream_t);
template cudaError_t launch_lj_euler<double>(double*, const double*, const void*, int, size_t, int,
                                             int, uint64_t, uint64_t, cudaStream_t);

// ------------------------------------------------------------------ pair-count diagnostic
// Ordered in-cutoff pairs per slice, single-precision rule, all pairs.
__global__ void __launch_bounds__(256)
    lj_pair_count_kernel(const float* __restrict__ pos, long long* __restrict__ counts, int N, int T,
                         long long sys_offset, const LJK<float> k)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double red[8];
    float4* xs = reinterpret_cast<float4*>(smem_raw);
    const int t = blockIdx.x, chain = blockIdx.y, s = 3 * N;
    const float* Xt = pos + sys_offset + (long long)chain * (T + 1) * s + (long long)t * s;
    load_slice<float>(xs, Xt, N);
    __syncthreads();
    long long c = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float4 p = xs[i];
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            float dx, dy, dz;
            if (pair_r2<float>(p.x, p.y, p.z, xs[j], k, dx, dy, dz) <= k.rc2) ++c;
        }
    }
    const double tot = block_sum((double)c, red);
    if (threadIdx.x == 0) counts[(long long)chain * (T + 1) + t] = (long long)tot;
}

cudaError_t launch_lj_pair_counts(const float* pos, long long* counts, int N, int T, int n_chains,
                                  long long sys_offset, double L, double rc, cudaStream_t st)
{
    LJConst c{};
    c.L = L;
    c.rc = rc;
    c.eps = 1.0;
    c.sigma = 1.0;
    const LJK<float> k = make_lj_consts<float>(c, 0.0);
    const size_t smem = (size_t)N * sizeof(float4);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(lj_pair_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    lj_pair_count_kernel<<<dim3(T + 1, n_chains), 256, smem, st>>>(pos, counts, N, T, sys_offset, k);
    return cudaGetLastError();
}

PAMD_DEBUG_FETCHER(lj)

}  // namespace pamd
