// lj_paired.cu -- single-precision Lennard-Jones path action and adjoint with two
// consecutive steps per thread.
//
// The forces of different time slices are independent (Sec. II.B), and along a
// Brownian path a particle moves ~sqrt(2 D dt) per step, so the neighbours of
// particle i are the same at steps t and t+1.  This kernel therefore evaluates
// every pair (i, j) at both steps at once: positions of the two slices sit side
// by side in shared memory, and every floating-point operation of the pair
// geometry, the force and the Hessian-vector product is one packed f32x2
// instruction acting on (step t, step t+1).  Each half of a packed operation is
// an IEEE single-precision operation, so the result of a step does not depend on
// the step it is paired with.
//
// Formulas (paper Eqs. (3), (11); the cut-and-force-shifted pair potential,
// u = 4 eps [(s/r)^12 - (s/r)^6], ir2 = 1/r^2, ir6 = ir2^3, w = 24 eps s^6 ir6 ir2):
//   fs    = -U'(r)/r = w (2 s^6 ir6 - 1) + u'(rc)/r
//   Bc    = (U''(r) - U'(r)/r)/r^2 = [w (26 s^6 ir6 - 7) + fs] ir2
//   F_i   = sum_j fs r_ij,                          r_ij = x_i - x_j (minimum image)
//   r_t   = x_{t+1} - x_t - a F(x_t),               a = beta D dt
//   (Hv)_i = sum_j [ -fs v_ij + Bc (r_ij . v_ij) r_ij ],   v_ij = v_i - v_j
//   g_t   = [r_{t-1} - r_t + a H(x_t) r_t] / (2 D dt),  r_{-1} = r_T = 0
//   S     = sum_t |r_t|^2 / (4 D dt)   (per-item partial sums in FP64)
// A pair outside the cutoff gets r^2 = +inf, which makes every coefficient an
// exact zero (rsqrt(+inf) = +0).
//
// Work decomposition: a persistent grid pulls (system, chain, tile of steps)
// items from an atomic queue.  Within an item the steps are walked in pairs
// (a, a+1).  An item that does not start at step 0 begins with the pair
// (t0-1, t0), whose first half only supplies the residual r_{t0-1}.
//
// Neighbour lists.  An item knows every slice it will visit, so its steps are
// cut into windows of W steps and each window gets a list that is exact for all
// of its slices: with reference positions x_c at the window's middle slice and
// delta_i = max over the window's slices of |x_t(i) - x_c(i)| (read from the
// path), a pair within rc at any slice of the window satisfies
// |r_ij(x_c)| <= rc + delta_i + delta_j (triangle inequality; the minimum image
// at x_c is no longer than the image that is within rc at t), so listing those
// pairs suffices.  The window lists are built from an outer list made once per
// item by the same rule with item-wide margins (reference at the item's middle
// slice), which holds every pair that any of the item's windows can need; it
// sits in global memory (one region per CTA, L2-resident).  A particle whose
// outer list overflows builds its window lists from all candidates; one whose
// window list overflows scans all candidates.  Candidates are visited in one
// fixed order in every case -- by class (j - tid) mod 8, then by increasing j --
// so each force and Hessian sum runs over the in-cutoff pairs in one order
// whatever the tiling, window or list capacity, and the results are bitwise
// independent of them.  The class order spreads a warp's gathers over the
// shared-memory banks: at the start of a walk the eight lanes of a quarter warp
// read particles j of eight different residues mod 8, i.e. eight different
// 16-byte bank groups, and they drift apart only as their classes run out.
#include <type_traits>

#include "pamd_internal.cuh"

namespace pamd {

namespace {

// ------------------------------------------------------------------ packed f32x2 arithmetic
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding: b * (-1) + a is exact before rounding.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, pk(-1.0f), a); }

__device__ __forceinline__ float rsqrt_approx(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Slot o8 = 8 j of a per-particle shared-memory array; a PAMD_DEBUG build checks
// j < NMAX and sends a bad access to the sink.
#ifdef PAMD_DEBUG
#define PAMD_SLOT(T, addr, o8) \
    (*(debug_in_bounds((o8) >> 3, NMAX, __LINE__) ? reinterpret_cast<T*>(addr) \
                                                   : reinterpret_cast<T*>(g_pamd_sink)))
#else
#define PAMD_SLOT(T, addr, o8) (*reinterpret_cast<T*>(addr))
#endif

// ------------------------------------------------------------------ shared-memory layout
// For a block of up to NMAX particles (NMAX = the kernel's maximum block size):
//   [0, 16 NMAX)        xy[j]  = {x_a, x_b, y_a, y_b} of the positions
//   [16 NMAX, 32 NMAX)  rxy[j] = the same for the residuals
//   [32 NMAX, 40 NMAX)  z[j]   = {z_a, z_b} of the positions
//   [40 NMAX, 48 NMAX)  rz[j]  = the same for the residuals
//   [48 NMAX, ...)      neighbour lists, two uint16 entries per 32-bit word
// Two arrays per quantity (16- and 8-byte strides) let a gather of random
// particles spread over all banks.  A list entry is the byte offset 8 j, so
// every array is addressed from it with a constant displacement.
template <int NMAX>
struct Smem {
    unsigned char* base;
    __device__ float4& xy(int o8) const { return PAMD_SLOT(float4, base + 2 * o8, o8); }
    __device__ float4& rxy(int o8) const
    {
        return PAMD_SLOT(float4, base + 16 * NMAX + 2 * o8, o8);
    }
    __device__ float2& z(int o8) const { return PAMD_SLOT(float2, base + 32 * NMAX + o8, o8); }
    __device__ float2& rz(int o8) const { return PAMD_SLOT(float2, base + 40 * NMAX + o8, o8); }
    __device__ uint32_t* list() const { return reinterpret_cast<uint32_t*>(base + 48 * NMAX); }
    // staging area of list references {x, y, z, delta}: the residual array
    __device__ float4& ref(int o8) const { return rxy(o8); }
};

// Layout of the pipelined form (see paired_item_pipe): two position buffers, the
// residuals and a separate staging area (the residuals stay live across list builds).
//   [0, 32 NMAX)        xy of buffers 0 and 1
//   [32 NMAX, 48 NMAX)  rxy
//   [48 NMAX, 64 NMAX)  staged references {x, y, z, delta}
//   [64 NMAX, 80 NMAX)  zz[j] = {z_a, z_b} of buffer 0, then of buffer 1
//   [80 NMAX, 88 NMAX)  rz
//   [88 NMAX, ...)      neighbour lists
// A walk that uses both buffers reads both z pairs with one 16-byte load.
template <int NMAX>
struct SmemP {
    unsigned char* base;
    __device__ float4& xy(int buf, int o8) const
    {
        return PAMD_SLOT(float4, base + 16 * NMAX * buf + 2 * o8, o8);
    }
    __device__ float2& z(int buf, int o8) const
    {
        return PAMD_SLOT(float2, base + 64 * NMAX + 2 * o8 + 8 * buf, o8);
    }
    __device__ float4& zz(int o8) const { return PAMD_SLOT(float4, base + 64 * NMAX + 2 * o8, o8); }
    __device__ float4& rxy(int o8) const { return PAMD_SLOT(float4, base + 32 * NMAX + 2 * o8, o8); }
    __device__ float2& rz(int o8) const { return PAMD_SLOT(float2, base + 80 * NMAX + o8, o8); }
    __device__ float4& ref(int o8) const { return PAMD_SLOT(float4, base + 48 * NMAX + 2 * o8, o8); }
    __device__ uint32_t* list() const { return reinterpret_cast<uint32_t*>(base + 88 * NMAX); }
};

// Packed constants of one system (built per item from the per-system table).
struct K2 {
    float2 nL, iL, mag, nmag, c12, nc1, c8, nc23, duc, nduc;
    float rc2, rcm, a, ginv, hb, iLs;
    __device__ explicit K2(const LJK<float>& k)
    {
        nL = pk(-k.L);
        iL = pk(k.iL);
        mag = pk(12582912.0f);  // 1.5 * 2^23: adding it rounds to an integer
        nmag = pk(-12582912.0f);
        c12 = pk(k.c12);
        nc1 = pk(k.nc1);
        c8 = pk(k.c8);
        nc23 = pk(k.nc23);
        duc = pk(k.duc);
        nduc = pk(-k.duc);
        rc2 = k.rc2;
        rcm = k.rcm;
        a = k.a;
        ginv = k.ginv;
        hb = k.hb;
        iLs = k.iL;
    }
};

// Minimum-image shift of one pair-vector component, round(d / L), by the same
// single-precision rule as the packed form below.
__device__ __forceinline__ float image_shift(float d, const K2& k)
{
    return __fadd_rn(__fmaf_rn(d, k.iLs, 12582912.0f), -12582912.0f);
}

// Pair vector d = x_i - x_j of (step a, step b) by the single-precision
// minimum-image rule  d = x_i - x_j;  d = fma(-L, round(d * (1/L)), d),  the shift
// rounded for each step.
__device__ __forceinline__ void pair_vec(float2 xi, float2 yi, float2 zi, float4 pxy, float2 pz,
                                         const K2& k, float2& dx, float2& dy, float2& dz)
{
    dx = sub2(xi, pk(pxy.x, pxy.y));
    dy = sub2(yi, pk(pxy.z, pxy.w));
    dz = sub2(zi, pz);
    dx = fma2(k.nL, add2(fma2(dx, k.iL, k.mag), k.nmag), dx);
    dy = fma2(k.nL, add2(fma2(dy, k.iL, k.mag), k.nmag), dy);
    dz = fma2(k.nL, add2(fma2(dz, k.iL, k.mag), k.nmag), dz);
}

// The same rule with the shift of step a applied to both steps; the shifts are
// returned for reuse.  Within a window whose particles all stay within delta_max
// of the reference, a pair inside the cutoff at any of its slices has one
// nearest image whenever rc + 4 delta_max < L/2, and the shift rounded at any
// slice is that image's: the result is then bitwise that of pair_vec (a pair
// outside the cutoff stays outside, since the rounded shift gives the nearest
// image of each component).
__device__ __forceinline__ void pair_vec_shift(float2 xi, float2 yi, float2 zi, float4 pxy, float2 pz,
                                               const K2& k, float2& dx, float2& dy, float2& dz,
                                               float& sx, float& sy, float& sz)
{
    dx = sub2(xi, pk(pxy.x, pxy.y));
    dy = sub2(yi, pk(pxy.z, pxy.w));
    dz = sub2(zi, pz);
    sx = image_shift(dx.x, k);
    sy = image_shift(dy.x, k);
    sz = image_shift(dz.x, k);
    dx = fma2(k.nL, pk(sx), dx);
    dy = fma2(k.nL, pk(sy), dy);
    dz = fma2(k.nL, pk(sz), dz);
}

// ... with shifts already known (from another pair of slices of the same window).
__device__ __forceinline__ void pair_vec_given(float2 xi, float2 yi, float2 zi, float4 pxy, float2 pz,
                                               const K2& k, float sx, float sy, float sz, float2& dx,
                                               float2& dy, float2& dz)
{
    dx = fma2(k.nL, pk(sx), sub2(xi, pk(pxy.x, pxy.y)));
    dy = fma2(k.nL, pk(sy), sub2(yi, pk(pxy.z, pxy.w)));
    dz = fma2(k.nL, pk(sz), sub2(zi, pz));
}

template <bool SK>
__device__ __forceinline__ void pair_vec_sel(float2 xi, float2 yi, float2 zi, float4 pxy, float2 pz,
                                             const K2& k, float2& dx, float2& dy, float2& dz)
{
    if (SK) {
        float sx, sy, sz;
        pair_vec_shift(xi, yi, zi, pxy, pz, k, dx, dy, dz, sx, sy, sz);
    } else {
        pair_vec(xi, yi, zi, pxy, pz, k, dx, dy, dz);
    }
}

// r^2 = fma(dz,dz,fma(dy,dy,dx*dx)), +inf for a half outside the cutoff.
__device__ __forceinline__ float2 pair_r2(float2 dx, float2 dy, float2 dz, const K2& k)
{
    float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const float inf = __int_as_float(0x7f800000);
    r2.x = r2.x <= k.rc2 ? r2.x : inf;
    r2.y = r2.y <= k.rc2 ? r2.y : inf;
    return r2;
}

// fs = -U'(r)/r = ir8 (c12 ir6 - c1) + u'(rc)/r, with 1/r, r^-2, r^-6, r^-8 for the
// Hessian coefficient.  r^2 = +inf gives exact zeros.
__device__ __forceinline__ float2 pair_fs(float2 r2, const K2& k, float2& ri, float2& ir2,
                                          float2& ir6, float2& ir8)
{
    ri = pk(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    ir2 = mul2(ri, ri);
    const float2 ir4 = mul2(ir2, ir2);
    ir6 = mul2(ir4, ir2);
    ir8 = mul2(ir4, ir4);
    return fma2(ir8, fma2(k.c12, ir6, k.nc1), mul2(k.duc, ri));
}

// -(U''(r) - U'(r)/r) / r^2 = [ir8 (8 c1 - c1 (c2 + c3) ir6) - u'(rc)/r] r^-2.
__device__ __forceinline__ float2 pair_nbc(float2 ri, float2 ir2, float2 ir6, float2 ir8, const K2& k)
{
    return mul2(fma2(ir8, fma2(k.nc23, ir6, k.c8), mul2(k.nduc, ri)), ir2);
}

// One pair's Hessian-vector term, added to h:  (H v)_i gets
//   sum_j [-fs v_ij + Bc (d . v_ij) d] = sum_j [fs w + (-Bc) (d . w) d],  w = v_j - v_i.
__device__ __forceinline__ void hvp_term(float2 dx, float2 dy, float2 dz, float2 fs, float2 nbc,
                                         float4 vj, float2 vjz, float2 vix, float2 viy, float2 viz,
                                         float2& hx, float2& hy, float2& hz)
{
    const float2 wx = sub2(pk(vj.x, vj.y), vix);
    const float2 wy = sub2(pk(vj.z, vj.w), viy);
    const float2 wz = sub2(vjz, viz);
    const float2 bd = mul2(nbc, fma2(dz, wz, fma2(dy, wy, mul2(dx, wx))));
    hx = fma2(fs, wx, fma2(bd, dx, hx));
    hy = fma2(fs, wy, fma2(bd, dy, hy));
    hz = fma2(fs, wz, fma2(bd, dz, hz));
}

// The particle a thread works for, its list, and the candidate loop.
template <int NMAX>
struct PairList {
    int N, NT, tid, i, q, tpp, cap, cnt, ocap, ocnt;
    bool active, ovf, oovf;
    uint32_t* nbr;
    uint32_t* outer;  // this CTA's outer lists (global memory), same word layout

    __device__ void init(int n, int tpp_, int lg, int cap_, uint32_t* list, int ocap_,
                         uint32_t* outer_)
    {
        ocap = ocap_ & ~1;
        outer = outer_;
        ocnt = 0;
        oovf = true;
        N = n;
        NT = blockDim.x;
        tid = threadIdx.x;
        tpp = tpp_;
        i = tid >> lg;
        q = tid & (tpp_ - 1);
        active = i < n;
        cap = cap_ & ~1;
        nbr = list;
        cnt = 0;
        ovf = false;
    }

    // Candidate order.  This thread's candidates are j = q (mod tpp); they are
    // visited class by class, class c holding j = tid + c (mod 8) for c = 0,
    // cstep(), ... < 8, each class in increasing j (stride cls_stride()).  For
    // tpp >= 8 all of them lie in class 0 (j = q = tid mod 8).
    __device__ __forceinline__ int cstep() const { return tpp < 8 ? tpp : 8; }
    __device__ __forceinline__ int cls_stride() const { return tpp < 8 ? 8 : tpp; }
    __device__ __forceinline__ int cls_first(int c) const { return tpp < 8 ? ((tid + c) & 7) : q; }

    // Calls f(j1, j2) over this thread's candidates in order, two at a time within
    // a class (j2 = j1 + cls_stride(), possibly >= N).
    template <typename F>
    __device__ __forceinline__ void candidate_pairs(F&& f) const
    {
        const int st = cls_stride();
        for (int c = 0; c < 8; c += cstep())
            for (int j = cls_first(c); j < N; j += 2 * st) f(j, j + st);
    }

    // Entry c of this thread is half (c & 1) of word (c >> 1) * NT + tid.
    __device__ __forceinline__ void put(int c, int o8) const
    {
        if (PAMD_OK_IDX((c >> 1) * NT + tid, (cap >> 1) * NT))
            reinterpret_cast<uint16_t*>(nbr + (c >> 1) * NT + tid)[c & 1] = (uint16_t)o8;
    }

    // Pair test at the staged reference {x, y, z, delta} (residual array) of
    // two candidates: r_ij(x_c) <= rc + delta_i + delta_j for each half.
    template <class SM>
    __device__ __forceinline__ void test2(const SM& P, const K2& k, float4 pi, int o1, int o2,
                                          bool& in1, bool& in2) const
    {
        const float4 A = P.ref(o1), B = P.ref(o2);
        float2 dx = sub2(pk(pi.x), pk(A.x, B.x));
        float2 dy = sub2(pk(pi.y), pk(A.y, B.y));
        float2 dz = sub2(pk(pi.z), pk(A.z, B.z));
        dx = fma2(k.nL, add2(fma2(dx, k.iL, k.mag), k.nmag), dx);
        dy = fma2(k.nL, add2(fma2(dy, k.iL, k.mag), k.nmag), dy);
        dz = fma2(k.nL, add2(fma2(dz, k.iL, k.mag), k.nmag), dz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 lim = add2(pk(k.rcm + pi.w), pk(A.w, B.w));
        const float2 lim2 = mul2(lim, lim);
        in1 = r2.x <= lim2.x;
        in2 = r2.y <= lim2.y;
    }

    // Outer list of the item (reference and item-wide margins staged): all
    // candidates, in the candidate order.
    template <class SM>
    __device__ void build_outer(const SM& P, const K2& k)
    {
        ocnt = 0;
        oovf = true;
        if (!active) return;
        const float4 pi = P.ref(8 * i);
        int c = 0;
        auto add = [&](bool in, int o8) {
            if (in) {
                if (c < ocap && PAMD_OK_IDX((c >> 1) * NT + tid, (ocap >> 1) * NT))
                    reinterpret_cast<uint16_t*>(outer + (c >> 1) * NT + tid)[c & 1] = (uint16_t)o8;
                ++c;
            }
        };
        candidate_pairs([&](int j, int j2) {
            const int j2c = j2 < N ? j2 : j;
            bool in1, in2;
            test2(P, k, pi, 8 * j, 8 * j2c, in1, in2);
            add(j != i && in1, 8 * j);
            add(j2 < N && j2 != i && in2, 8 * j2);
        });
        ocnt = c;
        oovf = c > ocap;
    }

    // Window list (window reference and margins staged) from the outer list,
    // or from all candidates if the outer list overflowed; candidate order.
    template <class SM>
    __device__ void build(const SM& P, const K2& k)
    {
        cnt = 0;
        ovf = false;
        if (!active) return;
        const float4 pi = P.ref(8 * i);
        int c = 0;
        auto add = [&](bool in, int o8) {
            if (in) {
                if (c < cap) put(c, o8);
                ++c;
            }
        };
        if (!oovf) {
            const uint32_t* w = outer + tid;
            for (int m = 0; m < ocnt; m += 2, w += NT) {
                const uint32_t v = PAMD_OK_IDX((m >> 1) * NT + tid, (ocap >> 1) * NT) ? *w : 0u;
                const int o1 = (int)(v & 0xFFFFu);
                const bool two = m + 1 < ocnt;
                const int o2 = two ? (int)(v >> 16) : o1;
                bool in1, in2;
                test2(P, k, pi, o1, o2, in1, in2);
                add(in1, o1);
                add(two && in2, o2);
            }
        } else {
            candidate_pairs([&](int j, int j2) {
                const int j2c = j2 < N ? j2 : j;
                bool in1, in2;
                test2(P, k, pi, 8 * j, 8 * j2c, in1, in2);
                add(j != i && in1, 8 * j);
                add(j2 < N && j2 != i && in2, 8 * j2);
            });
        }
        cnt = c;
        ovf = c > cap;
    }

    // Calls f(8 j) for the candidates j of particle i, in the candidate order.
    template <typename F>
    __device__ __forceinline__ void for_each_candidate(F&& f) const
    {
        if (!active) return;
        if (!ovf) {
            const uint32_t* w = nbr + tid;
            int m = 0;
            for (; m + 1 < cnt; m += 2, w += NT) {
                const uint32_t v = PAMD_OK_IDX((m >> 1) * NT + tid, (cap >> 1) * NT) ? *w : 0u;
                f((int)(v & 0xFFFFu));
                f((int)(v >> 16));
            }
            if (m < cnt) f((int)((PAMD_OK_IDX((m >> 1) * NT + tid, (cap >> 1) * NT) ? *w : 0u) & 0xFFFFu));
        } else {
            const int st = cls_stride();
            for (int c = 0; c < 8; c += cstep())
                for (int j = cls_first(c); j < N; j += st)
                    if (j != i) f(8 * j);
        }
    }

    __device__ __forceinline__ void group_sum(float2& x, float2& y, float2& z) const
    {
        for (int o = tpp >> 1; o > 0; o >>= 1) {
            x = add2(x, pk(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o)));
            y = add2(y, pk(__shfl_xor_sync(0xffffffffu, y.x, o), __shfl_xor_sync(0xffffffffu, y.y, o)));
            z = add2(z, pk(__shfl_xor_sync(0xffffffffu, z.x, o), __shfl_xor_sync(0xffffffffu, z.y, o)));
        }
    }

    // F(x_a), F(x_b) of particle i (complete in every thread of the group).
    // SK: the window allows one image shift per pair (pair_vec_shift).
    // HS: also raise `ov` when a pair lies within the hard-sphere radii (squared:
    // hs2 for the two steps) of the path bias.
    template <bool SK, bool HS = false>
    __device__ void force(const Smem<NMAX>& P, const K2& k, float2& fx, float2& fy, float2& fz,
                          float2 hs2 = float2(), bool* ov = nullptr) const
    {
        fx = fy = fz = pk(0.0f);
        if (active) {
            const float4 pxy = P.xy(8 * i);
            const float2 xi = pk(pxy.x, pxy.y), yi = pk(pxy.z, pxy.w), zi = P.z(8 * i);
            bool o = false;
            for_each_candidate([&](int o8) {
                float2 dx, dy, dz, ri, ir2, ir6, ir8;
                pair_vec_sel<SK>(xi, yi, zi, P.xy(o8), P.z(o8), k, dx, dy, dz);
                const float2 r2 = pair_r2(dx, dy, dz, k);
                if (HS) o |= (r2.x <= hs2.x) | (r2.y <= hs2.y);
                const float2 fs = pair_fs(r2, k, ri, ir2, ir6, ir8);
                fx = fma2(fs, dx, fx);
                fy = fma2(fs, dy, fy);
                fz = fma2(fs, dz, fz);
            });
            if (HS) *ov |= o;
        }
        group_sum(fx, fy, fz);
    }

    // (H(x_a) v_a, H(x_b) v_b) of particle i; v is the residual array, vi its own value.
    template <bool SK>
    __device__ void hvp(const Smem<NMAX>& P, float2 vix, float2 viy, float2 viz, const K2& k,
                        float2& hx, float2& hy, float2& hz) const
    {
        hx = hy = hz = pk(0.0f);
        if (active) {
            const float4 pxy = P.xy(8 * i);
            const float2 xi = pk(pxy.x, pxy.y), yi = pk(pxy.z, pxy.w), zi = P.z(8 * i);
            for_each_candidate([&](int o8) {
                float2 dx, dy, dz, ri, ir2, ir6, ir8;
                pair_vec_sel<SK>(xi, yi, zi, P.xy(o8), P.z(o8), k, dx, dy, dz);
                const float2 fs = pair_fs(pair_r2(dx, dy, dz, k), k, ri, ir2, ir6, ir8);
                hvp_term(dx, dy, dz, fs, pair_nbc(ri, ir2, ir6, ir8, k), P.rxy(o8), P.rz(o8), vix,
                         viy, viz, hx, hy, hz);
            });
        }
        group_sum(hx, hy, hz);
    }

    // One walk over the list for the pipelined form: the Hessian-vector product of
    // the pair in buffer hb with the residual array (DO_H) and the force of the
    // pair in buffer fb (DO_F).  Each result equals that of hvp() / force() on
    // the same slices: the two chains of arithmetic are only interleaved.  SK: one
    // image shift per list entry, rounded at the first slice walked and applied to
    // all four (the window keeps every particle within (L/2 - rc)/4 of its
    // reference, so the shift is the nearest image's at each of them).
    // HS: also raise `ov` when a pair of the force walk lies within the hard-sphere
    // radii (squared: hs2 for the force pair's two steps) of the path bias.
    // HB, FB: the position buffers of the Hessian-vector and force pairs.
    template <bool DO_H, bool DO_F, bool SK, bool HS, int HB, int FB>
    __device__ void combined(const SmemP<NMAX>& P, float2 vix, float2 viy, float2 viz, const K2& k,
                             float2& hx, float2& hy, float2& hz, float2& fx, float2& fy, float2& fz,
                             float2 hs2 = float2(), bool* ov = nullptr) const
    {
        hx = hy = hz = fx = fy = fz = pk(0.0f);
        if (active) {
            bool o = false;
            const float4 hxy = P.xy(HB, 8 * i);
            const float2 hxi = pk(hxy.x, hxy.y), hyi = pk(hxy.z, hxy.w), hzi = P.z(HB, 8 * i);
            const float4 fxy = P.xy(FB, 8 * i);
            const float2 fxi = pk(fxy.x, fxy.y), fyi = pk(fxy.z, fxy.w), fzi = P.z(FB, 8 * i);
            for_each_candidate([&](int o8) {
                float sx = 0.0f, sy = 0.0f, sz = 0.0f;
                float2 hzj, fzj;  // z of particle j in the two buffers
                if (DO_H && DO_F && HB != FB) {
                    const float4 zz = P.zz(o8);
                    hzj = HB ? pk(zz.z, zz.w) : pk(zz.x, zz.y);
                    fzj = FB ? pk(zz.z, zz.w) : pk(zz.x, zz.y);
                } else {
                    if (DO_H) hzj = P.z(HB, o8);
                    if (DO_F) fzj = P.z(FB, o8);
                }
                if (DO_H) {
                    float2 dx, dy, dz, ri, ir2, ir6, ir8;
                    if (SK)
                        pair_vec_shift(hxi, hyi, hzi, P.xy(HB, o8), hzj, k, dx, dy, dz, sx, sy, sz);
                    else
                        pair_vec(hxi, hyi, hzi, P.xy(HB, o8), hzj, k, dx, dy, dz);
                    const float2 fs = pair_fs(pair_r2(dx, dy, dz, k), k, ri, ir2, ir6, ir8);
                    hvp_term(dx, dy, dz, fs, pair_nbc(ri, ir2, ir6, ir8, k), P.rxy(o8), P.rz(o8),
                             vix, viy, viz, hx, hy, hz);
                }
                if (DO_F) {
                    float2 dx, dy, dz, ri, ir2, ir6, ir8;
                    if (SK && DO_H)
                        pair_vec_given(fxi, fyi, fzi, P.xy(FB, o8), fzj, k, sx, sy, sz, dx, dy, dz);
                    else if (SK)
                        pair_vec_shift(fxi, fyi, fzi, P.xy(FB, o8), fzj, k, dx, dy, dz, sx, sy, sz);
                    else
                        pair_vec(fxi, fyi, fzi, P.xy(FB, o8), fzj, k, dx, dy, dz);
                    const float2 r2 = pair_r2(dx, dy, dz, k);
                    if (HS) o |= (r2.x <= hs2.x) | (r2.y <= hs2.y);
                    const float2 fs = pair_fs(r2, k, ri, ir2, ir6, ir8);
                    fx = fma2(fs, dx, fx);
                    fy = fma2(fs, dy, fy);
                    fz = fma2(fs, dz, fz);
                }
            });
            if (HS && DO_F) *ov |= o;
        }
        if (DO_H) group_sum(hx, hy, hz);
        if (DO_F) group_sum(fx, fy, fz);
    }
};

__device__ __forceinline__ float sq3(float x, float y, float z)
{
    return __fmaf_rn(z, z, __fmaf_rn(y, y, x * x));
}

// Stage the reference of slices [lo, hi) of a chain X -- the middle slice -- with
// each particle's margin delta = max |x_t - x_c| over them, as {x, y, z, delta},
// and raise *dmax_bits (the bits of a non-negative float, so integer order is
// float order) to the largest delta.  Called by every thread of the block.
template <class SM>
__device__ __forceinline__ void stage_reference(const SM& P, const float* __restrict__ X, int N,
                                                int lo, int hi, int* dmax_bits, int n_slices)
{
    const int s = 3 * N;
    const int c = lo + (hi - 1 - lo) / 2;
    float dmax = 0.0f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float* A = X + n;
        const float* C = A + (long long)c * s;
        const bool okc = PAMD_OK_IDX((long long)c * s + n + 2 * N, (long long)s * n_slices);
        const float cx = okc ? __ldg(C) : 0.f, cy = okc ? __ldg(C + N) : 0.f,
                    cz = okc ? __ldg(C + 2 * N) : 0.f;
        float d2 = 0.0f;
#pragma unroll 4
        for (int t = lo; t < hi; ++t) {
            const float* Q = A + (long long)t * s;
            const bool okq = PAMD_OK_IDX((long long)t * s + n + 2 * N, (long long)s * n_slices);
            const float ux = (okq ? __ldg(Q) : 0.f) - cx, uy = (okq ? __ldg(Q + N) : 0.f) - cy,
                        uz = (okq ? __ldg(Q + 2 * N) : 0.f) - cz;
            d2 = fmaxf(d2, __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, ux * ux)));
        }
        // delta rounded up: sqrt and the sums above are within a few ulp
        const float delta = __fmaf_rn(sqrtf(d2), 1.0f + 1.0e-6f, 1.0e-6f);
        P.ref(8 * n) = make_float4(cx, cy, cz, delta);
        dmax = fmaxf(dmax, delta);
    }
    const int m = __reduce_max_sync(0xffffffffu, __float_as_int(dmax));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(dmax_bits, m);
}

// Whether the window just staged allows one image shift per list entry (see
// pair_vec_shift): rc + 4 delta_max below half the box (less a rounding allowance).
__device__ __forceinline__ bool window_shared_shift(const LJSysDev<float>& S, const K2& k,
                                                    const int* dmax_bits)
{
    return S.shared_shift && k.rcm + 4.0f * __int_as_float(*dmax_bits) <= k.hb;
}

// One work item: steps [t0, t1) of one chain.
template <bool GRAD, int NMAX, bool HS>
__device__ __forceinline__ void paired_item(const LJItem& I, const LJSysDev<float>& S,
                                            unsigned char* smem, const float* __restrict__ pos,
                                            float* __restrict__ grad, double* __restrict__ partials,
                                            double* red, uint32_t* outer, int* dmax_bits,
                                            const float* __restrict__ hs2, int* __restrict__ overlap)
{
    const int N = S.N;
    const Smem<NMAX> P{smem};
    PairList<NMAX> L;
    L.init(N, S.tpp, S.lg_tpp, S.cap, P.list(), S.outer_cap, outer);
    const K2 k(S.k);
    const float2 na = pk(-k.a), ginv = pk(k.ginv);

    const int t0 = I.t0, t1 = I.t1, T = S.T;
    const int s = 3 * N;
    const float* __restrict__ X = pos + S.off + (long long)I.chain * S.chain_len;
    float* __restrict__ G = GRAD ? grad + S.off + (long long)I.chain * S.chain_len : nullptr;
    const int i = L.i;
    const bool lead = L.active && L.q == 0;
    const int ts = t0 > 0 ? t0 - 1 : t0;  // first slice of the first pair

    // Slices (a, a+1) of particle n into registers (a + 1 <= T for every pair).
    auto fetch = [&](int a, int n, float (&v)[6]) {
        const float* A = X + (long long)a * s + n;
        const bool ok = PAMD_OK_IDX((long long)(a + 1) * s + n + 2 * N, (long long)(T + 1) * s);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[2 * c] = ok ? __ldg(A + c * N) : 0.f;
            v[2 * c + 1] = ok ? __ldg(A + s + c * N) : 0.f;
        }
    };
    auto store = [&](int n, const float (&v)[6]) {
        P.xy(8 * n) = make_float4(v[0], v[1], v[2], v[3]);
        P.z(8 * n) = make_float2(v[4], v[5]);
    };

    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float v[6];
        fetch(ts, n, v);
        store(n, v);
    }
    __syncthreads();

    float rpx = 0.0f, rpy = 0.0f, rpz = 0.0f;  // r_{a-1}
    double acc = 0.0;
    const int W = max(2, S.window);
    int win_end = ts;  // slices [.., win_end) are covered by the current list
    bool sk = false;   // the current window allows one image shift per entry
    bool ov = false;   // a pair within the hard-sphere radius of its slice (HS)

    for (int a = ts; a < t1; a += 2) {
        const int b = a + 1;
        const bool hasb = b < t1;
        const bool real_a = a >= t0;
        // Prefetch the next pair's slices, and this particle's x_{b+1}.
        const bool pf = a + 2 < t1 && (int)threadIdx.x < N;
        float nv[6];
        if (pf) fetch(a + 2, threadIdx.x, nv);
        float xn = 0.0f, yn = 0.0f, zn = 0.0f;
        if (hasb && L.active) {
            const float* Xb1 = X + (long long)(b + 1) * s + i;
            const bool ok = PAMD_OK_IDX((long long)(b + 1) * s + i + 2 * N, (long long)(T + 1) * s);
            xn = ok ? __ldg(Xb1) : 0.f;
            yn = ok ? __ldg(Xb1 + N) : 0.f;
            zn = ok ? __ldg(Xb1 + 2 * N) : 0.f;
        }

        if (a == ts) {
            // Outer list over the item's slices [ts, t1].
            stage_reference(P, X, N, ts, t1 + 1, dmax_bits, T + 1);
            __syncthreads();
            L.build_outer(P, k);
            __syncthreads();  // the staged reference is replaced below
            if (threadIdx.x == 0) *dmax_bits = 0;
        }
        if (b >= win_end) {
            // New window: slices [a, e) (every pair inside has b <= t1 <= T).
            const int e = min(a + W, t1 + 1);
            stage_reference(P, X, N, a, e, dmax_bits, T + 1);
            __syncthreads();
            sk = window_shared_shift(S, k, dmax_bits);
            L.build(P, k);
            __syncthreads();  // the staged reference is overwritten by residuals below
            if (threadIdx.x == 0) *dmax_bits = 0;  // read by all before the barrier above
            win_end = e;
        }

        float2 fx, fy, fz;
        const float2 hsab = HS ? pk(hs2[S.hs_off + a], hs2[S.hs_off + b]) : float2();
        if (sk)
            L.template force<true, HS>(P, k, fx, fy, fz, hsab, &ov);
        else
            L.template force<false, HS>(P, k, fx, fy, fz, hsab, &ov);
        float2 rx = pk(0.0f), ry = pk(0.0f), rz = pk(0.0f);
        if (L.active) {
            const float4 pxy = P.xy(8 * i);
            const float2 pz = P.z(8 * i);
            // (x_b - x_a, x_{b+1} - x_b) - a (F_a, F_b); the second half only when b is a step.
            rx = fma2(na, fx, sub2(pk(pxy.y, xn), pk(pxy.x, pxy.y)));
            ry = fma2(na, fy, sub2(pk(pxy.w, yn), pk(pxy.z, pxy.w)));
            rz = fma2(na, fz, sub2(pk(pz.y, zn), pz));
            if (!hasb) rx.y = ry.y = rz.y = 0.0f;
            if (lead) {
                if (GRAD) {
                    P.rxy(8 * i) = make_float4(rx.x, rx.y, ry.x, ry.y);
                    P.rz(8 * i) = rz;
                }
                if (real_a) acc += (double)sq3(rx.x, ry.x, rz.x);
                if (hasb) acc += (double)sq3(rx.y, ry.y, rz.y);
            }
        }
        if (GRAD) {
            __syncthreads();
            float2 hx, hy, hz;
            if (sk)
                L.template hvp<true>(P, rx, ry, rz, k, hx, hy, hz);
            else
                L.template hvp<false>(P, rx, ry, rz, k, hx, hy, hz);
            if (lead) {
                // g = (r_prev - r + a H r) / (2 D dt), packed over (a, b).
                const float2 gx = mul2(fma2(pk(k.a), hx, sub2(pk(rpx, rx.x), rx)), ginv);
                const float2 gy = mul2(fma2(pk(k.a), hy, sub2(pk(rpy, ry.x), ry)), ginv);
                const float2 gz = mul2(fma2(pk(k.a), hz, sub2(pk(rpz, rz.x), rz)), ginv);
                if (real_a) {
                    float* Ga = G + (long long)a * s + i;
                    if (PAMD_OK_IDX((long long)a * s + i + 2 * N, (long long)(T + 1) * s)) {
                        Ga[0] = gx.x;
                        Ga[N] = gy.x;
                        Ga[2 * N] = gz.x;
                    }
                }
                if (hasb) {
                    float* Gb = G + (long long)b * s + i;
                    if (PAMD_OK_IDX((long long)b * s + i + 2 * N, (long long)(T + 1) * s)) {
                        Gb[0] = gx.y;
                        Gb[N] = gy.y;
                        Gb[2 * N] = gz.y;
                    }
                }
            }
        }
        rpx = hasb ? rx.y : rx.x;
        rpy = hasb ? ry.y : ry.x;
        rpz = hasb ? rz.y : rz.x;
        __syncthreads();
        if (pf) store(threadIdx.x, nv);
        __syncthreads();
    }
    if (GRAD && t1 == T && S.write_nose && lead) {
        float* Gt = G + (long long)T * s + i;
        if (PAMD_OK_IDX((long long)T * s + i + 2 * N, (long long)(T + 1) * s)) {
            Gt[0] = rpx * k.ginv;
            Gt[N] = rpy * k.ginv;
            Gt[2 * N] = rpz * k.ginv;
        }
    }
    if (HS && __syncthreads_or(ov) && threadIdx.x == 0) atomicOr(overlap + S.chain0 + I.chain, 1);
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[I.slot] = tot;
}

// One work item, action and gradient, pipelined over step pairs: the list walk of
// pair p computes the Hessian-vector product of pair p and the force of pair p+1
// (two independent chains of arithmetic per list entry, one index load), so the
// positions of two pairs are resident.  Window lists cover two consecutive pairs;
// windows are at least 4 steps long and overlap by one pair.  Every sum is the
// same as in paired_item.
template <int NMAX, bool HS>
__device__ __forceinline__ void paired_item_pipe(const LJItem& I, const LJSysDev<float>& S,
                                                 unsigned char* smem, const float* __restrict__ pos,
                                                 float* __restrict__ grad,
                                                 double* __restrict__ partials, double* red,
                                                 uint32_t* outer, int* dmax_bits,
                                                 const float* __restrict__ hs2,
                                                 int* __restrict__ overlap)
{
    const int N = S.N;
    const SmemP<NMAX> P{smem};
    PairList<NMAX> L;
    L.init(N, S.tpp, S.lg_tpp, S.cap, P.list(), S.outer_cap, outer);
    const K2 k(S.k);
    const float2 na = pk(-k.a), ginv = pk(k.ginv);

    const int t0 = I.t0, t1 = I.t1, T = S.T;
    const int s = 3 * N;
    const float* __restrict__ X = pos + S.off + (long long)I.chain * S.chain_len;
    float* __restrict__ G = grad + S.off + (long long)I.chain * S.chain_len;
    const int i = L.i;
    const bool lead = L.active && L.q == 0;
    const int ts = t0 > 0 ? t0 - 1 : t0;  // first slice of the first pair

    auto fetch = [&](int a, int n, float (&v)[6]) {
        const float* A = X + (long long)a * s + n;
        const bool ok = PAMD_OK_IDX((long long)(a + 1) * s + n + 2 * N, (long long)(T + 1) * s);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[2 * c] = ok ? __ldg(A + c * N) : 0.f;
            v[2 * c + 1] = ok ? __ldg(A + s + c * N) : 0.f;
        }
    };
    auto store = [&](int buf, int n, const float (&v)[6]) {
        P.xy(buf, 8 * n) = make_float4(v[0], v[1], v[2], v[3]);
        P.z(buf, 8 * n) = make_float2(v[4], v[5]);
    };
    const int W = max(4, S.window);
    int win_end = ts;
    bool sk = false;  // the current window allows one image shift per entry
    bool ov = false;  // a pair within the hard-sphere radius of its slice (HS)
    // squared hard-sphere radii of slices a, a+1 (the force pair starting at a)
    auto hs_pair = [&](int a) { return HS ? pk(hs2[S.hs_off + a], hs2[S.hs_off + a + 1]) : float2(); };
    // Window list covering slices up to `last` (the b slice of the later of the two
    // pairs the next walk touches), starting at slice a.
    auto ensure_window = [&](int a, int last) {
        if (last < win_end) return;
        const int e = min(a + W, t1 + 1);  // > last: last <= a + 3 <= a + W, or last <= t1
        stage_reference(P, X, N, a, e, dmax_bits, T + 1);
        __syncthreads();
        sk = window_shared_shift(S, k, dmax_bits);
        L.build(P, k);
        __syncthreads();
        if (threadIdx.x == 0) *dmax_bits = 0;  // read by all before the barrier above
        win_end = e;
    };
    // residuals of the pair starting at slice a (in buffer buf), F its force
    auto residual = [&](int buf, int a, float2 fx, float2 fy, float2 fz, float2& rx, float2& ry,
                        float2& rz) {
        rx = ry = rz = pk(0.0f);
        if (!L.active) return;
        const int b = a + 1;
        const bool hb = b < t1;
        float xn = 0.0f, yn = 0.0f, zn = 0.0f;
        if (hb) {
            const float* Xb1 = X + (long long)(b + 1) * s + i;
            const bool ok = PAMD_OK_IDX((long long)(b + 1) * s + i + 2 * N, (long long)(T + 1) * s);
            xn = ok ? __ldg(Xb1) : 0.f;
            yn = ok ? __ldg(Xb1 + N) : 0.f;
            zn = ok ? __ldg(Xb1 + 2 * N) : 0.f;
        }
        const float4 pxy = P.xy(buf, 8 * i);
        const float2 pz = P.z(buf, 8 * i);
        rx = fma2(na, fx, sub2(pk(pxy.y, xn), pk(pxy.x, pxy.y)));
        ry = fma2(na, fy, sub2(pk(pxy.w, yn), pk(pxy.z, pxy.w)));
        rz = fma2(na, fz, sub2(pk(pz.y, zn), pz));
        if (!hb) rx.y = ry.y = rz.y = 0.0f;
    };
    double acc = 0.0;
    auto account = [&](int a, float2 rx, float2 ry, float2 rz) {
        if (!lead) return;
        P.rxy(8 * i) = make_float4(rx.x, rx.y, ry.x, ry.y);
        P.rz(8 * i) = rz;
        if (a >= t0) acc += (double)sq3(rx.x, ry.x, rz.x);
        if (a + 1 < t1) acc += (double)sq3(rx.y, ry.y, rz.y);
    };

    // Item-wide outer list.
    stage_reference(P, X, N, ts, t1 + 1, dmax_bits, T + 1);
    __syncthreads();
    L.build_outer(P, k);
    __syncthreads();
    if (threadIdx.x == 0) *dmax_bits = 0;

    // Pairs a = ts + 2p, p < np; buffers: pair p in buffer p & 1.
    const int np = (t1 - ts + 1) / 2;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float v[6];
        fetch(ts, n, v);
        store(0, n, v);
        if (np > 1) {
            fetch(ts + 2, n, v);
            store(1, n, v);
        }
    }
    __syncthreads();
    ensure_window(ts, min(ts + (np > 1 ? 3 : 1), t1));

    // Prologue: force and residuals of pair 0.
    float2 rx, ry, rz;  // residuals of the current pair
    {
        float2 hx, hy, hz, fx, fy, fz;
        if (sk)
            L.template combined<false, true, true, HS, 0, 0>(P, pk(0.0f), pk(0.0f), pk(0.0f), k, hx,
                                                             hy, hz, fx, fy, fz, hs_pair(ts), &ov);
        else
            L.template combined<false, true, false, HS, 0, 0>(P, pk(0.0f), pk(0.0f), pk(0.0f), k, hx,
                                                              hy, hz, fx, fy, fz, hs_pair(ts), &ov);
        residual(0, ts, fx, fy, fz, rx, ry, rz);
        account(ts, rx, ry, rz);
    }
    __syncthreads();

    float rpx = 0.0f, rpy = 0.0f, rpz = 0.0f;  // r_{a-1}
    for (int p = 0; p < np; ++p) {
        const int cur = p & 1, nxt = cur ^ 1;
        const int a = ts + 2 * p, b = a + 1;
        const bool hasb = b < t1, real_a = a >= t0;
        const bool next = p + 1 < np;
        // prefetch pair p+2 (its slices a+4, a+5 <= t1 when it exists)
        const bool pf = p + 2 < np && (int)threadIdx.x < N;
        float nv[6];
        if (pf) fetch(a + 4, threadIdx.x, nv);

        float2 hx, hy, hz, fx, fy, fz;
        // buffer indices as template arguments: immediate shared-memory offsets and
        // a compile-time choice of the halves of the shared z slot
        auto walk = [&](auto cur_c) {
            constexpr int C = decltype(cur_c)::value;
            if (next && sk)
                L.template combined<true, true, true, HS, C, C ^ 1>(P, rx, ry, rz, k, hx, hy, hz, fx,
                                                                    fy, fz, hs_pair(a + 2), &ov);
            else if (next)
                L.template combined<true, true, false, HS, C, C ^ 1>(P, rx, ry, rz, k, hx, hy, hz, fx,
                                                                     fy, fz, hs_pair(a + 2), &ov);
            else if (sk)
                L.template combined<true, false, true, false, C, C>(P, rx, ry, rz, k, hx, hy, hz, fx,
                                                                    fy, fz);
            else
                L.template combined<true, false, false, false, C, C>(P, rx, ry, rz, k, hx, hy, hz, fx,
                                                                     fy, fz);
        };
        if (cur)
            walk(std::integral_constant<int, 1>{});
        else
            walk(std::integral_constant<int, 0>{});
        if (lead) {
            const float2 gx = mul2(fma2(pk(k.a), hx, sub2(pk(rpx, rx.x), rx)), ginv);
            const float2 gy = mul2(fma2(pk(k.a), hy, sub2(pk(rpy, ry.x), ry)), ginv);
            const float2 gz = mul2(fma2(pk(k.a), hz, sub2(pk(rpz, rz.x), rz)), ginv);
            if (real_a) {
                float* Ga = G + (long long)a * s + i;
                if (PAMD_OK_IDX((long long)a * s + i + 2 * N, (long long)(T + 1) * s)) {
                    Ga[0] = gx.x;
                    Ga[N] = gy.x;
                    Ga[2 * N] = gz.x;
                }
            }
            if (hasb) {
                float* Gb = G + (long long)b * s + i;
                if (PAMD_OK_IDX((long long)b * s + i + 2 * N, (long long)(T + 1) * s)) {
                    Gb[0] = gx.y;
                    Gb[N] = gy.y;
                    Gb[2 * N] = gz.y;
                }
            }
        }
        rpx = hasb ? rx.y : rx.x;
        rpy = hasb ? ry.y : ry.x;
        rpz = hasb ? rz.y : rz.x;
        float2 nrx, nry, nrz;
        if (next) residual(nxt, a + 2, fx, fy, fz, nrx, nry, nrz);
        __syncthreads();  // every walk is done with the residuals and buffer cur
        if (next) {
            account(a + 2, nrx, nry, nrz);
            rx = nrx;
            ry = nry;
            rz = nrz;
        }
        if (pf) store(cur, threadIdx.x, nv);
        if (next) ensure_window(a + 2, min(a + (p + 2 < np ? 5 : 3), t1));
        __syncthreads();
    }
    if (t1 == T && S.write_nose && lead) {
        float* Gt = G + (long long)T * s + i;
        if (PAMD_OK_IDX((long long)T * s + i + 2 * N, (long long)(T + 1) * s)) {
            Gt[0] = rpx * k.ginv;
            Gt[N] = rpy * k.ginv;
            Gt[2 * N] = rpz * k.ginv;
        }
    }
    if (HS && __syncthreads_or(ov) && threadIdx.x == 0) atomicOr(overlap + S.chain0 + I.chain, 1);
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[I.slot] = tot;
}

// Persistent grid: each CTA takes items from *counter until none is left.
// Systems must have N <= MAXT (the block size is at most MAXT).
// HS: the hard-sphere path bias is on (hs2: squared radii per slice of every LJ
// system, at LJSysDev::hs_off; overlap: a flag per global chain).
template <bool GRAD, int MAXT, bool PIPE, bool HS>
__global__ void __launch_bounds__(MAXT, 1)
    lj_paired_kernel(const LJItem* __restrict__ items, int n_items,
                     const LJSysDev<float>* __restrict__ systems, const float* __restrict__ pos,
                     float* __restrict__ grad, double* __restrict__ partials,
                     int* __restrict__ counter, uint32_t* __restrict__ outer, long long outer_words,
                     const float* __restrict__ hs2, int* __restrict__ overlap)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_item;
    __shared__ int s_dmax;  // bits of the largest margin of the window being staged
    if (threadIdx.x == 0) s_dmax = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const LJItem I = items[it];
        const LJSysDev<float> S = systems[I.sys];
        if (GRAD && PIPE)
            paired_item_pipe<MAXT, HS>(I, S, smem_raw, pos, grad, partials, red,
                                       outer + (long long)blockIdx.x * outer_words, &s_dmax, hs2,
                                       overlap);
        else
            paired_item<GRAD, MAXT, HS>(I, S, smem_raw, pos, grad, partials, red,
                                        outer + (long long)blockIdx.x * outer_words, &s_dmax, hs2,
                                        overlap);
    }
}

// The pipelined form is used with the gradient for blocks of up to 512 threads
// (its two position buffers and staging area take 88 bytes per particle slot).
template <bool GRAD, bool HS>
auto paired_kernel_ptr(int NT, bool pipe)
{
    if (GRAD && pipe && NT <= 512) return lj_paired_kernel<GRAD, 512, true, HS>;
    return NT <= 512 ? lj_paired_kernel<GRAD, 512, false, HS> : lj_paired_kernel<GRAD, 1024, false, HS>;
}

using PairedKernel = void (*)(const LJItem*, int, const LJSysDev<float>*, const float*, float*,
                              double*, int*, uint32_t*, long long, const float*, int*);
PairedKernel paired_kernel_sel(int NT, bool with_grad, bool pipe, bool hs)
{
    if (with_grad) return hs ? paired_kernel_ptr<true, true>(NT, pipe) : paired_kernel_ptr<true, false>(NT, pipe);
    return hs ? paired_kernel_ptr<false, true>(NT, pipe) : paired_kernel_ptr<false, false>(NT, pipe);
}

}  // namespace

size_t lj_paired_smem_bytes(int NT, int cap_lane, bool pipe)
{
    const size_t nmax = NT <= 512 ? 512 : 1024;
    const size_t slots = (pipe && NT <= 512) ? 88 : 48;
    return slots * nmax + (size_t)(cap_lane / 2) * NT * sizeof(uint32_t);
}

int lj_paired_blocks_per_sm(int NT, size_t smem, bool with_grad, bool pipe)
{
    auto kern = paired_kernel_sel(NT, with_grad, pipe, false);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_lj_paired(const LJItem* items, int n_items, const void* sys_table,
                             const float* pos, float* grad, double* partials, int* counter, int NT,
                             size_t smem, int grid, bool with_grad, bool pipe, uint32_t* outer,
                             long long outer_words, cudaStream_t st, const float* hs2, int* overlap)
{
    if (n_items <= 0) return cudaSuccess;
    if (NT > 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    auto kern = paired_kernel_sel(NT, with_grad, pipe, hs2 != nullptr);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, smem, st>>>(items, n_items, static_cast<const LJSysDev<float>*>(sys_table),
                                 pos, grad, partials, counter, outer, outer_words, hs2, overlap);
    return cudaGetLastError();
}

PAMD_DEBUG_FETCHER(lj_paired)

}  // namespace pamd
