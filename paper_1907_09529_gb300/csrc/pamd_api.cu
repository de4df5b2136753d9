// pamd_api.cu -- the C ABI of libpamd: argument checks, cached plans (work
// descriptors, workspace, captured graphs), host-buffer staging, dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <initializer_list>
#include <type_traits>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pamd_internal.cuh"
#include "fragment.cuh"

using namespace pamd;

namespace {

// NVTX range around every entry point (visible in Nsight tools; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Host-side fault injection, for tests of the error paths (nothing faults on the
// device): PAMD_FAULT_INJECT=alloc makes every workspace allocation fail,
// =launch makes every CUDA call the library checks report failure, =nonfinite
// flags every action computed as non-finite.
bool fault_injected(const char* what)
{
    const char* e = std::getenv("PAMD_FAULT_INJECT");
    return e && std::strcmp(e, what) == 0;
}

#define PAMD_CUDA_TRY(expr)                                                    \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess || fault_injected("launch")) return PAMD_ERR_CUDA; \
    } while (0)

struct LJTune {
    int tile_steps = 0, tpp = 0, maxnb = 0;
    double skin = -1.0;
    int window = 0;     // paired kernel: steps per neighbour-list window
    int outer_cap = 0;  // paired kernel: outer-list entries per thread
};

LJTune g_tune_override;  // 0 / negative fields mean "automatic"
constexpr int kMaxListPerThread = 1024;  // list entries per thread (uint16 indices)
std::mutex g_mutex;

struct SysInfo {
    int N, T, d, chains, kind, chain0;
    long long off, chain_len;
    pamd_potential pot;
    LJTune tune;       // LJ only
    int lj_index = -1; // row in the LJ system table
    int ho_b0 = 0, ho_b1 = 0;  // harmonic: range of this system's element blocks
    int slot0 = 0;     // first S slot (LJ tiles)
    int n_tiles = 0;
    long long first_slice = 0;   // time slab (0 / 0 / 0 for whole paths)
    int halo_lo = 0, halo_hi = 0;
    long long hs_off = 0;        // LJ: first of its slices in the hard-sphere radii array
    int lj_class = 0;            // LJ: block-size class (launch) of the system
    int NT = 0;                  // LJ: block size of that class
};

// LJ systems launched together: one block size, shared-memory size and grid.
// Single-precision batches that mix systems of N <= 512 and N > 512 get two
// classes, so the smaller systems run the pipelined 512-thread kernel instead of
// leaving most of a 1024-thread block idle.
struct LJClass {
    int NT = 0, nmax = 0, grid_grad = 0, grid_nograd = 0;
    bool pipe = false;           // gradient pass pipelined over step pairs
    size_t smem = 0;
    long long outer_words = 0;   // 32-bit words of each CTA's outer-list region
    int item_off = 0, n_items = 0;  // its items in d_lj_items (cost-sorted)
    int grp_off = 0;             // its items in d_lj_items_grp (grouped by chain)
    std::vector<int> grp_first;  // per global chain c: [grp_first[c], grp_first[c + 1]), relative
};

// Buffers and update count of a captured update graph.  Compared field by field:
// the struct has padding after n_updates, which a byte comparison would read.
struct GraphKey {
    const void *pos, *grad, *S, *nacc, *la;
    int n_updates;
    bool operator<(const GraphKey& o) const
    {
        const void* a[5] = {pos, grad, S, nacc, la};
        const void* b[5] = {o.pos, o.grad, o.S, o.nacc, o.la};
        for (int q = 0; q < 5; ++q)
            if (a[q] != b[q]) return std::less<const void*>()(a[q], b[q]);
        return n_updates < o.n_updates;
    }
};

struct Plan {
    std::string key;
    bool fp64 = false;
    int n_chains = 0;
    size_t esz = 4;
    long long span = 0;  // elements spanned by the pos buffer
    std::vector<SysInfo> sys;
    std::vector<ElemBlock> h_all, h_ho;
    std::vector<int> ho_chain_first;  // per chain: first HO block index (or -1), and count
    std::vector<int> ho_chain_count;
    int max_s_ho = 0;
    ElemBlock* d_all = nullptr;
    ElemBlock* d_ho = nullptr;
    ChainSlots* d_S_slots = nullptr;
    ChainSlots* d_E_slots = nullptr;
    int n_S_slots = 0;
    double* d_part_S = nullptr;
    double* d_part_qf = nullptr;
    double* d_part_qr = nullptr;
    // LJ work items (persistent kernels, one launch per block-size class)
    bool lj_paired = false;  // single precision: two steps per thread (lj_paired.cu)
    std::vector<LJClass> lj_cls;
    std::vector<unsigned char> h_lj_sys;  // host copy of the system table
    size_t lj_sys_stride = 0;
    void* d_lj_sys = nullptr;
    LJItem* d_lj_items = nullptr;
    int n_lj_items = 0;
    std::vector<int> lj_chain_first, lj_chain_count;  // per global chain (plain form)
    std::vector<int> lj_chain_class;                  // per global chain: its class (-1: none)
    LJItem* d_lj_items_grp = nullptr;  // the same items, per class grouped by chain
    std::vector<ChainSlots> h_E_slots;  // per chain: its element blocks in h_all
    int* d_counter = nullptr;
    int* d_err = nullptr;  // device status word (PAMD_OK or PAMD_ERR_NONFINITE)
    // update workspace (allocated on first use)
    void* d_prop = nullptr;
    void* d_gprop = nullptr;
    double* d_Sprop = nullptr;
    double* d_qf = nullptr;
    double* d_qr = nullptr;
    int* d_flag = nullptr;
    MalaDev* d_md = nullptr;
    // host-pointer staging (allocated on first use)
    void* d_stage_pos = nullptr;
    void* d_stage_grad = nullptr;
    void* d_stage_noise = nullptr;
    double* d_stage_S = nullptr;
    double* d_stage_dbl = nullptr;  // log_alpha
    double* d_stage_logu = nullptr;
    int* d_stage_int = nullptr;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::vector<void*> allocs;
    // paired LJ kernel: outer lists, one set per compute lane of one region per CTA
    // (the classes of a lane run one after another and share its set)
    uint32_t* d_outer = nullptr;
    long long outer_lane_words = 0;  // 32-bit words of one lane's set
    int n_lanes = 1;            // compute lanes of the host-buffer pipeline
    // hard-sphere path bias (pamd_action_grad_hs): radii of every LJ slice, per-chain flags
    long long hs_slices = 0;
    void* d_hs2 = nullptr;
    bool any_slab = false;      // some system is a time slab
    int* d_overlap = nullptr;
    // host-buffer pipeline: copy streams, the extra compute streams (lanes 1..), events
    // and one LJ work counter per chunk (created on first use)
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaStream_t> s_cmp;
    std::vector<cudaEvent_t> events;
    int* d_chunk_counters = nullptr;

    ~Plan()
    {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_out) cudaStreamDestroy(s_out);
        for (cudaStream_t c : s_cmp) cudaStreamDestroy(c);
        for (void* p : allocs) cudaFree(p);
    }
    template <typename T>
    int alloc(T** p, size_t bytes)
    {
        void* q = nullptr;
        if (bytes == 0) bytes = 16;
        if (fault_injected("alloc") || cudaMalloc(&q, bytes) != cudaSuccess) return PAMD_ERR_ALLOC;
        allocs.push_back(q);
        *p = reinterpret_cast<T*>(q);
        return PAMD_OK;
    }
};

std::map<std::string, std::unique_ptr<Plan>> g_plans;

int check_problem(const pamd_problem* p)
{
    if (!p || !p->systems || p->n_systems <= 0) return PAMD_ERR_ARG;
    if (p->flags & ~(PAMD_FLAG_ONE_CHAIN_PER_LAUNCH | PAMD_FLAG_HO_EXACT_PROPAGATOR |
                     PAMD_FLAG_REGENERATE_FLAT))
        return PAMD_ERR_ARG;
    if (p->precision != PAMD_FP32 && p->precision != PAMD_FP64) return PAMD_ERR_ARG;
    if (!(p->D > 0) || !(p->dt > 0) || !(p->beta > 0)) return PAMD_ERR_ARG;
    for (int q = 0; q < p->n_systems; ++q) {
        const pamd_system& s = p->systems[q];
        if (s.n_particles < 1 || s.n_steps < 1 || s.dim < 1 || s.dim > 3 || s.n_chains < 1 ||
            s.pos_offset < 0)
            return PAMD_ERR_ARG;
        const long long chain_len = (long long)(s.n_steps + 1) * s.dim * s.n_particles;
        if (chain_len >= (1LL << 31)) return PAMD_ERR_UNSUPPORTED;
        // time slab: halo flags 0/1, a lower halo needs a slice before it, and at
        // least one owned step
        if (s.first_slice < 0 || (s.halo_lo != 0 && s.halo_lo != 1) ||
            (s.halo_hi != 0 && s.halo_hi != 1) || (s.halo_lo && s.first_slice < 1) ||
            s.n_steps - s.halo_lo < 1)
            return PAMD_ERR_ARG;
        if (s.first_slice + s.n_steps >= (1LL << 31) / std::max(1, s.dim * s.n_particles))
            return PAMD_ERR_UNSUPPORTED;
        if (s.pot.kind == PAMD_HARMONIC) {
            if (s.dim * s.n_particles > 8192) return PAMD_ERR_UNSUPPORTED;
        } else if (s.pot.kind == PAMD_LJ) {
            if (s.dim != 3 || s.n_particles < 2) return PAMD_ERR_ARG;
            if (s.n_particles > 1024) return PAMD_ERR_UNSUPPORTED;
            if (!(s.pot.box > 0) || !(s.pot.rc > 0) || s.pot.rc > 0.5 * s.pot.box ||
                !(s.pot.sigma > 0) || !(s.pot.eps >= 0))
                return PAMD_ERR_ARG;
        } else {
            return PAMD_ERR_ARG;
        }
    }
    return PAMD_OK;
}

// Entry points that need whole paths (no time slab).
int check_whole_paths(const pamd_problem* p)
{
    for (int q = 0; q < p->n_systems; ++q) {
        const pamd_system& s = p->systems[q];
        if (s.first_slice || s.halo_lo || s.halo_hi) return PAMD_ERR_UNSUPPORTED;
    }
    return PAMD_OK;
}

// The Eq. (3) entry points: the exact-propagator flag belongs to the sampler.
int check_em_problem(const pamd_problem* p)
{
    const int rc = check_problem(p);
    if (rc) return rc;
    return (p->flags & PAMD_FLAG_HO_EXACT_PROPAGATOR) ? PAMD_ERR_UNSUPPORTED : PAMD_OK;
}

// Width of a regeneration step: free-particle steps sqrt(2 D dt) z, or 0 (the
// path continues as the horizontal line x_T; fma(0, z, x) = x exactly).
double regen_sigma(const pamd_problem* p)
{
    return (p->flags & PAMD_FLAG_REGENERATE_FLAT) ? 0.0 : std::sqrt(2.0 * p->D * p->dt);
}

// Drift factor g and action scale c of one harmonic system's steps,
// S_t = c |x_{t+1} - x_t + g x_t|^2: Eq. (3) (g = beta D k dt, c = 1/(4 D dt)) or
// the exact transition density (g = 1 - phi, c = beta k / (2 (1 - phi^2))).
void ho_step_constants(const pamd_problem* p, double k, double* g, double* c)
{
    if (p->flags & PAMD_FLAG_HO_EXACT_PROPAGATOR) {
        const double phi = std::exp(-p->beta * p->D * k * p->dt);
        *g = 1.0 - phi;
        *c = p->beta * k / (2.0 * (1.0 - phi * phi));
    } else {
        *g = p->beta * p->D * p->dt * k;
        *c = 1.0 / (4.0 * p->D * p->dt);
    }
}

std::string plan_key(const pamd_problem* p)
{
    std::ostringstream os;
    os.precision(17);
    os << p->precision << '|' << p->flags << '|' << p->D << ',' << p->beta << ',' << p->dt << '|'
       << p->n_systems << '|' << g_tune_override.tile_steps
       << ',' << g_tune_override.tpp << ',' << g_tune_override.maxnb << ',' << g_tune_override.skin
       << ',' << g_tune_override.window << '|';
    // launch-shape switches read when a plan is built: a change builds a new plan
    for (const char* v : {"PAMD_LJ_ONE_STEP", "PAMD_LJ_NO_PIPE", "PAMD_LJ_ONE_CLASS",
                          "PAMD_LJ_PER_STEP_SHIFT", "PAMD_PIPE_LANES"}) {
        const char* e = std::getenv(v);
        os << (e ? e : "-") << ',';
    }
    for (int q = 0; q < p->n_systems; ++q) {
        const pamd_system& s = p->systems[q];
        os << '|' << s.n_particles << ',' << s.n_steps << ',' << s.dim << ',' << s.n_chains << ','
           << s.pos_offset << ',' << s.pot.kind << ',' << s.pot.k << ',' << s.pot.eps << ','
           << s.pot.sigma << ',' << s.pot.rc << ',' << s.pot.box << ',' << s.first_slice << ','
           << s.halo_lo << ',' << s.halo_hi;
    }
    return os.str();
}

int max_dynamic_smem()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 48 * 1024;
    return v;
}

// Block size of a class of LJ systems: its largest N times the threads per
// particle -- the forced count, else the largest power of two up to 8 that fits
// 512 threads, so that small systems are spread over more warps -- rounded up to
// a warp multiple, at least 128 and at most 1024.
int choose_lj_block(int nmax)
{
    int tpp = 1;
    if (g_tune_override.tpp > 0)
        tpp = g_tune_override.tpp;
    else
        while (tpp < 8 && nmax * tpp * 2 <= 512) tpp *= 2;
    return std::max(128, std::min(1024, ((nmax * tpp + 31) / 32) * 32));
}

// Per-system LJ launch shape: threads per particle (largest power of two <= 8
// with N * tpp <= NT), Verlet skin (one-step kernel) or window length (paired
// kernel), list capacity per thread, tile length.  sig_step = sqrt(2 D dt), the
// per-component spread of one Brownian step.
LJTune choose_lj_tune(const pamd_system& s, int NT, int cap_lane_max, bool paired, double sig_step)
{
    LJTune t;
    const int N = s.n_particles;
    int tpp = 1;
    while (tpp < 8 && N * tpp * 2 <= NT) tpp *= 2;
    if (g_tune_override.tpp > 0) {
        const int lim = std::min(g_tune_override.tpp, std::max(1, NT / N));
        tpp = 1;
        while (tpp * 2 <= lim) tpp *= 2;  // a power of two (lane = tid mod tpp)
    }
    while (tpp > 1 && N * tpp > NT) tpp >>= 1;
    t.tpp = tpp;
    t.skin = g_tune_override.skin >= 0 ? g_tune_override.skin : 0.3;
    t.tile_steps = g_tune_override.tile_steps > 0 ? g_tune_override.tile_steps : 32;
    t.window = g_tune_override.window > 0 ? g_tune_override.window : 12;
    double rl = s.pot.rc + t.skin;
    if (paired) {
        // Window lists reach rc + delta_i + delta_j; size them for margins of about
        // 3.5 times the spread of a 3D displacement over half a window.
        const double dmax = 3.5 * sig_step * std::sqrt(3.0 * 0.5 * t.window);
        rl = s.pot.rc + 2.0 * dmax;
    }
    const double L = s.pot.box, rho = N / (L * L * L);
    if (paired) {
        // Outer lists reach rc + Delta_i + Delta_j with item-wide margins; size them
        // for about 2.5 times the spread of a 3D displacement over half a tile (a
        // particle beyond that builds its window lists from every candidate).
        const double dmax = 2.5 * sig_step * std::sqrt(3.0 * 0.5 * (t.tile_steps + 1));
        const double ro = s.pot.rc + 2.0 * dmax;
        int ow = (int)(1.2 * 4.18879020478639 * ro * ro * ro * rho) + 16;
        ow = std::min(ow, N - 1 + 2 * tpp);
        t.outer_cap = std::max(2, std::min((ow + tpp - 1) / tpp, kMaxListPerThread)) & ~1;
    }
    const double expect = 4.18879020478639 * rl * rl * rl * rho;  // 4/3 pi rl^3 rho
    int want = (int)(1.2 * expect) + 8;
    if (want > N - 1 + tpp) want = N - 1 + tpp;
    if (g_tune_override.maxnb > 0) want = g_tune_override.maxnb;
    int lane = (want + tpp - 1) / tpp;
    t.maxnb = std::max(1, std::min(std::min(lane, cap_lane_max), kMaxListPerThread));  // per thread
    return t;
}

template <typename R>
void fill_lj_sys(Plan* P, const pamd_problem* p)
{
    P->lj_sys_stride = sizeof(LJSysDev<R>);
    int nlj = 0;
    for (auto& si : P->sys) nlj += si.kind == PAMD_LJ;
    P->h_lj_sys.assign(P->lj_sys_stride * std::max(nlj, 1), 0);
    for (auto& si : P->sys) {
        if (si.kind != PAMD_LJ) continue;
        LJSysDev<R> d;
        d.off = si.off;
        d.chain_len = si.chain_len;
        d.N = si.N;
        d.T = si.T;
        d.tpp = si.tune.tpp;
        d.lg_tpp = 0;
        while ((1 << d.lg_tpp) < d.tpp) ++d.lg_tpp;
        d.cap = si.tune.maxnb;
        d.window = si.tune.window;
        d.outer_cap = si.tune.outer_cap;
        // (PAMD_LJ_PER_STEP_SHIFT=1 rounds the image shift at every slice instead; the
        // results are bitwise the same, which a test checks)
        d.shared_shift = std::getenv("PAMD_LJ_PER_STEP_SHIFT") == nullptr;
        d.write_nose = !si.halo_hi;
        d.chain0 = si.chain0;
        d.hs_off = si.hs_off = P->hs_slices;  // this system's slices in the hard-sphere radii
        P->hs_slices += si.T + 1;
        LJConst c;
        c.L = si.pot.box;
        c.rc = si.pot.rc;
        c.eps = si.pot.eps;
        c.sigma = si.pot.sigma;
        c.a = p->beta * p->D * p->dt;
        c.ginv = 1.0 / (2.0 * p->D * p->dt);
        c.skin = si.tune.skin;
        d.k = make_lj_consts<R>(c, std::sqrt(2.0 * p->D * p->dt));
        std::memcpy(&P->h_lj_sys[P->lj_sys_stride * si.lj_index], &d, sizeof(d));
    }
}

// Compute lanes (streams) of the host-buffer pipeline: chunk k is updated on lane
// k mod lanes, so that up to `lanes` chunks' kernels share the GPU while later
// chunks are copied in.  PAMD_PIPE_LANES overrides the default (1..4).
constexpr int kMaxPipeLanes = 4;
int pipeline_lanes()
{
    const char* e = std::getenv("PAMD_PIPE_LANES");
    const int v = e ? std::atoi(e) : 3;
    return std::max(1, std::min(kMaxPipeLanes, v));
}

// Timeline of the last pipelined host-buffer update (milliseconds after its start):
// [total, then per chunk: inputs on the device, update done, results on the host].
std::vector<float> g_last_timeline;

int build_plan(const pamd_problem* p, Plan** out)
{
    std::string key = plan_key(p);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second.get();
        return PAMD_OK;
    }
    std::unique_ptr<Plan> P(new Plan());
    int rc0;
    P->key = key;
    P->fp64 = p->precision == PAMD_FP64;
    P->esz = P->fp64 ? 8 : 4;
    int chain = 0;
    std::vector<ChainSlots> Sslots, Eslots;
    for (int q = 0; q < p->n_systems; ++q) {
        const pamd_system& s = p->systems[q];
        SysInfo si;
        si.N = s.n_particles;
        si.T = s.n_steps;
        si.d = s.dim;
        si.chains = s.n_chains;
        si.kind = s.pot.kind;
        si.chain0 = chain;
        si.off = s.pos_offset;
        si.chain_len = (long long)(s.n_steps + 1) * s.dim * s.n_particles;
        si.pot = s.pot;
        si.first_slice = s.first_slice;
        si.halo_lo = s.halo_lo;
        si.halo_hi = s.halo_hi;
        P->any_slab = P->any_slab || s.first_slice || s.halo_lo || s.halo_hi;
        P->span = std::max(P->span, si.off + si.chain_len * si.chains);
        P->sys.push_back(si);
        chain += s.n_chains;
    }
    P->n_chains = chain;
    Sslots.resize(chain);
    Eslots.resize(chain);
    P->ho_chain_first.assign(chain, -1);
    P->ho_chain_count.assign(chain, 0);
    // element blocks: all systems (update passes) and harmonic systems (action)
    for (auto& si : P->sys) {
        const int s = si.d * si.N;
        for (int b = 0; b < si.chains; ++b) {
            const int c = si.chain0 + b;
            Eslots[c].begin = (int)P->h_all.size();
            if (si.kind == PAMD_HARMONIC) {
                if (b == 0) si.ho_b0 = (int)P->h_ho.size();
                Sslots[c].begin = (int)P->h_ho.size();
                P->ho_chain_first[c] = (int)P->h_ho.size();
            }
            for (long long e0 = 0; e0 < si.chain_len; e0 += kElemChunk) {
                ElemBlock B;
                B.chain_base = si.off + b * si.chain_len;
                B.e0 = (int)e0;
                B.n = (int)std::min<long long>(kElemChunk, si.chain_len - e0);
                B.s = s;
                B.chain_len = (int)si.chain_len;
                B.chain = c;
                B.sys = (int)(&si - &P->sys[0]);
                B.k = si.pot.k;
                B.e_glob = si.first_slice * s;
                B.own_lo = si.halo_lo * s;
                B.own_hi = (int)si.chain_len - si.halo_hi * s;
                B.sum_lo = si.halo_lo * s;
                P->h_all.push_back(B);
                if (si.kind == PAMD_HARMONIC) P->h_ho.push_back(B);
            }
            Eslots[c].end = (int)P->h_all.size();
            if (si.kind == PAMD_HARMONIC) {
                si.ho_b1 = (int)P->h_ho.size();
                Sslots[c].end = (int)P->h_ho.size();
                P->ho_chain_count[c] = Sslots[c].end - Sslots[c].begin;
                P->max_s_ho = std::max(P->max_s_ho, s);
            }
        }
    }
    int slot = (int)P->h_ho.size();
    // LJ: block-size classes, shared-memory budgets, per-system shapes, items.
    std::vector<LJItem> items, grouped;
    P->lj_chain_first.assign(chain, -1);
    P->lj_chain_count.assign(chain, 0);
    P->lj_chain_class.assign(chain, -1);
    P->lj_cls.clear();
    {
        const bool one = (p->flags & PAMD_FLAG_ONE_CHAIN_PER_LAUNCH) != 0;
        int nlj = 0, n_small = 0, n_big = 0;
        for (auto& si : P->sys)
            if (si.kind == PAMD_LJ) {
                si.lj_index = nlj++;
                (si.N <= 512 ? n_small : n_big) += 1;
            }
        if (nlj) {
            P->lj_paired = !P->fp64 && std::getenv("PAMD_LJ_ONE_STEP") == nullptr;
            const bool split = P->lj_paired && n_small && n_big && std::getenv("PAMD_LJ_ONE_CLASS") == nullptr;
            P->lj_cls.resize(split ? 2 : 1);
            for (auto& si : P->sys)
                if (si.kind == PAMD_LJ) si.lj_class = (split && si.N > 512) ? 1 : 0;
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const size_t v4 = P->fp64 ? 32 : 16;
            std::vector<int> bg_cls(P->lj_cls.size(), 0);
            for (int k = 0; k < (int)P->lj_cls.size(); ++k) {
                LJClass& C = P->lj_cls[k];
                for (auto& si : P->sys)
                    if (si.kind == PAMD_LJ && si.lj_class == k) C.nmax = std::max(C.nmax, si.N);
                const int NT = choose_lj_block(C.nmax);
                const int nmax = C.nmax;
                // Single precision runs the paired-step kernel, one CTA per SM: its lists
                // may use all the shared memory beside the packed slices (48 bytes per
                // particle slot, 88 in the pipelined gradient form).
                C.NT = NT;
                C.pipe = P->lj_paired && NT <= 512 && std::getenv("PAMD_LJ_NO_PIPE") == nullptr;
                const long long slices = P->lj_paired ? (C.pipe ? 88LL * 512 : 48LL * (NT <= 512 ? 512 : 1024))
                                                      : 3 * (long long)nmax * v4;
                const int budget = (NT <= 512 && !P->fp64 && !P->lj_paired && g_tune_override.maxnb <= 0)
                                       ? 113 * 1024
                                       : max_dynamic_smem() - 1024;
                // (the one-step Euler kernel shares the capacity: its slices must fit too)
                const long long slices_euler = 3 * (long long)nmax * v4;
                const int cap_lane_max = std::max(
                    1, (int)((budget - std::max(slices, slices_euler)) / (2 * (long long)NT)));
                int cap_used = 1;
                for (int q = 0; q < (int)P->sys.size(); ++q) {
                    SysInfo& si = P->sys[q];
                    if (si.kind != PAMD_LJ || si.lj_class != k) continue;
                    si.tune = choose_lj_tune(p->systems[q], NT, cap_lane_max, P->lj_paired,
                                             std::sqrt(2.0 * p->D * p->dt));
                    si.NT = NT;
                    cap_used = std::max(cap_used, si.tune.maxnb);
                }
                C.smem = P->lj_paired ? lj_paired_smem_bytes(NT, cap_used, C.pipe)
                                      : lj_smem_bytes(nmax, NT, cap_used, P->fp64);
                const int bg = P->lj_paired ? lj_paired_blocks_per_sm(NT, C.smem, true, C.pipe)
                               : P->fp64    ? lj_blocks_per_sm<double>(NT, C.smem, true)
                                            : lj_blocks_per_sm<float>(NT, C.smem, true);
                const int bn = P->lj_paired ? lj_paired_blocks_per_sm(NT, C.smem, false, C.pipe)
                               : P->fp64    ? lj_blocks_per_sm<double>(NT, C.smem, false)
                                            : lj_blocks_per_sm<float>(NT, C.smem, false);
                if (bg <= 0 || bn <= 0) return PAMD_ERR_UNSUPPORTED;
                bg_cls[k] = bg;
                C.grid_grad = bg * sms;  // trimmed to the item count below
                C.grid_nograd = bn * sms;
            }
            // One LJ system of equal items: pick the tile near the chosen one whose item
            // count fills whole rounds of the persistent grid (no part-empty last round),
            // keeping at least 16 steps per item.
            if (nlj == 1 && !one) {
                for (auto& si : P->sys) {
                    if (si.kind != PAMD_LJ) continue;
                    const long long G = (long long)bg_cls[si.lj_class] * sms;
                    const int Tow = si.T - si.halo_lo;  // owned steps
                    const long long items0 = (long long)si.chains * ((Tow + si.tune.tile_steps - 1) / si.tune.tile_steps);
                    const long long rounds = (items0 + G - 1) / G;
                    const long long per_chain = (rounds * G) / si.chains;
                    if (per_chain >= 1) {
                        const int tile = (int)((Tow + per_chain - 1) / per_chain);
                        if (tile >= std::min(16, si.tune.tile_steps)) si.tune.tile_steps = tile;
                    }
                }
            }
            // Items of every system (S slots in system order), with their cost.
            std::vector<std::vector<LJItem>> sys_items(P->sys.size());
            std::vector<std::vector<double>> sys_cost(P->sys.size());
            for (int q = 0; q < (int)P->sys.size(); ++q) {
                SysInfo& si = P->sys[q];
                if (si.kind != PAMD_LJ) continue;
                si.n_tiles = (si.T - si.halo_lo + si.tune.tile_steps - 1) / si.tune.tile_steps;
                si.slot0 = slot;
                for (int b = 0; b < si.chains; ++b) {
                    const int c = si.chain0 + b;
                    Sslots[c].begin = slot + b * si.n_tiles;
                    Sslots[c].end = slot + (b + 1) * si.n_tiles;
                    P->lj_chain_count[c] = si.n_tiles;
                    P->lj_chain_class[c] = si.lj_class;
                    for (int tl = 0; tl < si.n_tiles; ++tl) {
                        LJItem it;
                        it.sys = si.lj_index;
                        it.chain = b;
                        it.t0 = si.halo_lo + tl * si.tune.tile_steps;  // owned steps only
                        it.t1 = std::min(si.T, it.t0 + si.tune.tile_steps);
                        it.slot = slot + b * si.n_tiles + tl;
                        sys_items[q].push_back(it);
                        sys_cost[q].push_back((double)si.N * si.tune.maxnb * si.tune.tpp * (it.t1 - it.t0 + 1));
                    }
                }
                slot += si.chains * si.n_tiles;
            }
            // Per class: its items (largest first unless one chain per launch) and a
            // copy grouped by chain (chains in order, each chain's items largest first)
            // for launches over a range of chains.
            for (int k = 0; k < (int)P->lj_cls.size(); ++k) {
                LJClass& C = P->lj_cls[k];
                std::vector<LJItem> ci;
                std::vector<double> cc;
                std::vector<int> cchain;
                for (int q = 0; q < (int)P->sys.size(); ++q) {
                    const SysInfo& si = P->sys[q];
                    if (si.kind != PAMD_LJ || si.lj_class != k) continue;
                    for (size_t m = 0; m < sys_items[q].size(); ++m) {
                        const int c = si.chain0 + sys_items[q][m].chain;
                        if (P->lj_chain_first[c] < 0) P->lj_chain_first[c] = (int)(items.size() + ci.size());
                        ci.push_back(sys_items[q][m]);
                        cc.push_back(sys_cost[q][m]);
                        cchain.push_back(c);
                    }
                }
                std::vector<int> ord(ci.size());
                for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
                std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
                    return cchain[x] != cchain[y] ? cchain[x] < cchain[y] : cc[x] > cc[y];
                });
                C.grp_off = (int)grouped.size();
                C.grp_first.assign(chain + 1, 0);
                for (int q : ord) {
                    grouped.push_back(ci[q]);
                    ++C.grp_first[cchain[q] + 1];
                }
                for (int c = 0; c < chain; ++c) C.grp_first[c + 1] += C.grp_first[c];
                if (!one) {  // largest items first
                    for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
                    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cc[x] > cc[y]; });
                    std::vector<LJItem> sorted;
                    for (int q : ord) sorted.push_back(ci[q]);
                    ci.swap(sorted);
                }
                C.item_off = (int)items.size();
                C.n_items = (int)ci.size();
                items.insert(items.end(), ci.begin(), ci.end());
                C.grid_grad = std::max(1, std::min(C.n_items, C.grid_grad));
                C.grid_nograd = std::max(1, std::min(C.n_items, C.grid_nograd));
            }
            if (P->lj_paired) {
                P->n_lanes = pipeline_lanes();
                for (auto& C : P->lj_cls) {
                    int ocap = 2;
                    for (auto& si : P->sys)
                        if (si.kind == PAMD_LJ && &P->lj_cls[si.lj_class] == &C)
                            ocap = std::max(ocap, si.tune.outer_cap);
                    C.outer_words = (long long)(ocap / 2) * C.NT;
                    P->outer_lane_words = std::max(P->outer_lane_words,
                                                   (long long)std::max(C.grid_grad, C.grid_nograd) * C.outer_words);
                }
                if ((rc0 = P->alloc(&P->d_outer, sizeof(uint32_t) * P->n_lanes * P->outer_lane_words)))
                    return rc0;
            }
            if (P->fp64)
                fill_lj_sys<double>(P.get(), p);
            else
                fill_lj_sys<float>(P.get(), p);
            if (std::getenv("PAMD_DEBUG_PLAN")) {
                for (auto& C : P->lj_cls)
                    std::fprintf(stderr, "pamd plan: paired=%d class NT=%d nmax=%d pipe=%d smem=%zu grid grad=%d "
                                 "nograd=%d items=%d\n", (int)P->lj_paired, C.NT, C.nmax, (int)C.pipe, C.smem,
                                 C.grid_grad, C.grid_nograd, C.n_items);
                for (auto& si : P->sys)
                    if (si.kind == PAMD_LJ)
                        std::fprintf(stderr, "  N=%d T=%d class=%d tpp=%d cap/thread=%d skin=%.3f tile=%d\n",
                                     si.N, si.T, si.lj_class, si.tune.tpp, si.tune.maxnb, si.tune.skin,
                                     si.tune.tile_steps);
            }
        }
    }
    P->n_lj_items = (int)items.size();
    P->n_S_slots = slot;
    P->h_E_slots = Eslots;
    int rc;
    if ((rc = P->alloc(&P->d_all, sizeof(ElemBlock) * P->h_all.size()))) return rc;
    if ((rc = P->alloc(&P->d_ho, sizeof(ElemBlock) * P->h_ho.size()))) return rc;
    if ((rc = P->alloc(&P->d_S_slots, sizeof(ChainSlots) * chain))) return rc;
    if ((rc = P->alloc(&P->d_E_slots, sizeof(ChainSlots) * chain))) return rc;
    if ((rc = P->alloc(&P->d_part_S, sizeof(double) * P->n_S_slots))) return rc;
    if ((rc = P->alloc(&P->d_part_qf, sizeof(double) * P->h_all.size()))) return rc;
    if ((rc = P->alloc(&P->d_part_qr, sizeof(double) * P->h_all.size()))) return rc;
    if ((rc = P->alloc(&P->d_lj_items, sizeof(LJItem) * items.size()))) return rc;
    if ((rc = P->alloc(&P->d_lj_items_grp, sizeof(LJItem) * grouped.size()))) return rc;
    if ((rc = P->alloc(&P->d_lj_sys, P->h_lj_sys.size()))) return rc;
    if ((rc = P->alloc(&P->d_counter, sizeof(int)))) return rc;
    if ((rc = P->alloc(&P->d_err, sizeof(int)))) return rc;
    PAMD_CUDA_TRY(cudaMemset(P->d_err, 0, sizeof(int)));
    if (!items.empty())
        PAMD_CUDA_TRY(cudaMemcpy(P->d_lj_items, items.data(), sizeof(LJItem) * items.size(),
                                 cudaMemcpyHostToDevice));
    if (!grouped.empty())
        PAMD_CUDA_TRY(cudaMemcpy(P->d_lj_items_grp, grouped.data(), sizeof(LJItem) * grouped.size(),
                                 cudaMemcpyHostToDevice));
    if (!P->h_lj_sys.empty())
        PAMD_CUDA_TRY(cudaMemcpy(P->d_lj_sys, P->h_lj_sys.data(), P->h_lj_sys.size(),
                                 cudaMemcpyHostToDevice));
    if (!P->h_all.empty())
        PAMD_CUDA_TRY(cudaMemcpy(P->d_all, P->h_all.data(), sizeof(ElemBlock) * P->h_all.size(),
                                 cudaMemcpyHostToDevice));
    if (!P->h_ho.empty())
        PAMD_CUDA_TRY(cudaMemcpy(P->d_ho, P->h_ho.data(), sizeof(ElemBlock) * P->h_ho.size(),
                                 cudaMemcpyHostToDevice));
    PAMD_CUDA_TRY(cudaMemcpy(P->d_S_slots, Sslots.data(), sizeof(ChainSlots) * chain,
                             cudaMemcpyHostToDevice));
    PAMD_CUDA_TRY(cudaMemcpy(P->d_E_slots, Eslots.data(), sizeof(ChainSlots) * chain,
                             cudaMemcpyHostToDevice));
    *out = P.get();
    g_plans[key] = std::move(P);
    return PAMD_OK;
}

int ensure_update_ws(Plan* P)
{
    if (P->d_prop) return PAMD_OK;
    int rc;
    if ((rc = P->alloc(&P->d_prop, P->esz * (size_t)P->span))) return rc;
    if ((rc = P->alloc(&P->d_gprop, P->esz * (size_t)P->span))) return rc;
    if ((rc = P->alloc(&P->d_Sprop, sizeof(double) * P->n_chains))) return rc;
    if ((rc = P->alloc(&P->d_qf, sizeof(double) * P->n_chains))) return rc;
    if ((rc = P->alloc(&P->d_qr, sizeof(double) * P->n_chains))) return rc;
    if ((rc = P->alloc(&P->d_flag, sizeof(int) * P->n_chains))) return rc;
    if (!P->d_md && (rc = P->alloc(&P->d_md, sizeof(MalaDev)))) return rc;
    PAMD_CUDA_TRY(cudaMemset(P->d_prop, 0, P->esz * (size_t)P->span));
    PAMD_CUDA_TRY(cudaMemset(P->d_gprop, 0, P->esz * (size_t)P->span));
    return PAMD_OK;
}

bool is_host_ptr(const void* ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

// S (and grad) of chains [c0, c1) into S_out (indexed by global chain), from
// device pointers; c1 < 0 means every chain.  The results of a chain do not
// depend on the range it is computed in.
template <typename R>
int run_action(const pamd_problem* p, Plan* P, const R* pos, R* grad, double* S_out, bool with_grad,
               cudaStream_t st, int c0 = 0, int c1 = -1, int* counter = nullptr, int lane = 0,
               const R* hs2 = nullptr, int* overlap = nullptr)
{
    if (c1 < 0) c1 = P->n_chains;
    if (!counter) counter = P->d_counter;  // LJ work-queue counter of this launch sequence
    const bool all = c0 == 0 && c1 == P->n_chains;
    const double a = p->beta * p->D * p->dt, ginv = 1.0 / (2.0 * p->D * p->dt);
    const bool one = (p->flags & PAMD_FLAG_ONE_CHAIN_PER_LAUNCH) != 0;
    // harmonic systems: one launch per system (per chain in the plain form)
    for (const auto& si : P->sys) {
        if (si.kind != PAMD_HARMONIC) continue;
        const int lo_c = std::max(c0, si.chain0), hi_c = std::min(c1, si.chain0 + si.chains);
        if (lo_c >= hi_c) continue;
        const int sz = si.d * si.N;
        const long long lo = si.off, hi = si.off + si.chain_len * si.chains;
        const bool slab = si.halo_lo || si.halo_hi;
        auto ho = [&](int b0, int nb) -> int {
            if (std::is_same<R, float>::value && sz <= 4)
                PAMD_CUDA_TRY(launch_ho_action_vec(P->d_ho + b0, nb, sz, (const float*)pos,
                                                   (float*)grad, P->d_part_S, b0, a, ginv, with_grad,
                                                   lo, hi, st, slab));
            else
                PAMD_CUDA_TRY(launch_ho_action<R>(P->d_ho + b0, nb, P->max_s_ho, pos, grad, P->d_part_S,
                                                  b0, a, ginv, with_grad, st, slab));
            return PAMD_OK;
        };
        int rc;
        if (one) {
            for (int c = lo_c; c < hi_c; ++c)
                if ((rc = ho(P->ho_chain_first[c], P->ho_chain_count[c]))) return rc;
        } else {
            const int b0 = P->ho_chain_first[lo_c];
            const int b1 = P->ho_chain_first[hi_c - 1] + P->ho_chain_count[hi_c - 1];
            if ((rc = ho(b0, b1 - b0))) return rc;
        }
    }
    // LJ systems: one persistent launch per block-size class, one after another on st
    for (int k = 0; k < (int)P->lj_cls.size(); ++k) {
        const LJClass& C = P->lj_cls[k];
        if (C.n_items <= 0) continue;
        const int grid = with_grad ? C.grid_grad : C.grid_nograd;
        auto launch = [&](const LJItem* items, int n, int g) {
            if (std::is_same<R, float>::value && P->lj_paired)
                return launch_lj_paired(items, n, P->d_lj_sys, (const float*)pos, (float*)grad,
                                        P->d_part_S, counter, C.NT, C.smem, g, with_grad, C.pipe,
                                        P->d_outer + (long long)lane * P->outer_lane_words,
                                        C.outer_words, st, (const float*)hs2, overlap);
            return launch_lj_items<R>(items, n, P->d_lj_sys, C.nmax, pos, grad, P->d_part_S, counter,
                                      C.NT, C.smem, g, with_grad, st, hs2, overlap);
        };
        if (one) {
            for (int c = c0; c < c1; ++c) {
                const int f = P->lj_chain_first[c];
                if (f < 0 || P->lj_chain_class[c] != k) continue;
                const int n = P->lj_chain_count[c];
                PAMD_CUDA_TRY(launch(P->d_lj_items + f, n, std::min(grid, n)));
            }
        } else if (all) {
            PAMD_CUDA_TRY(launch(P->d_lj_items + C.item_off, C.n_items, grid));
        } else {
            const int f = C.grp_first[c0], n = C.grp_first[c1] - f;
            if (n > 0) PAMD_CUDA_TRY(launch(P->d_lj_items_grp + C.grp_off + f, n, std::min(grid, n)));
        }
    }
    PAMD_CUDA_TRY(launch_finalize(P->d_part_S, P->d_S_slots + c0, c1 - c0, 1.0 / (4.0 * p->D * p->dt),
                                  S_out + c0, st, P->d_err));
    if (fault_injected("nonfinite")) PAMD_CUDA_TRY(launch_set_status(P->d_err, PAMD_ERR_NONFINITE, st));
    return PAMD_OK;
}

// One path update of chains [c0, c1) (c1 < 0: every chain); arrays indexed by
// global chain.
template <typename R>
int run_one_update(const pamd_problem* p, Plan* P, R* pos, R* grad, double* S, const R* noise,
                   const double* log_u, int* n_acc, double* la, int u, cudaStream_t st, int c0 = 0,
                   int c1 = -1, int* counter = nullptr, int lane = 0)
{
    if (c1 < 0) c1 = P->n_chains;
    const int eb0 = P->h_E_slots[c0].begin, eb1 = P->h_E_slots[c1 - 1].end;
    R* prop = reinterpret_cast<R*>(P->d_prop);
    R* gprop = reinterpret_cast<R*>(P->d_gprop);
    PAMD_CUDA_TRY(launch_mala_propose<R>(P->d_all + eb0, eb1 - eb0, pos, grad, noise, prop,
                                         P->d_part_qf + eb0, P->d_md, u, st, P->any_slab));
    int rc = run_action<R>(p, P, prop, gprop, P->d_Sprop, true, st, c0, c1, counter, lane);
    if (rc) return rc;
    PAMD_CUDA_TRY(launch_mala_reverse<R>(P->d_all + eb0, eb1 - eb0, pos, prop, gprop,
                                         P->d_part_qr + eb0, P->d_md, st, P->any_slab));
    PAMD_CUDA_TRY(launch_finalize(P->d_part_qf, P->d_E_slots + c0, c1 - c0, 1.0, P->d_qf + c0, st));
    PAMD_CUDA_TRY(launch_finalize(P->d_part_qr, P->d_E_slots + c0, c1 - c0, 1.0, P->d_qr + c0, st));
    PAMD_CUDA_TRY(launch_mala_accept(c0, c1 - c0, S, P->d_Sprop, P->d_qf, P->d_qr, log_u, P->d_md, u,
                                     P->d_flag, n_acc, la, st));
    PAMD_CUDA_TRY(launch_mala_commit<R>(P->d_all + eb0, eb1 - eb0, pos, grad, prop, gprop, P->d_flag,
                                        S, P->d_Sprop, st));
    return PAMD_OK;
}

// Path updates with host buffers (no explicit noise or uniforms), pipelined over
// chunks of chains: chunk k's inputs are copied in on one stream while earlier
// chunks are updated and copied back on others.  Updates alternate between the
// caller's stream and a second compute stream, each chunk with its own LJ work
// counter, so that the last items of one chunk overlap the next chunk.  Chains
// are independent, so the results equal those of one update over all.
template <typename R>
int path_update_pipelined(const pamd_problem* prob, Plan* P, void* pos, void* grad, double* S,
                          int n_updates, int* n_accepted, double* log_alpha, cudaStream_t st)
{
    int rc;
    const size_t esz = P->esz;
    const int nc = P->n_chains;
    const size_t bytes = esz * (size_t)P->span;
    const bool hp = is_host_ptr(pos), hg = is_host_ptr(grad), hS = is_host_ptr(S);
    const bool hn = n_accepted && is_host_ptr(n_accepted);
    const bool hl = log_alpha && is_host_ptr(log_alpha);
    if (hp && !P->d_stage_pos && (rc = P->alloc(&P->d_stage_pos, bytes))) return rc;
    if (hg && !P->d_stage_grad && (rc = P->alloc(&P->d_stage_grad, bytes))) return rc;
    if (hS && !P->d_stage_S && (rc = P->alloc(&P->d_stage_S, sizeof(double) * nc))) return rc;
    if (hn && !P->d_stage_int && (rc = P->alloc(&P->d_stage_int, sizeof(int) * nc))) return rc;
    if (hl && !P->d_stage_dbl && (rc = P->alloc(&P->d_stage_dbl, sizeof(double) * nc))) return rc;
    char* dpos = hp ? (char*)P->d_stage_pos : (char*)pos;
    char* dgrad = hg ? (char*)P->d_stage_grad : (char*)grad;
    double* dS = hS ? P->d_stage_S : S;
    int* dnacc = hn ? P->d_stage_int : n_accepted;
    double* dla = hl ? P->d_stage_dbl : log_alpha;
    constexpr int kMaxChunks = 8;
    if (!P->s_in) {
        PAMD_CUDA_TRY(cudaStreamCreateWithFlags(&P->s_in, cudaStreamNonBlocking));
        PAMD_CUDA_TRY(cudaStreamCreateWithFlags(&P->s_out, cudaStreamNonBlocking));
    }
    while ((int)P->s_cmp.size() < P->n_lanes - 1) {
        cudaStream_t c;
        PAMD_CUDA_TRY(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        P->s_cmp.push_back(c);
    }
    if (!P->d_chunk_counters && (rc = P->alloc(&P->d_chunk_counters, sizeof(int) * kMaxChunks)))
        return rc;
    // events: per chunk inputs-copied, updated, results-copied; start and end (timed,
    // for the timeline that pamd_pipeline_timeline reports)
    while ((int)P->events.size() < 3 * kMaxChunks + 2) {
        cudaEvent_t e;
        PAMD_CUDA_TRY(cudaEventCreate(&e));
        P->events.push_back(e);
    }
    // Element extent of each chain, and chunk boundaries balanced by elements.
    auto e_begin = [&](int c) { return P->h_all[P->h_E_slots[c].begin].chain_base; };
    auto e_end = [&](int c) {
        const ElemBlock& B = P->h_all[P->h_E_slots[c].begin];
        return B.chain_base + B.chain_len;
    };
    const int K = std::min(nc, kMaxChunks);
    long long total = 0;
    for (int c = 0; c < nc; ++c) total += e_end(c) - e_begin(c);
    std::vector<int> cut(K + 1, nc);
    cut[0] = 0;
    {
        long long run = 0;
        int k = 1;
        for (int c = 0; c < nc && k < K; ++c) {
            run += e_end(c) - e_begin(c);
            // close chunk k-1 after chain c once it holds its share, leaving a chain per later chunk
            if ((run * K >= total * k || nc - (c + 1) == K - k) && nc - (c + 1) >= K - k) cut[k++] = c + 1;
        }
    }
    cudaEvent_t ev_start = P->events[3 * kMaxChunks], ev_fin = P->events[3 * kMaxChunks + 1];
    PAMD_CUDA_TRY(cudaEventRecord(ev_start, st));  // host buffers may be written by earlier work on st
    PAMD_CUDA_TRY(cudaStreamWaitEvent(P->s_in, ev_start, 0));
    for (cudaStream_t c : P->s_cmp) PAMD_CUDA_TRY(cudaStreamWaitEvent(c, ev_start, 0));
    for (int k = 0; k < K; ++k) {
        const int c0 = cut[k], c1 = cut[k + 1];
        if (c0 >= c1) continue;
        const long long e0 = e_begin(c0), e1 = e_end(c1 - 1);
        const size_t off = esz * (size_t)e0, nb = esz * (size_t)(e1 - e0);
        if (hp) PAMD_CUDA_TRY(cudaMemcpyAsync(dpos + off, (char*)pos + off, nb, cudaMemcpyHostToDevice, P->s_in));
        if (hg) PAMD_CUDA_TRY(cudaMemcpyAsync(dgrad + off, (char*)grad + off, nb, cudaMemcpyHostToDevice, P->s_in));
        if (hS)
            PAMD_CUDA_TRY(cudaMemcpyAsync(dS + c0, S + c0, sizeof(double) * (c1 - c0), cudaMemcpyHostToDevice,
                                          P->s_in));
        if (hn)
            PAMD_CUDA_TRY(cudaMemcpyAsync(dnacc + c0, n_accepted + c0, sizeof(int) * (c1 - c0),
                                          cudaMemcpyHostToDevice, P->s_in));
        const int lane = k % P->n_lanes;
        cudaStream_t cs = lane ? P->s_cmp[lane - 1] : st;
        PAMD_CUDA_TRY(cudaEventRecord(P->events[3 * k], P->s_in));
        PAMD_CUDA_TRY(cudaStreamWaitEvent(cs, P->events[3 * k], 0));
        for (int u = 0; u < n_updates; ++u)
            if ((rc = run_one_update<R>(prob, P, (R*)dpos, (R*)dgrad, dS, nullptr, nullptr, dnacc, dla,
                                        u, cs, c0, c1, P->d_chunk_counters + k, lane)))
                return rc;
        PAMD_CUDA_TRY(cudaEventRecord(P->events[3 * k + 1], cs));
        PAMD_CUDA_TRY(cudaStreamWaitEvent(P->s_out, P->events[3 * k + 1], 0));
        if (hp) PAMD_CUDA_TRY(cudaMemcpyAsync((char*)pos + off, dpos + off, nb, cudaMemcpyDeviceToHost, P->s_out));
        if (hg) PAMD_CUDA_TRY(cudaMemcpyAsync((char*)grad + off, dgrad + off, nb, cudaMemcpyDeviceToHost, P->s_out));
        if (hS)
            PAMD_CUDA_TRY(cudaMemcpyAsync(S + c0, dS + c0, sizeof(double) * (c1 - c0), cudaMemcpyDeviceToHost,
                                          P->s_out));
        if (hn)
            PAMD_CUDA_TRY(cudaMemcpyAsync(n_accepted + c0, dnacc + c0, sizeof(int) * (c1 - c0),
                                          cudaMemcpyDeviceToHost, P->s_out));
        if (hl)
            PAMD_CUDA_TRY(cudaMemcpyAsync(log_alpha + c0, dla + c0, sizeof(double) * (c1 - c0),
                                          cudaMemcpyDeviceToHost, P->s_out));
        PAMD_CUDA_TRY(cudaEventRecord(P->events[3 * k + 2], P->s_out));
    }
    PAMD_CUDA_TRY(cudaEventRecord(ev_fin, P->s_out));
    PAMD_CUDA_TRY(cudaStreamWaitEvent(st, ev_fin, 0));
    PAMD_CUDA_TRY(cudaStreamSynchronize(st));
    // timeline of this call
    std::vector<float> tl(1 + 3 * K, 0.0f);
    PAMD_CUDA_TRY(cudaEventElapsedTime(&tl[0], ev_start, ev_fin));
    for (int k = 0; k < K; ++k) {
        if (cut[k] >= cut[k + 1]) continue;
        for (int q = 0; q < 3; ++q)
            PAMD_CUDA_TRY(cudaEventElapsedTime(&tl[1 + 3 * k + q], ev_start, P->events[3 * k + q]));
    }
    g_last_timeline.swap(tl);
    return PAMD_OK;
}

}  // namespace

extern "C" {

int pamd_version(void) { return 1; }

const char* pamd_status_string(int status)
{
    switch (status) {
        case PAMD_OK: return "ok";
        case PAMD_ERR_ARG: return "invalid argument";
        case PAMD_ERR_UNSUPPORTED: return "unsupported shape";
        case PAMD_ERR_CUDA: return "CUDA error";
        case PAMD_ERR_TIMEOUT: return "device wait timed out";
        case PAMD_ERR_NONFINITE: return "non-finite action";
        case PAMD_ERR_ALLOC: return "workspace allocation failed";
        default: return "unknown status";
    }
}

int pamd_release_cache(void)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    cudaDeviceSynchronize();
    g_plans.clear();
    return PAMD_OK;
}

int pamd_debug_status(int* checked, int* count, int* site, long long* index, long long* bound)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    if (cudaDeviceSynchronize() != cudaSuccess) return PAMD_ERR_CUDA;
#ifdef PAMD_DEBUG
    const int compiled = 1;
#else
    const int compiled = 0;
#endif
    int (*const fetch[])(DebugRecord*) = {debug_fetch_ho, debug_fetch_lj, debug_fetch_lj_paired,
                                          debug_fetch_update, debug_fetch_fragment};
    int total = 0, first_site = 0;
    long long first_index = 0, first_bound = 0;
    for (int f = 0; f < 5; ++f) {
        DebugRecord r;
        if (fetch[f](&r)) return PAMD_ERR_CUDA;
        if (r.count && !total) {
            first_site = (f + 1) * 100000 + r.site;
            first_index = r.index;
            first_bound = r.bound;
        }
        total += r.count;
    }
    if (checked) *checked = compiled;
    if (count) *count = total;
    if (site) *site = first_site;
    if (index) *index = first_index;
    if (bound) *bound = first_bound;
    return PAMD_OK;
}

int pamd_pipeline_timeline(float* ms, int max_entries, int* n_chunks)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    if (max_entries < 0 || (max_entries > 0 && !ms)) return PAMD_ERR_ARG;
    const int n = (int)g_last_timeline.size();
    if (n_chunks) *n_chunks = n ? (n - 1) / 3 : 0;
    for (int q = 0; q < std::min(n, max_entries); ++q) ms[q] = g_last_timeline[q];
    return PAMD_OK;
}

int pamd_cache_stats(int* n_plans, int* n_graphs)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    int g = 0;
    for (auto& kv : g_plans) g += (int)kv.second->graphs.size();
    if (n_plans) *n_plans = (int)g_plans.size();
    if (n_graphs) *n_graphs = g;
    return PAMD_OK;
}

int pamd_device_status(void* stream)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PAMD_ERR_CUDA;
    int worst = PAMD_OK;
    for (auto& kv : g_plans) {
        int v = 0;
        if (cudaMemcpy(&v, kv.second->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return PAMD_ERR_CUDA;
        if (v != PAMD_OK) {
            worst = v;
            cudaMemset(kv.second->d_err, 0, sizeof(int));
        }
    }
    return worst;
}

int pamd_tune(int tile_steps, int threads_per_particle, int max_neighbours, double skin,
              int window_steps)
{
    if (threads_per_particle != 0 && threads_per_particle != 1 && threads_per_particle != 2 &&
        threads_per_particle != 4)
        return PAMD_ERR_ARG;
    if (tile_steps < 0 || max_neighbours < 0 || window_steps < 0 || window_steps == 1)
        return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    g_tune_override.tile_steps = tile_steps;
    g_tune_override.tpp = threads_per_particle;
    g_tune_override.maxnb = max_neighbours;
    g_tune_override.skin = skin;
    g_tune_override.window = window_steps;
    return PAMD_OK;
}

static int action_common(const pamd_problem* prob, const void* pos, double* S, void* grad,
                         bool with_grad, void* stream)
{
    NvtxRange nvtx_(with_grad ? "pamd_action_grad" : "pamd_action");
    if (any_misaligned({pos, grad})) return PAMD_ERR_ARG;
    int rc = check_em_problem(prob);
    if (rc) return rc;
    if (!pos || !S || (with_grad && !grad)) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    if ((rc = build_plan(prob, &P))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const bool host = is_host_ptr(pos) || is_host_ptr(S) || (with_grad && is_host_ptr(grad));
    const void* dpos = pos;
    void* dgrad = grad;
    double* dS = S;
    const size_t bytes = P->esz * (size_t)P->span;
    if (host) {
        if (!P->d_stage_pos && (rc = P->alloc(&P->d_stage_pos, bytes))) return rc;
        if (with_grad && !P->d_stage_grad && (rc = P->alloc(&P->d_stage_grad, bytes))) return rc;
        if (!P->d_stage_S && (rc = P->alloc(&P->d_stage_S, sizeof(double) * P->n_chains))) return rc;
        if (is_host_ptr(pos)) {
            PAMD_CUDA_TRY(cudaMemcpyAsync(P->d_stage_pos, pos, bytes, cudaMemcpyHostToDevice, st));
            dpos = P->d_stage_pos;
        }
        if (with_grad && is_host_ptr(grad)) dgrad = P->d_stage_grad;
        if (is_host_ptr(S)) dS = P->d_stage_S;
    }
    if (P->fp64)
        rc = run_action<double>(prob, P, (const double*)dpos, (double*)dgrad, dS, with_grad, st);
    else
        rc = run_action<float>(prob, P, (const float*)dpos, (float*)dgrad, dS, with_grad, st);
    if (rc) return rc;
    if (host) {
        if (with_grad && dgrad != grad)
            PAMD_CUDA_TRY(cudaMemcpyAsync(grad, dgrad, bytes, cudaMemcpyDeviceToHost, st));
        if (dS != S)
            PAMD_CUDA_TRY(cudaMemcpyAsync(S, dS, sizeof(double) * P->n_chains, cudaMemcpyDeviceToHost, st));
        PAMD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return PAMD_OK;
}

int pamd_action_grad_hs(const pamd_problem* prob, const void* pos, const double* sigma_hs, double* S,
                        void* grad, void* stream)
{
    NvtxRange nvtx_("pamd_action_grad_hs");
    if (any_misaligned({pos, grad})) return PAMD_ERR_ARG;
    int rc = check_em_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !sigma_hs || !S) return PAMD_ERR_ARG;
    for (const void* b : {pos, (const void*)sigma_hs, (const void*)S, (const void*)grad})
        if (b && is_host_ptr(b)) return PAMD_ERR_ARG;  // device buffers only
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    if ((rc = build_plan(prob, &P))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->hs_slices > 0 && !P->d_hs2) {
        if ((rc = P->alloc(&P->d_hs2, P->esz * (size_t)P->hs_slices))) return rc;
        if ((rc = P->alloc(&P->d_overlap, sizeof(int) * (size_t)P->n_chains))) return rc;
    }
    const bool with_grad = grad != nullptr;
    if (P->hs_slices > 0) {
        PAMD_CUDA_TRY(cudaMemsetAsync(P->d_overlap, 0, sizeof(int) * (size_t)P->n_chains, st));
        if (P->fp64)
            PAMD_CUDA_TRY(launch_hs_square<double>(sigma_hs, (double*)P->d_hs2, P->hs_slices, st));
        else
            PAMD_CUDA_TRY(launch_hs_square<float>(sigma_hs, (float*)P->d_hs2, P->hs_slices, st));
    }
    if (P->fp64)
        rc = run_action<double>(prob, P, (const double*)pos, (double*)grad, S, with_grad, st, 0, -1,
                                nullptr, 0, (const double*)P->d_hs2, P->d_overlap);
    else
        rc = run_action<float>(prob, P, (const float*)pos, (float*)grad, S, with_grad, st, 0, -1,
                               nullptr, 0, (const float*)P->d_hs2, P->d_overlap);
    if (rc) return rc;
    if (P->hs_slices > 0) {
        // the last slice of every chain that owns it (the force walks stop at T-1)
        for (const auto& si : P->sys) {
            if (si.kind != PAMD_LJ || si.halo_hi) continue;
            const void* row = &P->h_lj_sys[P->lj_sys_stride * si.lj_index];
            const long long off = si.hs_off + si.T;
            if (P->fp64)
                PAMD_CUDA_TRY(launch_lj_hs_slice<double>((const double*)pos, row, si.chains, si.T,
                                                         (const double*)P->d_hs2 + off, P->d_overlap, st));
            else
                PAMD_CUDA_TRY(launch_lj_hs_slice<float>((const float*)pos, row, si.chains, si.T,
                                                        (const float*)P->d_hs2 + off, P->d_overlap, st));
        }
        PAMD_CUDA_TRY(launch_hs_fixup(S, P->d_overlap, P->n_chains, st));
    }
    return PAMD_OK;
}

int pamd_action(const pamd_problem* prob, const void* pos, double* S, void* stream)
{
    return action_common(prob, pos, S, nullptr, false, stream);
}

int pamd_action_grad(const pamd_problem* prob, const void* pos, double* S, void* grad, void* stream)
{
    return action_common(prob, pos, S, grad, true, stream);
}

int pamd_path_update(const pamd_problem* prob, void* pos, void* grad, double* S, double h,
                     int n_updates, uint64_t seed, uint64_t counter, const void* noise,
                     const double* log_u, int* n_accepted, double* log_alpha, void* stream)
{
    NvtxRange nvtx_("pamd_path_update");
    if (any_misaligned({pos, grad, noise})) return PAMD_ERR_ARG;
    int rc = check_em_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !grad || !S || !(h > 0) || n_updates < 0) return PAMD_ERR_ARG;
    if ((noise || log_u) && n_updates != 1) return PAMD_ERR_ARG;
    if (n_updates == 0) return PAMD_OK;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    if ((rc = build_plan(prob, &P))) return rc;
    if ((rc = ensure_update_ws(P))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = P->esz * (size_t)P->span;
    const size_t nc = (size_t)P->n_chains;
    const bool host = is_host_ptr(pos) || is_host_ptr(grad) || is_host_ptr(S) ||
                      is_host_ptr(noise) || is_host_ptr(log_u) || is_host_ptr(n_accepted) ||
                      is_host_ptr(log_alpha);
    if (host && !noise && !log_u && P->n_chains >= 2) {
        PAMD_CUDA_TRY(launch_set_mala_params(P->d_md, seed, counter, h, st));
        return P->fp64 ? path_update_pipelined<double>(prob, P, pos, grad, S, n_updates, n_accepted,
                                                       log_alpha, st)
                       : path_update_pipelined<float>(prob, P, pos, grad, S, n_updates, n_accepted,
                                                      log_alpha, st);
    }
    void *dpos = pos, *dgrad = grad;
    double* dS = S;
    const void* dnoise = noise;
    const double* dlogu = log_u;
    int* dnacc = n_accepted;
    double* dla = log_alpha;
    if (host) {
        if (!P->d_stage_pos && (rc = P->alloc(&P->d_stage_pos, bytes))) return rc;
        if (!P->d_stage_grad && (rc = P->alloc(&P->d_stage_grad, bytes))) return rc;
        if (!P->d_stage_S && (rc = P->alloc(&P->d_stage_S, sizeof(double) * nc))) return rc;
        if (!P->d_stage_dbl && (rc = P->alloc(&P->d_stage_dbl, sizeof(double) * nc))) return rc;
        if (!P->d_stage_logu && (rc = P->alloc(&P->d_stage_logu, sizeof(double) * nc))) return rc;
        if (!P->d_stage_int && (rc = P->alloc(&P->d_stage_int, sizeof(int) * nc))) return rc;
        if (noise && !P->d_stage_noise && (rc = P->alloc(&P->d_stage_noise, bytes))) return rc;
        if (is_host_ptr(pos)) {
            dpos = P->d_stage_pos;
            PAMD_CUDA_TRY(cudaMemcpyAsync(dpos, pos, bytes, cudaMemcpyHostToDevice, st));
        }
        if (is_host_ptr(grad)) {
            dgrad = P->d_stage_grad;
            PAMD_CUDA_TRY(cudaMemcpyAsync(dgrad, grad, bytes, cudaMemcpyHostToDevice, st));
        }
        if (is_host_ptr(S)) {
            dS = P->d_stage_S;
            PAMD_CUDA_TRY(cudaMemcpyAsync(dS, S, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
        }
        if (noise && is_host_ptr(noise)) {
            dnoise = P->d_stage_noise;
            PAMD_CUDA_TRY(cudaMemcpyAsync(P->d_stage_noise, noise, bytes, cudaMemcpyHostToDevice, st));
        }
        if (log_u && is_host_ptr(log_u)) {
            dlogu = P->d_stage_logu;
            PAMD_CUDA_TRY(cudaMemcpyAsync(P->d_stage_logu, log_u, sizeof(double) * nc,
                                          cudaMemcpyHostToDevice, st));
        }
        if (n_accepted && is_host_ptr(n_accepted)) {
            dnacc = P->d_stage_int;
            PAMD_CUDA_TRY(cudaMemcpyAsync(dnacc, n_accepted, sizeof(int) * nc, cudaMemcpyHostToDevice, st));
        }
        if (log_alpha && is_host_ptr(log_alpha)) dla = P->d_stage_dbl;
    }
    PAMD_CUDA_TRY(launch_set_mala_params(P->d_md, seed, counter, h, st));
    const bool use_graph = !host && n_updates > 1;
    if (!use_graph) {
        for (int u = 0; u < n_updates; ++u) {
            rc = P->fp64 ? run_one_update<double>(prob, P, (double*)dpos, (double*)dgrad, dS,
                                                  (const double*)dnoise, dlogu, dnacc, dla, u, st)
                         : run_one_update<float>(prob, P, (float*)dpos, (float*)dgrad, dS,
                                                 (const float*)dnoise, dlogu, dnacc, dla, u, st);
            if (rc) return rc;
        }
    } else {
        GraphKey gk{dpos, dgrad, dS, dnacc, dla, n_updates};
        auto it = P->graphs.find(gk);
        if (it == P->graphs.end()) {
            cudaStream_t cap;
            PAMD_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                cudaStreamDestroy(cap);
                return PAMD_ERR_CUDA;
            }
            for (int u = 0; u < n_updates && !rc; ++u)
                rc = P->fp64 ? run_one_update<double>(prob, P, (double*)dpos, (double*)dgrad, dS,
                                                      nullptr, nullptr, dnacc, dla, u, cap)
                             : run_one_update<float>(prob, P, (float*)dpos, (float*)dgrad, dS,
                                                     nullptr, nullptr, dnacc, dla, u, cap);
            cudaError_t ce = cudaStreamEndCapture(cap, &g);
            cudaStreamDestroy(cap);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return PAMD_ERR_CUDA;
            cudaGraphExec_t ex;
            ce = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return PAMD_ERR_CUDA;
            it = P->graphs.emplace(gk, ex).first;
        }
        PAMD_CUDA_TRY(cudaGraphLaunch(it->second, st));
    }
    if (host) {
        if (dpos != pos) PAMD_CUDA_TRY(cudaMemcpyAsync(pos, dpos, bytes, cudaMemcpyDeviceToHost, st));
        if (dgrad != grad) PAMD_CUDA_TRY(cudaMemcpyAsync(grad, dgrad, bytes, cudaMemcpyDeviceToHost, st));
        if (dS != S) PAMD_CUDA_TRY(cudaMemcpyAsync(S, dS, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
        if (dnacc != n_accepted)
            PAMD_CUDA_TRY(cudaMemcpyAsync(n_accepted, dnacc, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
        if (dla != log_alpha)
            PAMD_CUDA_TRY(cudaMemcpyAsync(log_alpha, dla, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
        PAMD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return PAMD_OK;
}

// ------------------------------------------------------------------ update in pieces
// The kernels of run_one_update, one piece per call, on the caller's buffers.
static int mala_piece_plan(const pamd_problem* prob, std::initializer_list<const void*> bufs,
                           Plan** P)
{
    int rc = check_em_problem(prob);
    if (rc) return rc;
    for (const void* b : bufs)
        if (!b || is_host_ptr(b)) return PAMD_ERR_ARG;  // device buffers only
    if ((rc = build_plan(prob, P))) return rc;
    if (!(*P)->d_md && (rc = (*P)->alloc(&(*P)->d_md, sizeof(MalaDev)))) return rc;
    return PAMD_OK;
}

int pamd_mala_propose(const pamd_problem* prob, const void* pos, const void* grad, void* prop,
                      double h, uint64_t seed, uint64_t counter, const void* noise, double* q_fwd,
                      void* stream)
{
    NvtxRange nvtx_("pamd_mala_propose");
    if (any_misaligned({pos, grad, prop, noise})) return PAMD_ERR_ARG;
    if (!(h > 0) || (noise && is_host_ptr(noise))) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    int rc = mala_piece_plan(prob, {pos, grad, prop, q_fwd}, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)P->h_all.size();
    PAMD_CUDA_TRY(launch_set_mala_params(P->d_md, seed, counter, h, st));
    if (P->fp64)
        PAMD_CUDA_TRY(launch_mala_propose<double>(P->d_all, nb, (const double*)pos, (const double*)grad,
                                                  (const double*)noise, (double*)prop, P->d_part_qf,
                                                  P->d_md, 0, st, P->any_slab));
    else
        PAMD_CUDA_TRY(launch_mala_propose<float>(P->d_all, nb, (const float*)pos, (const float*)grad,
                                                 (const float*)noise, (float*)prop, P->d_part_qf,
                                                 P->d_md, 0, st, P->any_slab));
    PAMD_CUDA_TRY(launch_finalize(P->d_part_qf, P->d_E_slots, P->n_chains, 1.0, q_fwd, st));
    return PAMD_OK;
}

int pamd_mala_reverse(const pamd_problem* prob, const void* pos, const void* prop,
                      const void* grad_prop, double h, double* q_rev, void* stream)
{
    NvtxRange nvtx_("pamd_mala_reverse");
    if (any_misaligned({pos, prop, grad_prop})) return PAMD_ERR_ARG;
    if (!(h > 0)) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    int rc = mala_piece_plan(prob, {pos, prop, grad_prop, q_rev}, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)P->h_all.size();
    PAMD_CUDA_TRY(launch_set_mala_params(P->d_md, 0, 0, h, st));
    if (P->fp64)
        PAMD_CUDA_TRY(launch_mala_reverse<double>(P->d_all, nb, (const double*)pos, (const double*)prop,
                                                  (const double*)grad_prop, P->d_part_qr, P->d_md, st,
                                                  P->any_slab));
    else
        PAMD_CUDA_TRY(launch_mala_reverse<float>(P->d_all, nb, (const float*)pos, (const float*)prop,
                                                 (const float*)grad_prop, P->d_part_qr, P->d_md, st,
                                                 P->any_slab));
    PAMD_CUDA_TRY(launch_finalize(P->d_part_qr, P->d_E_slots, P->n_chains, 1.0, q_rev, st));
    return PAMD_OK;
}

int pamd_mala_accept(const pamd_problem* prob, const double* S, const double* S_prop,
                     const double* q_fwd, const double* q_rev, double h, uint64_t seed,
                     uint64_t counter, const double* log_u, int* accept, int* n_accepted,
                     double* log_alpha, void* stream)
{
    NvtxRange nvtx_("pamd_mala_accept");
    if (!(h > 0)) return PAMD_ERR_ARG;
    for (const void* b : {(const void*)log_u, (const void*)n_accepted, (const void*)log_alpha})
        if (b && is_host_ptr(b)) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    int rc = mala_piece_plan(prob, {S, S_prop, q_fwd, q_rev, accept}, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    PAMD_CUDA_TRY(launch_set_mala_params(P->d_md, seed, counter, h, st));
    PAMD_CUDA_TRY(launch_mala_accept(0, P->n_chains, S, S_prop, q_fwd, q_rev, log_u, P->d_md, 0,
                                     accept, n_accepted, log_alpha, st));
    return PAMD_OK;
}

int pamd_mala_commit(const pamd_problem* prob, void* pos, void* grad, double* S, const void* prop,
                     const void* grad_prop, const double* S_prop, const int* accept, void* stream)
{
    NvtxRange nvtx_("pamd_mala_commit");
    if (any_misaligned({pos, grad, prop, grad_prop})) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    int rc = mala_piece_plan(prob, {pos, grad, S, prop, grad_prop, S_prop, accept}, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)P->h_all.size();
    if (P->fp64)
        PAMD_CUDA_TRY(launch_mala_commit<double>(P->d_all, nb, (double*)pos, (double*)grad,
                                                 (const double*)prop, (const double*)grad_prop,
                                                 accept, S, S_prop, st));
    else
        PAMD_CUDA_TRY(launch_mala_commit<float>(P->d_all, nb, (float*)pos, (float*)grad,
                                                (const float*)prop, (const float*)grad_prop, accept,
                                                S, S_prop, st));
    return PAMD_OK;
}

int pamd_euler_reference(const pamd_problem* prob, void* pos, uint64_t seed, uint64_t counter,
                         const void* noise, void* stream)
{
    NvtxRange nvtx_("pamd_euler_reference");
    if (any_misaligned({pos, noise})) return PAMD_ERR_ARG;
    int rc = check_em_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos) return PAMD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mutex);
    Plan* P;
    if ((rc = build_plan(prob, &P))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = P->esz * (size_t)P->span;
    const bool host = is_host_ptr(pos) || is_host_ptr(noise);
    void* dpos = pos;
    const void* dnoise = noise;
    if (host) {
        if (!P->d_stage_pos && (rc = P->alloc(&P->d_stage_pos, bytes))) return rc;
        if (noise && !P->d_stage_noise && (rc = P->alloc(&P->d_stage_noise, bytes))) return rc;
        if (is_host_ptr(pos)) {
            dpos = P->d_stage_pos;
            PAMD_CUDA_TRY(cudaMemcpyAsync(dpos, pos, bytes, cudaMemcpyHostToDevice, st));
        }
        if (noise && is_host_ptr(noise)) {
            dnoise = P->d_stage_noise;
            PAMD_CUDA_TRY(cudaMemcpyAsync(P->d_stage_noise, noise, bytes, cudaMemcpyHostToDevice, st));
        }
    }
    const double a = prob->beta * prob->D * prob->dt, sig = std::sqrt(2.0 * prob->D * prob->dt);
    for (const auto& si : P->sys) {
        if (si.kind == PAMD_HARMONIC) {
            if (P->fp64)
                PAMD_CUDA_TRY(launch_ho_euler<double>((double*)dpos, (const double*)dnoise, si.d * si.N,
                                                      si.T, si.chains, si.off, si.chain0, si.pot.k, a,
                                                      sig, seed, counter, st));
            else
                PAMD_CUDA_TRY(launch_ho_euler<float>((float*)dpos, (const float*)dnoise, si.d * si.N,
                                                     si.T, si.chains, si.off, si.chain0, si.pot.k, a,
                                                     sig, seed, counter, st));
        } else {
            const void* row = &P->h_lj_sys[P->lj_sys_stride * si.lj_index];
            const size_t smem = lj_smem_bytes(si.N, si.NT, si.tune.maxnb, P->fp64);
            if (P->fp64)
                PAMD_CUDA_TRY(launch_lj_euler<double>((double*)dpos, (const double*)dnoise, row,
                                                      si.NT, smem, si.chains, si.chain0, seed,
                                                      counter, st));
            else
                PAMD_CUDA_TRY(launch_lj_euler<float>((float*)dpos, (const float*)dnoise, row,
                                                     si.NT, smem, si.chains, si.chain0, seed,
                                                     counter, st));
        }
    }
    if (host) {
        if (dpos != pos) PAMD_CUDA_TRY(cudaMemcpyAsync(pos, dpos, bytes, cudaMemcpyDeviceToHost, st));
        PAMD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return PAMD_OK;
}

int pamd_fragment_mc(const pamd_problem* prob, void* pos, int l_min, int l_max, int n_steps,
                     uint64_t seed, uint64_t counter, const int* levels, const int* offsets,
                     const void* noise, const double* log_u, int* n_accepted, int* n_proposed,
                     void* stream)
{
    NvtxRange nvtx_("pamd_fragment_mc");
    if (any_misaligned({pos, noise})) return PAMD_ERR_ARG;
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !n_accepted || !n_proposed || n_steps < 0 || l_min < 1 || l_max < l_min || l_max > 30)
        return PAMD_ERR_ARG;
    if ((levels || offsets || noise || log_u) && n_steps != 1) return PAMD_ERR_ARG;
    if ((levels == nullptr) != (offsets == nullptr)) return PAMD_ERR_ARG;
    int Tmax = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        if (s.pot.kind != PAMD_HARMONIC) return PAMD_ERR_UNSUPPORTED;
        if ((1LL << l_max) > s.n_steps) return PAMD_ERR_ARG;
        Tmax = std::max(Tmax, s.n_steps);
    }
    for (const void* ptr : {(const void*)pos, (const void*)levels, (const void*)offsets, noise,
                            (const void*)log_u, (const void*)n_accepted, (const void*)n_proposed})
        if (ptr && is_host_ptr(ptr)) return PAMD_ERR_ARG;  // device buffers only
    const int fstride = (Tmax >> l_min) + 2;
    cudaStream_t st = (cudaStream_t)stream;
    const double sig = std::sqrt(2.0 * prob->D * prob->dt), c0 = 1.0 / (4.0 * prob->D * prob->dt);
    for (int u = 0; u < n_steps; ++u) {
        int chain0 = 0;
        for (int q = 0; q < prob->n_systems; ++q) {
            const pamd_system& s = prob->systems[q];
            const int M = s.dim * s.n_particles;
            double g, cS;
            ho_step_constants(prob, s.pot.k, &g, &cS);
            if (prob->precision == PAMD_FP64)
                PAMD_CUDA_TRY(launch_fragment_mc<double>((double*)pos, s.pos_offset, s.n_steps, M,
                                                         s.n_chains, chain0, l_min, l_max, seed,
                                                         counter + u, levels, offsets,
                                                         (const double*)noise, log_u, fstride, g,
                                                         sig, cS, c0, n_accepted, n_proposed, st));
            else
                PAMD_CUDA_TRY(launch_fragment_mc<float>((float*)pos, s.pos_offset, s.n_steps, M,
                                                        s.n_chains, chain0, l_min, l_max, seed,
                                                        counter + u, levels, offsets,
                                                        (const float*)noise, log_u, fstride, g, sig,
                                                        cS, c0, n_accepted, n_proposed, st));
            chain0 += s.n_chains;
        }
    }
    return PAMD_OK;
}

int pamd_event(const pamd_problem* prob, void* pos, void* pos_out, int n_sample, int n_shift,
               int l_min, int l_max, void* traj, uint64_t seed, uint64_t event, int* n_accepted,
               int* n_proposed, void* stream)
{
    NvtxRange nvtx_("pamd_event");
    if (any_misaligned({pos, pos_out, traj})) return PAMD_ERR_ARG;
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !pos_out || !traj || pos == pos_out || !n_accepted || !n_proposed || n_sample < 1 ||
        n_shift < 1 || l_min < 1 || l_max < l_min || l_max > 30)
        return PAMD_ERR_ARG;
    int Tmax = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        if (s.pot.kind != PAMD_HARMONIC) return PAMD_ERR_UNSUPPORTED;
        if ((1LL << l_max) > s.n_steps || n_shift > s.n_steps) return PAMD_ERR_ARG;
        Tmax = std::max(Tmax, s.n_steps);
    }
    for (const void* ptr : {(const void*)pos, (const void*)pos_out, (const void*)traj,
                            (const void*)n_accepted, (const void*)n_proposed})
        if (is_host_ptr(ptr)) return PAMD_ERR_ARG;
    const int fstride = (Tmax >> l_min) + 2;
    cudaStream_t st = (cudaStream_t)stream;
    const double sig = std::sqrt(2.0 * prob->D * prob->dt), c0 = 1.0 / (4.0 * prob->D * prob->dt);
    const bool fp64 = prob->precision == PAMD_FP64;
    long long traj_off = 0;
    int chain0 = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        const int M = s.dim * s.n_particles, T = s.n_steps;
        const bool fuse = fp64 ? fragment_event_fusable<double>(T, M, l_min, n_shift)
                               : fragment_event_fusable<float>(T, M, l_min, n_shift);
        double g, cS;
        ho_step_constants(prob, s.pot.k, &g, &cS);
        for (int u = 0; u < n_sample; ++u) {
            const uint64_t ctr = event * (uint64_t)n_sample + (uint64_t)u;
            const bool last = fuse && u == n_sample - 1;
            if (fp64)
                PAMD_CUDA_TRY(launch_fragment_mc<double>(
                    (double*)pos, s.pos_offset, T, M, s.n_chains, chain0, l_min, l_max, seed, ctr,
                    nullptr, nullptr, nullptr, nullptr, fstride, g, sig, cS, c0, n_accepted,
                    n_proposed, st, last ? (double*)pos_out : nullptr,
                    last ? (double*)traj + traj_off : nullptr, n_shift, event, regen_sigma(prob)));
            else
                PAMD_CUDA_TRY(launch_fragment_mc<float>(
                    (float*)pos, s.pos_offset, T, M, s.n_chains, chain0, l_min, l_max, seed, ctr,
                    nullptr, nullptr, nullptr, nullptr, fstride, g, sig, cS, c0, n_accepted,
                    n_proposed, st, last ? (float*)pos_out : nullptr,
                    last ? (float*)traj + traj_off : nullptr, n_shift, event, regen_sigma(prob)));
        }
        if (!fuse) {
            if (fp64)
                PAMD_CUDA_TRY(launch_shift_regenerate<double>(
                    (const double*)pos, (double*)pos_out, (double*)traj, s.pos_offset, traj_off, T, M,
                    n_shift, s.n_chains, chain0, regen_sigma(prob), seed, event, nullptr, st));
            else
                PAMD_CUDA_TRY(launch_shift_regenerate<float>(
                    (const float*)pos, (float*)pos_out, (float*)traj, s.pos_offset, traj_off, T, M,
                    n_shift, s.n_chains, chain0, regen_sigma(prob), seed, event, nullptr, st));
        }
        traj_off += (long long)s.n_chains * n_shift * M;
        chain0 += s.n_chains;
    }
    return PAMD_OK;
}

int pamd_shift_regenerate(const pamd_problem* prob, const void* pos, void* pos_out, int n_shift,
                          void* traj, uint64_t seed, uint64_t counter, const void* noise,
                          void* stream)
{
    NvtxRange nvtx_("pamd_shift_regenerate");
    if (any_misaligned({pos, pos_out, traj, noise})) return PAMD_ERR_ARG;
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !pos_out || !traj || pos == pos_out || n_shift < 1) return PAMD_ERR_ARG;
    for (int q = 0; q < prob->n_systems; ++q)
        if (n_shift > prob->systems[q].n_steps) return PAMD_ERR_ARG;
    for (const void* ptr : {pos, (const void*)pos_out, (const void*)traj, noise})
        if (ptr && is_host_ptr(ptr)) return PAMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const double sig = regen_sigma(prob);
    long long traj_off = 0;
    int chain0 = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        const int M = s.dim * s.n_particles;
        if (prob->precision == PAMD_FP64)
            PAMD_CUDA_TRY(launch_shift_regenerate<double>(
                (const double*)pos, (double*)pos_out, (double*)traj, s.pos_offset, traj_off, s.n_steps, M,
                n_shift, s.n_chains, chain0, sig, seed, counter, (const double*)noise, st));
        else
            PAMD_CUDA_TRY(launch_shift_regenerate<float>(
                (const float*)pos, (float*)pos_out, (float*)traj, s.pos_offset, traj_off, s.n_steps, M,
                n_shift, s.n_chains, chain0, sig, seed, counter, (const float*)noise, st));
        traj_off += (long long)s.n_chains * n_shift * M;
        chain0 += s.n_chains;
    }
    return PAMD_OK;
}

int pamd_lj_pair_counts(const pamd_problem* prob, const void* pos, long long* counts, void* stream)
{
    NvtxRange nvtx_("pamd_lj_pair_counts");
    if (any_misaligned({pos})) return PAMD_ERR_ARG;
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_whole_paths(prob))) return rc;
    if (!pos || !counts || prob->precision != PAMD_FP32) return PAMD_ERR_ARG;
    if (is_host_ptr(pos) || is_host_ptr(counts)) return PAMD_ERR_ARG;
    for (int q = 0; q < prob->n_systems; ++q)  // one grid row per chain
        if (prob->systems[q].pot.kind == PAMD_LJ && prob->systems[q].n_chains > 65535)
            return PAMD_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    long long out_off = 0;
    for (int q = 0; q < prob->n_systems; ++q) {
        const pamd_system& s = prob->systems[q];
        if (s.pot.kind != PAMD_LJ) continue;
        PAMD_CUDA_TRY(launch_lj_pair_counts((const float*)pos, counts + out_off, s.n_particles,
                                            s.n_steps, s.n_chains, s.pos_offset, s.pot.box, s.pot.rc,
                                            st));
        out_off += (long long)s.n_chains * (s.n_steps + 1);
    }
    return PAMD_OK;
}

int pamd_philox(uint32_t ctr0, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, uint32_t key0,
                uint32_t key1, long long n, uint32_t* out, void* stream)
{
    if (n < 0 || !out) return PAMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (is_host_ptr(out)) {
        uint32_t* d = nullptr;
        if (cudaMalloc(&d, sizeof(uint32_t) * 4 * (size_t)std::max(n, 1LL)) != cudaSuccess)
            return PAMD_ERR_ALLOC;
        int rc = launch_philox(make_uint4(ctr0, ctr1, ctr2, ctr3), make_uint2(key0, key1), n, d, st) ==
                         cudaSuccess
                     ? PAMD_OK
                     : PAMD_ERR_CUDA;
        if (!rc && cudaMemcpyAsync(out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = PAMD_ERR_CUDA;
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = PAMD_ERR_CUDA;
        cudaFree(d);
        return rc;
    }
    PAMD_CUDA_TRY(launch_philox(make_uint4(ctr0, ctr1, ctr2, ctr3), make_uint2(key0, key1), n, out, st));
    return PAMD_OK;
}

int pamd_normals(uint64_t seed, uint64_t counter, uint32_t stream_id, uint32_t chain, long long e0,
                 long long n, float* out, void* stream)
{
    if (n < 0 || e0 < 0 || !out) return PAMD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (is_host_ptr(out)) {
        float* d = nullptr;
        if (cudaMalloc(&d, sizeof(float) * (size_t)std::max(n, 1LL)) != cudaSuccess) return PAMD_ERR_ALLOC;
        int rc = launch_normals(seed, counter, stream_id, chain, e0, n, d, st) == cudaSuccess ? PAMD_OK
                                                                                               : PAMD_ERR_CUDA;
        if (!rc && cudaMemcpyAsync(out, d, sizeof(float) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = PAMD_ERR_CUDA;
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = PAMD_ERR_CUDA;
        cudaFree(d);
        return rc;
    }
    PAMD_CUDA_TRY(launch_normals(seed, counter, stream_id, chain, e0, n, out, st));
    return PAMD_OK;
}

}  // extern "C"
