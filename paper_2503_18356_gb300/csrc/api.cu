// Host side of the C ABI declared in include/grins_racipe.h: handle
// lifetime, argument validation, the incoming-edge CSR, the half-functional
// median table and the kernel launch sequence of each entry point.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <set>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "integrate_grp.cuh"

// An NVTX range over one call of the C ABI, named after it (a timeline
// marker for Nsight tools; a null-pointer check when no tool is attached).
struct AbiRange {
    explicit AbiRange(const char *name) { nvtxRangePushA(name); }
    ~AbiRange() { nvtxRangePop(); }
    AbiRange(const AbiRange &) = delete;
    AbiRange &operator=(const AbiRange &) = delete;
};

using namespace grins;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

static grins_status fail(grins_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

static grins_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? GRINS_E_NOMEM : GRINS_E_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, what);    \
    } while (0)

// ------------------------------------------------------- device allocations
// Every device allocation the library makes goes through these three
// helpers, which count the calls (grins_device_allocations reports the
// count), so a caller can check that an entry point allocated nothing.
static std::atomic<long long> g_device_allocations{0};

template <typename T>
static cudaError_t dev_malloc(T **p, size_t bytes)
{
    g_device_allocations.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

template <typename T>
static cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    g_device_allocations.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, st);
}

template <typename T>
static cudaError_t dev_malloc_pool(T **p, size_t bytes, cudaMemPool_t pool, cudaStream_t st)
{
    g_device_allocations.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, pool, st);
}

extern "C" int64_t grins_device_allocations(void)
{
    return g_device_allocations.load(std::memory_order_relaxed);
}

// ------------------------------------------------------------------ handle
// A lane-group layout on the device (host copy of the row table).
struct GrpDev {
    int L = 0, R = 0, P = 0;
    std::vector<int32_t> row_off, row_deg, link_to;
    // device arrays: parts of the handle's workspace block (grins_racipe::d_block)
    int32_t *d_pos_edge = nullptr, *d_pos_off = nullptr, *d_row_node = nullptr, *d_row_link = nullptr;
    void free_device() { d_pos_edge = d_pos_off = d_row_node = d_row_link = nullptr; }
    GrpTopo topo() const
    {
        GrpTopo g{};
        g.L = L; g.R = R; g.P = P;
        g.pos_edge = d_pos_edge; g.pos_off = d_pos_off; g.row_node = d_row_node; g.row_link = d_row_link;
        for (int r = 0; r < R && r < kGrpMaxRows; ++r) {
            g.row_off[r] = row_off[r];
            g.row_deg[r] = row_deg[r];
            g.link_to[r] = r < (int)link_to.size() ? link_to[r] : -1;
        }
        return g;
    }
};

struct grins_racipe {
    int N = 0, E = 0, device = 0, num_sms = 1;
    size_t smem_optin = 0;
    std::vector<int32_t> src, dst;
    std::vector<int8_t> sign;
    std::vector<int32_t> csr_off, csr_src, csr_edge;
    std::vector<int8_t> csr_sign;
    std::vector<int32_t> n_act_in, n_inh_in;          // in-degree class per node
    ParamLayout layout{};
    // device workspace: the topology, the layouts' tables, the median and
    // counter arrays are parts of one allocation (d_block), filled by one copy
    unsigned char *d_block = nullptr;
    int32_t *d_off = nullptr, *d_src = nullptr, *d_edge = nullptr;
    int8_t *d_sign = nullptr, *d_edge_sign = nullptr;
    double *d_edge_median = nullptr;
    unsigned long long *d_queue = nullptr;
    double *d_grid = nullptr;
    // lane-group layouts of the FP32 integrator (see GrpTopo): for the
    // shared-record kernels (run-time layout, batched plans) and for the
    // register-record kernel compiled at run time
    GrpDev grp, rr;
    std::string jit_why = "not compiled yet";          // why no run-time compiled kernel is used
    bool jit_used = false;
    std::string jit_why64;                             // the same for the last FP64 launch
    bool jit_used64 = false, ran64 = false;
    int used_L = 0, used_R = 0, used_P = 0;            // layout of the last FP32 launch
    int used_method = 0;                               // and its 5(4) pair
    std::string info;                                  // grins_racipe_integrator text
    int grid_cap = 0;
    // borderline re-pass workspace: two counters (items listed, FP64
    // attempts) then the item list, room for tail_cap solves
    unsigned char *d_tail = nullptr;
    int64_t tail_cap = 0;
    // a second stream for the polish that runs beside the re-pass, with the
    // events that fork it from and join it to the caller's stream (created
    // on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool tail_ran = false;                             // the last FP32 integrate ran the re-pass
    std::string tail_why = "off";                      // what the last FP32 integrate did about it
    // cached median table
    bool median_valid = false;
    grins_racipe_ranges median_ranges{};
    std::vector<grins_param_range> median_table;   // per-parameter rows the medians were taken with
    std::vector<double> node_median;
    // d_edge_median is written once, by the first sampling call, and then
    // only read: calls whose medians differ stage their own copy on their
    // stream, so no queued sampler ever sees it change
    bool edge_median_set = false;
    std::vector<double> edge_median_host;          // what d_edge_median holds
    std::mutex median_mu;                          // the median cache and the fields above
};

extern "C" void grins_racipe_default_ranges(grins_racipe_ranges *r)
{
    if (!r) return;
    r->G_min = 1.0; r->G_max = 100.0;
    r->k_min = 0.1; r->k_max = 1.0;
    r->lam_act_min = 1.0; r->lam_act_max = 100.0;
    r->lam_inh_min = 0.01; r->lam_inh_max = 1.0;
    r->n_min = 1; r->n_max = 6;
    r->thr_lo = 0.02; r->thr_hi = 1.98;
    r->median_samples = 10000;
    r->median_mode = GRINS_MEDIAN_PER_INDEGREE;
    r->dist_G = r->dist_k = r->dist_lam_act = r->dist_lam_inh = GRINS_DIST_TABLE1;
    r->lhs_sets = 0;
    r->sobol = GRINS_SOBOL_OFF;
    r->sobol_dims = 0;
    r->sobol_poly = nullptr;
    r->sobol_m = nullptr;
    r->sobol_m_cols = 0;
    r->reserved = 0;
    r->param_ranges = nullptr;
    r->ic_ranges = nullptr;
}

extern "C" void grins_solver_default_opts(grins_solver_opts *o)
{
    if (!o) return;
    o->precision = GRINS_FP32;
    o->polish = 1;
    o->rtol = 1e-6; o->atol = 1e-9;
    o->t0 = 0.0; o->t_end = 200.0;
    o->ss_tol = 1e-6;
    o->max_steps = 100000;
    o->t_grid = nullptr; o->n_t = 0;
    o->polish_tol = 1e-13;
    o->polish_iters = 16;
    o->polish_max_move = 0.1;
    o->ss_tighten = 0.3;
    o->method = GRINS_METHOD_DOPRI5;
    o->tail_rtol = 1e-9;
    o->tail_start = 20.0;
    o->tail_rho = 10.0;
    o->tail_late = 0.2;
    o->tail_work = 96;
    o->tail_precision = GRINS_TAIL_DD;
    o->pass_event = nullptr;
}

extern "C" const char *grins_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *grins_version(void) { return "grins_racipe 0.1 (sm_103a)"; }

static void free_device(grins_racipe *h)
{
    cudaFree(h->d_block); cudaFree(h->d_grid); cudaFree(h->d_tail);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
    h->d_block = nullptr;
    h->d_tail = nullptr;
    h->tail_cap = 0;
    h->grp.free_device();
    h->rr.free_device();
    h->d_off = h->d_src = h->d_edge = nullptr;
    h->d_sign = h->d_edge_sign = nullptr;
    h->d_edge_median = h->d_grid = nullptr;
    h->d_queue = nullptr;
}

// Lane-group layout (GrpTopo) with L lanes per solve: nodes sorted by
// in-degree (descending, ties by index) fill rows of L; row r takes D_r = its
// largest in-degree positions.  Within a row the host orders each lane's
// in-edges so that, position by position, the L lanes read sources in
// distinct gather columns (distinct shared-memory banks) where it can,
// filling the gaps with neutral edges.
struct GrpHost {
    int L = 0, R = 0, P = 0;
    std::vector<int32_t> row_off, row_deg, pos_edge, pos_off, row_node;
    std::vector<int32_t> row_link;      // [R * L]: 1 where slot (r, j) continues slot (link_to[r], j)
    std::vector<int32_t> link_to;       // [R]: the row a row's continuations multiply into, or -1
};

static GrpHost build_grp(int N, int L, const std::vector<int32_t> &csr_off, const std::vector<int32_t> &csr_src,
                         const std::vector<int32_t> &csr_edge, bool split = false)
{
    GrpHost g;
    const int R = (N + L - 1) / L;
    if (R > kGrpMaxRows) return g;
    const int GS = kWarp / L;
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return csr_off[a + 1] - csr_off[a] > csr_off[b + 1] - csr_off[b];
    });
    g.L = L; g.R = R;
    g.row_node.assign((size_t)R * L, -1);
    g.row_link.assign((size_t)R * L, 0);
    g.link_to.assign(R, -1);
    std::vector<int> gslot(N, 0);
    for (int q = 0; q < N; ++q) { g.row_node[q] = order[q]; gslot[order[q]] = q; }
    // in-edges (CSR positions) handled by each slot
    std::vector<std::vector<int>> slot_lst((size_t)R * L);
    for (int q = 0; q < N; ++q)
        for (int c = csr_off[order[q]]; c < csr_off[order[q] + 1]; ++c) slot_lst[q].push_back(c);
    // Splitting (register-record layouts): row 0 may be cut to a width t
    // below its widest node when every node wider than t can hand its edges
    // beyond t to a free slot of the last row in its own lane (a
    // continuation: the lane multiplies that partial product into the
    // node's own).  t minimises t + the last row's width, and those nodes
    // move to the free slots' lanes.
    if (split && R >= 2) {
        std::vector<int> spare;
        for (int j = 0; j < L; ++j)
            if (g.row_node[(R - 1) * L + j] < 0) spare.push_back(j);
        std::vector<int> d0(L);
        int D0 = 0, Dl = 0;
        for (int j = 0; j < L; ++j) { d0[j] = (int)slot_lst[j].size(); D0 = std::max(D0, d0[j]); }
        for (int j = 0; j < L; ++j) Dl = std::max(Dl, (int)slot_lst[(R - 1) * L + j].size());
        int best_t = D0, best_cost = D0 + Dl;
        for (int t = D0 - 1; t >= 1; --t) {
            int over = 0;
            for (int j = 0; j < L; ++j) over += d0[j] > t;
            if (over > (int)spare.size()) break;
            const int cost = t + std::max(Dl, D0 - t);
            if (cost < best_cost) { best_cost = cost; best_t = t; }
        }
        if (best_t < D0) {
            // new row 0: the wide nodes in the free slots' lanes, the others
            // in the remaining lanes in their order
            std::vector<int> wide, rest;
            for (int j = 0; j < L; ++j) (d0[j] > best_t ? wide : rest).push_back(j);
            std::vector<int> lane_of(L, -1);      // old row-0 lane -> new lane
            std::vector<char> taken(L, 0);
            for (size_t k = 0; k < wide.size(); ++k) { lane_of[wide[k]] = spare[k]; taken[spare[k]] = 1; }
            int nxt = 0;
            for (int j : rest) {
                while (taken[nxt]) ++nxt;
                lane_of[j] = nxt;
                taken[nxt] = 1;
            }
            std::vector<int32_t> node0(L);
            std::vector<std::vector<int>> lst0(L);
            for (int j = 0; j < L; ++j) { node0[lane_of[j]] = g.row_node[j]; lst0[lane_of[j]] = slot_lst[j]; }
            for (int j = 0; j < L; ++j) {
                g.row_node[j] = node0[j];
                slot_lst[j] = lst0[j];
                if (node0[j] >= 0) gslot[node0[j]] = j;
            }
            for (size_t k = 0; k < wide.size(); ++k) {
                const int js = spare[k], cont = (R - 1) * L + js;
                slot_lst[cont].assign(slot_lst[js].begin() + best_t, slot_lst[js].end());
                slot_lst[js].resize(best_t);
                g.row_link[cont] = 1;
            }
            g.link_to[R - 1] = 0;
        }
    }
    auto col_of = [&](int node) { return gslot[node] % L; };
    auto off_of_slot = [&](int slot) { return slot * GS * 4; };
    // Order of one row's edges: position by position, each lane (in lane
    // order) takes its first unplaced edge whose source column no other
    // source at this position uses (or whose source another lane already
    // reads), else -- when it has no neutral slot left -- its first unplaced
    // edge; a lane with nothing to place reads a neutral edge at the address
    // of the position's first real source (a broadcast, no extra wavefront).
    // Returns the position count weighted by wavefronts (the largest number
    // of distinct sources sharing a column at each position).
    int trials = 64;
    if (const char *ev = std::getenv("GRINS_GRP_ORDER_TRIALS")) trials = std::max(1, std::atoi(ev));
    auto order_row = [&](const std::vector<std::vector<int>> &lst0, int D, uint64_t seed,
                         std::vector<int32_t> &E, std::vector<int32_t> &O) -> int {
        uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        auto next = [&]() {      // splitmix64
            uint64_t z = (st += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        std::vector<std::vector<int>> lst = lst0;
        std::vector<int> lanes(L);
        for (int j = 0; j < L; ++j) lanes[j] = j;
        if (seed) {
            for (int i = L - 1; i > 0; --i) std::swap(lanes[i], lanes[next() % (uint64_t)(i + 1)]);
            for (auto &v : lst)
                for (int i = (int)v.size() - 1; i > 0; --i) std::swap(v[i], v[next() % (uint64_t)(i + 1)]);
        }
        std::vector<std::vector<char>> used(L);
        std::vector<int> left(L);
        for (int j = 0; j < L; ++j) { used[j].assign(lst[j].size(), 0); left[j] = (int)lst[j].size(); }
        E.assign((size_t)D * L, -1);
        O.assign((size_t)D * L, 0);
        int score = 0;
        for (int m = 0; m < D; ++m) {
            std::vector<int> col_cnt(L, 0);
            std::vector<int> src_here;
            std::vector<int> neutral;
            for (int jj = 0; jj < L; ++jj) {
                const int j = lanes[jj];
                const int spare = (D - m) - left[j];       // neutral slots still to place
                int pick = -1;
                for (size_t q = 0; q < lst[j].size() && pick < 0; ++q) {
                    if (used[j][q]) continue;
                    const int sn = csr_src[lst[j][q]];
                    bool same = false;
                    for (int x : src_here) same = same || x == sn;
                    if (same || col_cnt[col_of(sn)] == 0) pick = (int)q;
                }
                if (pick < 0 && spare == 0) {
                    for (size_t q = 0; q < lst[j].size() && pick < 0; ++q)
                        if (!used[j][q]) pick = (int)q;
                }
                if (pick < 0) { neutral.push_back(j); continue; }
                used[j][pick] = 1;
                --left[j];
                const int c = lst[j][pick], sn = csr_src[c];
                bool seen = false;
                for (int x : src_here) seen = seen || x == sn;
                if (!seen) { src_here.push_back(sn); col_cnt[col_of(sn)]++; }
                E[(size_t)m * L + j] = csr_edge[c];
                O[(size_t)m * L + j] = off_of_slot(gslot[sn]);
            }
            const int nof = src_here.empty() ? 0 : off_of_slot(gslot[src_here[0]]);
            for (int j : neutral) { E[(size_t)m * L + j] = -1; O[(size_t)m * L + j] = nof; }
            score += std::max(1, *std::max_element(col_cnt.begin(), col_cnt.end()));
        }
        return score;
    };
    int P = 0;
    for (int r = 0; r < R; ++r) {
        int D = 0;
        std::vector<std::vector<int>> lst(L);            // CSR positions per lane
        for (int j = 0; j < L; ++j) {
            lst[j] = slot_lst[(size_t)r * L + j];
            D = std::max(D, (int)lst[j].size());
        }
        g.row_off.push_back(P);
        g.row_deg.push_back(D);
        // trial 0 is the plain greedy order; later trials shuffle the lane
        // order and each lane's candidate order; the order with the fewest
        // shared-memory wavefronts wins
        std::vector<int32_t> best_e, best_o, e, o;
        int best = -1;
        for (int trial = 0; trial < trials && best != D; ++trial) {   // D: one wavefront per position
            const int sc = order_row(lst, D, (uint64_t)trial, e, o);
            if (best < 0 || sc < best) { best = sc; best_e.swap(e); best_o.swap(o); }
        }
        g.pos_edge.insert(g.pos_edge.end(), best_e.begin(), best_e.end());
        g.pos_off.insert(g.pos_off.end(), best_o.begin(), best_o.end());
        P += D;
    }
    g.P = P;
    return g;
}

// GRINS_GRP_L (1, 2, 4, 8, 16 or 32): lanes per solve for both layouts when
// it gives at most 12 rows (a tuning override); 0 when unset.
static int grp_l_override(int N)
{
    if (const char *ev = std::getenv("GRINS_GRP_L")) {
        const int f = std::atoi(ev);
        if ((f == 1 || f == 2 || f == 4 || f == 8 || f == 16 || f == 32) && (N + f - 1) / f <= 12) return f;
    }
    return 0;
}

// Shared-record kernels: the smallest power of two L with at most 8 node
// rows (their register arrays stay small enough for 12 warps per SM).
static GrpHost choose_grp_shared(int N, const std::vector<int32_t> &off, const std::vector<int32_t> &src,
                                 const std::vector<int32_t> &edge)
{
    int L = 1;
    while ((N + L - 1) / L > 8 && L < kWarp) L *= 2;
    if (const int f = grp_l_override(N)) L = f;
    if ((N + L - 1) / L > kGrpMaxRows) return GrpHost{};
    return build_grp(N, L, off, src, edge);
}

// Positions per lane of the layout with L lanes: nodes sorted by
// in-degree, each row of L taking its largest in-degree (no edge ordering
// needed for the count).
static int grp_positions(int N, int L, const std::vector<int32_t> &off)
{
    std::vector<int> deg(N);
    for (int i = 0; i < N; ++i) deg[i] = off[i + 1] - off[i];
    std::sort(deg.begin(), deg.end(), [](int a, int b) { return a > b; });
    int P = 0;
    for (int q = 0; q < N; q += L) P += deg[q];
    return P;
}

// Register-record kernel: a lane holds about 4 registers per edge position
// and 11 per row on top of ~40.  The smallest power of two L (at most 12
// rows) whose estimate allows 3 resident blocks of 4 warps per SM (168
// registers), else 2 (255); none when no L fits.
static GrpHost choose_grp_registers(int N, const std::vector<int32_t> &off, const std::vector<int32_t> &src,
                                    const std::vector<int32_t> &edge)
{
    auto est = [&](int L) { return 4 * grp_positions(N, L, off) + 11 * ((N + L - 1) / L) + 40; };
    if (const int f = grp_l_override(N)) return est(f) <= 255 ? build_grp(N, f, off, src, edge, true) : GrpHost{};
    for (int limit : {168, 255}) {
        for (int L = 1; L <= kWarp; L *= 2) {
            if ((N + L - 1) / L > 12) continue;
            if (est(L) <= limit) return build_grp(N, L, off, src, edge, true);
        }
    }
    return GrpHost{};
}

// Host staging of the handle's device block: parts placed at 256-byte
// aligned offsets, copied to the device in one transfer.
struct BlockStage {
    std::vector<unsigned char> host;
    // reserves `bytes` (zero-filled) and copies `src` (may be null) into it
    size_t add(const void *src, size_t bytes)
    {
        const size_t o = host.size();
        host.resize((o + std::max<size_t>(bytes, 1) + 255) & ~(size_t)255, 0);
        if (src && bytes) std::memcpy(host.data() + o, src, bytes);
        return o;
    }
};

// Layout g's tables into the staging block; d keeps the host row table and
// the offsets, turned into device pointers by place_grp.
struct GrpOffsets { size_t pos_edge = 0, pos_off = 0, row_node = 0, row_link = 0; };

static GrpOffsets stage_grp(const GrpHost &g, GrpDev &d, BlockStage &b)
{
    d.L = g.L; d.R = g.R; d.P = g.P;
    d.row_off = g.row_off; d.row_deg = g.row_deg; d.link_to = g.link_to;
    GrpOffsets o;
    if (g.L <= 0) return o;
    const size_t np = std::max<size_t>(g.pos_edge.size(), 1), nr = g.row_node.size();
    o.pos_edge = b.add(g.pos_edge.empty() ? nullptr : g.pos_edge.data(), sizeof(int32_t) * np);
    o.pos_off = b.add(g.pos_off.empty() ? nullptr : g.pos_off.data(), sizeof(int32_t) * np);
    o.row_node = b.add(g.row_node.data(), sizeof(int32_t) * nr);
    o.row_link = b.add(g.row_link.data(), sizeof(int32_t) * nr);
    return o;
}

static void place_grp(GrpDev &d, const GrpOffsets &o, unsigned char *block)
{
    if (d.L <= 0) return;
    d.d_pos_edge = reinterpret_cast<int32_t *>(block + o.pos_edge);
    d.d_pos_off = reinterpret_cast<int32_t *>(block + o.pos_off);
    d.d_row_node = reinterpret_cast<int32_t *>(block + o.row_node);
    d.d_row_link = reinterpret_cast<int32_t *>(block + o.row_link);
}

extern "C" grins_status grins_racipe_create(int32_t n_nodes, int32_t n_edges, const int32_t *src,
                                            const int32_t *dst, const int8_t *sign,
                                            grins_racipe_t *out)
{
    AbiRange nvtx_range_("grins_racipe_create");
    g_last_error.clear();
    if (!out) return fail(GRINS_E_INVALID_ARG, "create: out is NULL");
    *out = nullptr;
    if (n_nodes < 1 || n_nodes > kMaxNodes)
        return fail(GRINS_E_TOPOLOGY, "create: n_nodes = %d outside [1, %d]", n_nodes, kMaxNodes);
    if (n_edges < 0 || n_edges > kMaxEdges)
        return fail(GRINS_E_TOPOLOGY, "create: n_edges = %d outside [0, %d]", n_edges, kMaxEdges);
    if (n_edges > 0 && (!src || !dst || !sign)) return fail(GRINS_E_INVALID_ARG, "create: NULL edge array");
    std::vector<char> seen((size_t)n_nodes * n_nodes, 0);
    for (int e = 0; e < n_edges; ++e) {
        if (src[e] < 0 || src[e] >= n_nodes || dst[e] < 0 || dst[e] >= n_nodes)
            return fail(GRINS_E_TOPOLOGY, "create: edge %d (%d -> %d) has a node index outside [0, %d)", e,
                        src[e], dst[e], n_nodes);
        if (sign[e] != 1 && sign[e] != -1)
            return fail(GRINS_E_TOPOLOGY, "create: edge %d has sign %d (must be +1 or -1)", e, (int)sign[e]);
        char &s = seen[(size_t)src[e] * n_nodes + dst[e]];
        if (s) return fail(GRINS_E_TOPOLOGY, "create: edge %d repeats the pair (%d -> %d)", e, src[e], dst[e]);
        s = 1;
    }
    grins_racipe *h = new (std::nothrow) grins_racipe();
    if (!h) return fail(GRINS_E_NOMEM, "create: host allocation failed");
    h->N = n_nodes; h->E = n_edges;
    h->src.assign(src, src + n_edges);
    h->dst.assign(dst, dst + n_edges);
    h->sign.assign(sign, sign + n_edges);
    // CSR of incoming edges, stable in creation order within a target
    h->csr_off.assign(n_nodes + 1, 0);
    h->n_act_in.assign(n_nodes, 0);
    h->n_inh_in.assign(n_nodes, 0);
    for (int e = 0; e < n_edges; ++e) {
        h->csr_off[dst[e] + 1]++;
        if (sign[e] > 0) h->n_act_in[dst[e]]++; else h->n_inh_in[dst[e]]++;
    }
    for (int i = 0; i < n_nodes; ++i) h->csr_off[i + 1] += h->csr_off[i];
    h->csr_src.resize(n_edges); h->csr_edge.resize(n_edges); h->csr_sign.resize(n_edges);
    std::vector<int> fillp(h->csr_off.begin(), h->csr_off.end() - 1);
    for (int e = 0; e < n_edges; ++e) {
        const int p = fillp[dst[e]]++;
        h->csr_src[p] = src[e]; h->csr_edge[p] = e; h->csr_sign[p] = sign[e];
    }
    h->layout = make_layout(n_nodes, n_edges);
    const GrpHost grp = choose_grp_shared(n_nodes, h->csr_off, h->csr_src, h->csr_edge);
    const GrpHost grr = choose_grp_registers(n_nodes, h->csr_off, h->csr_src, h->csr_edge);

    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    int optin = 0;
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->smem_optin = (size_t)optin;
    // one device allocation and one copy for the whole workspace (each CUDA
    // call can stall behind other threads' driver work -- module loads of
    // run-time compiled kernels -- so creation makes as few as it can)
    const size_t Eb = (size_t)std::max(n_edges, 1);
    BlockStage bs;
    const size_t o_off = bs.add(h->csr_off.data(), sizeof(int32_t) * (n_nodes + 1));
    const size_t o_src = bs.add(n_edges ? h->csr_src.data() : nullptr, sizeof(int32_t) * Eb);
    const size_t o_edge = bs.add(n_edges ? h->csr_edge.data() : nullptr, sizeof(int32_t) * Eb);
    const size_t o_sign = bs.add(n_edges ? h->csr_sign.data() : nullptr, Eb);
    const size_t o_esign = bs.add(n_edges ? h->sign.data() : nullptr, Eb);
    const size_t o_median = bs.add(nullptr, sizeof(double) * Eb);
    // d_queue: [0, 1] the integrator's work counters, [2, 3] check words,
    // [4, 5] the unit counters of the two polish launches beside the re-pass
    const size_t o_queue = bs.add(nullptr, sizeof(unsigned long long) * 8);
    const GrpOffsets og = stage_grp(grp, h->grp, bs);
    const GrpOffsets orr = stage_grp(grr, h->rr, bs);
    if (ce == cudaSuccess) ce = dev_malloc(&h->d_block, bs.host.size());
    if (ce == cudaSuccess) ce = cudaMemcpy(h->d_block, bs.host.data(), bs.host.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        unsigned char *b = h->d_block;
        h->d_off = reinterpret_cast<int32_t *>(b + o_off);
        h->d_src = reinterpret_cast<int32_t *>(b + o_src);
        h->d_edge = reinterpret_cast<int32_t *>(b + o_edge);
        h->d_sign = reinterpret_cast<int8_t *>(b + o_sign);
        h->d_edge_sign = reinterpret_cast<int8_t *>(b + o_esign);
        h->d_edge_median = reinterpret_cast<double *>(b + o_median);
        h->d_queue = reinterpret_cast<unsigned long long *>(b + o_queue);
        place_grp(h->grp, og, b);
        place_grp(h->rr, orr, b);
    }
    if (ce != cudaSuccess) {
        free_device(h);
        delete h;
        return cuda_fail(ce, "create: device workspace");
    }
    *out = h;
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_destroy(grins_racipe_t h)
{
    if (!h) return fail(GRINS_E_INVALID_ARG, "destroy: NULL handle");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_device(h);
    if (cur != h->device) cudaSetDevice(cur);
    delete h;
    return GRINS_OK;
}

extern "C" const char *grins_racipe_integrator(grins_racipe_t h)
{
    if (!h) return "";
    char buf[160];
    const bool ran = h->used_L > 0;
    const int L = ran ? h->used_L : h->grp.L, R = ran ? h->used_R : h->grp.R, P = ran ? h->used_P : h->grp.P;
    if (L > 0)
        std::snprintf(buf, sizeof(buf), "lane-group %s, L=%d lanes per solve, R=%d node rows, P=%d edge positions",
                      h->used_method == GRINS_METHOD_TSIT5 ? "Tsit5(4)" : "DP5(4)", L, R, P);
    else
        std::snprintf(buf, sizeof(buf), "generic shared-memory DP5(4) (no lane-group layout)");
    h->info = buf;
    if (L > 0) h->info += h->jit_used ? "; compiled for this network at run time (" + h->jit_why + ")"
                              : "; run-time layout (" + h->jit_why + ")";
    if (h->ran64)
        h->info += h->jit_used64 ? "; FP64 solver compiled for this network at run time (" + h->jit_why64 + ")"
                                 : "; FP64 solver generic (" + h->jit_why64 + ")";
    if (ran) h->info += "; borderline re-pass: " + h->tail_why;
    return h->info.c_str();
}

extern "C" int64_t grins_racipe_param_stride(grins_racipe_t h)
{
    return h ? h->layout.stride : -1;
}

// ----------------------------------------------------- half-functional rule
// Host Philox4x64-10 (Salmon et al., SC'11), identical in definition to the
// device generator of common.cuh.
static void philox_host(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
        const unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
        const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c[1] ^ k0;
        const uint64_t n2 = (uint64_t)(p0 >> 64) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (uint64_t)p1; c[2] = n2; c[3] = (uint64_t)p0;
        k0 += W0; k1 += W1;
    }
}

namespace {

struct MedianStream {
    uint64_t key1;
    uint64_t draw(uint64_t sample, uint64_t d) const
    {
        uint64_t c[4] = {sample, d / 4, 0, 0};
        philox_host(c, kKeyMedian, key1);
        return c[d % 4];
    }
};

inline double span_map(double lo, double hi, double u) { return lo + (hi - lo) * u; }

// A continuous parameter of class distribution `dist` over [lo, hi] from one
// 64-bit draw (GRINS_DIST_*; Table 1's uniform map when dist is 0).
double dist_draw(int dist, double lo, double hi, uint64_t r)
{
    if (dist == GRINS_DIST_LOGUNIFORM) return std::exp(span_map(std::log(lo), std::log(hi), unit_double(r)));
    if (dist == GRINS_DIST_NORMAL || dist == GRINS_DIST_LOGNORMAL) {
        const double uh = ((double)(r >> 32) + 0.5) * 0x1.0p-32, ul = ((double)(r & 0xffffffffu) + 0.5) * 0x1.0p-32;
        const double z = std::sqrt(-2.0 * std::log(uh)) * std::cos(6.283185307179586 * ul);
        if (dist == GRINS_DIST_NORMAL) return std::min(hi, std::max(lo, (lo + hi) / 2.0 + z * ((hi - lo) / 6.0)));
        const double a = std::log(lo), b = std::log(hi);
        return std::min(hi, std::max(lo, std::exp((a + b) / 2.0 + z * ((b - a) / 6.0))));
    }
    return span_map(lo, hi, unit_double(r));
}

// The inhibiting fold change: Table 1's inverse-range rule, or dist_draw.
double lam_inh_draw(const grins_racipe_ranges &r, uint64_t x)
{
    if (r.dist_lam_inh == GRINS_DIST_TABLE1) return 1.0 / span_map(1.0 / r.lam_inh_max, 1.0 / r.lam_inh_min, unit_double(x));
    return dist_draw(r.dist_lam_inh, r.lam_inh_min, r.lam_inh_max, x);
}

// Eq. 2 in its printed form, H = B0^n/(B0^n+B^n) + lambda B^n/(B0^n+B^n),
// times 1/lambda for an activating input (Eq. 1).
inline double hill_factor(bool act, double B, double B0, double n, double lam)
{
    if (B < 0.0) B = 0.0;
    const double b0n = std::pow(B0, n), bn = std::pow(B, n);
    const double h = b0n / (b0n + bn) + lam * bn / (b0n + bn);
    return act ? h / lam : h;
}

double median_sorted(std::vector<double> &v)
{
    std::sort(v.begin(), v.end());
    const size_t K = v.size();
    return K % 2 ? v[K / 2] : (v[K / 2 - 1] + v[K / 2]) / 2.0;
}

// Levels of a node with `na` activating and `ni` inhibiting inputs: the node
// at its own steady state (G/k times its input factors), each input at an
// unregulated level G'/k' with threshold U[thr_lo, thr_hi] * M0 and n, lambda
// from the ranges.  Draw layout of sample s: 0 -> G, 1 -> k, then for input m
// (activating inputs first) draws 2+5m .. 6+5m -> G', k', threshold, lambda, n.
std::vector<double> level_samples(int na, int ni, const grins_racipe_ranges &r, double M0)
{
    const MedianStream ms{((uint64_t)(uint32_t)na << 32) | (uint64_t)(uint32_t)ni};
    const int K = r.median_samples;
    std::vector<double> out((size_t)K);
    for (int s = 0; s < K; ++s) {
        const double G = dist_draw(r.dist_G, r.G_min, r.G_max, ms.draw(s, 0));
        const double k = dist_draw(r.dist_k, r.k_min, r.k_max, ms.draw(s, 1));
        double level = G / k;
        for (int m = 0; m < na + ni; ++m) {
            const uint64_t d = 2 + 5 * (uint64_t)m;
            const double Gs = dist_draw(r.dist_G, r.G_min, r.G_max, ms.draw(s, d));
            const double ks = dist_draw(r.dist_k, r.k_min, r.k_max, ms.draw(s, d + 1));
            const double T = span_map(r.thr_lo, r.thr_hi, unit_double(ms.draw(s, d + 2))) * M0;
            const uint64_t xl = ms.draw(s, d + 3);
            const int n = unit_int(ms.draw(s, d + 4), r.n_min, r.n_max - r.n_min + 1);
            const bool act = m < na;
            const double lam = act ? dist_draw(r.dist_lam_act, r.lam_act_min, r.lam_act_max, xl) : lam_inh_draw(r, xl);
            level = level * hill_factor(act, Gs / ks, T, (double)n, lam);
        }
        out[(size_t)s] = level;
    }
    return out;
}

// Equal in what the medians depend on (the set-stratification fields --
// Latin hypercube, Sobol tables -- do not enter the median samples).
bool same_ranges(const grins_racipe_ranges &a, const grins_racipe_ranges &b)
{
    grins_racipe_ranges x, y;
    std::memcpy(&x, &a, sizeof(x));
    std::memcpy(&y, &b, sizeof(y));
    for (grins_racipe_ranges *r : {&x, &y}) {
        r->lhs_sets = 0;
        r->sobol = 0;
        r->sobol_dims = 0;
        r->sobol_poly = nullptr;
        r->sobol_m = nullptr;
        r->sobol_m_cols = 0;
        r->reserved = 0;
        r->param_ranges = nullptr;        // its rows are compared by the caller
        r->ic_ranges = nullptr;           // initial conditions do not enter the medians
    }
    static_assert(sizeof(grins_racipe_ranges) == 168, "grins_racipe_ranges has no padding bytes");
    return std::memcmp(&x, &y, sizeof(x)) == 0;
}

grins_status check_ranges(const grins_racipe_ranges &r)
{
    auto ok_pair = [](double lo, double hi) { return std::isfinite(lo) && std::isfinite(hi) && lo > 0 && lo <= hi; };
    if (!ok_pair(r.G_min, r.G_max)) return fail(GRINS_E_INVALID_ARG, "ranges: need 0 < G_min <= G_max");
    if (!ok_pair(r.k_min, r.k_max)) return fail(GRINS_E_INVALID_ARG, "ranges: need 0 < k_min <= k_max");
    if (!ok_pair(r.lam_act_min, r.lam_act_max) || r.lam_act_min < 1.0)
        return fail(GRINS_E_INVALID_ARG, "ranges: need 1 <= lam_act_min <= lam_act_max");
    if (!ok_pair(r.lam_inh_min, r.lam_inh_max) || r.lam_inh_max > 1.0)
        return fail(GRINS_E_INVALID_ARG, "ranges: need 0 < lam_inh_min <= lam_inh_max <= 1");
    if (r.n_min < 1 || r.n_max > 255 || r.n_min > r.n_max)
        return fail(GRINS_E_INVALID_ARG, "ranges: need 1 <= n_min <= n_max <= 255");
    if (!ok_pair(r.thr_lo, r.thr_hi)) return fail(GRINS_E_INVALID_ARG, "ranges: need 0 < thr_lo <= thr_hi");
    if (r.median_samples < 1 || r.median_samples > 10000000)
        return fail(GRINS_E_INVALID_ARG, "ranges: median_samples outside [1, 1e7]");
    if (r.median_mode != GRINS_MEDIAN_PER_INDEGREE && r.median_mode != GRINS_MEDIAN_UNREGULATED)
        return fail(GRINS_E_INVALID_ARG, "ranges: unknown median_mode %d", r.median_mode);
    for (int d : {r.dist_G, r.dist_k, r.dist_lam_act, r.dist_lam_inh}) {
        if (d < GRINS_DIST_TABLE1 || d > GRINS_DIST_LOGNORMAL)
            return fail(GRINS_E_INVALID_ARG, "ranges: unknown distribution %d", d);
        if (r.lhs_sets > 0 && d > GRINS_DIST_LOGUNIFORM)
            return fail(GRINS_E_INVALID_ARG, "ranges: the Latin hypercube takes Table 1 and log-uniform draws only");
        if (r.sobol != GRINS_SOBOL_OFF && d > GRINS_DIST_LOGUNIFORM)
            return fail(GRINS_E_INVALID_ARG, "ranges: Sobol sets take Table 1 and log-uniform draws only");
    }
    if (r.lhs_sets < 0) return fail(GRINS_E_INVALID_ARG, "ranges: lhs_sets < 0");
    if (r.sobol < GRINS_SOBOL_OFF || r.sobol > GRINS_SOBOL_SCRAMBLED)
        return fail(GRINS_E_INVALID_ARG, "ranges: unknown sobol mode %d", r.sobol);
    if (r.sobol != GRINS_SOBOL_OFF && r.lhs_sets > 0)
        return fail(GRINS_E_INVALID_ARG, "ranges: Sobol sets and the Latin hypercube exclude each other");
    return GRINS_OK;
}

// Median level of the in-degree class (na activating, ni inhibiting inputs)
// under ranges r.  It depends on the class and the ranges only (the samples
// use a fixed key), so it is computed once per process and shared by every
// network; (0, 0) is the unregulated level, m0 the median the regulated
// classes' sources are drawn around.
// Process-wide cache of class medians, keyed by (na, ni, ranges).
struct ClassMedianCache {
    struct Entry { grins_racipe_ranges r; int na, ni; double m; };
    std::mutex mu;
    std::vector<Entry> tab;
    bool find(int na, int ni, const grins_racipe_ranges &r, double *m)
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : tab)
            if (e.na == na && e.ni == ni && same_ranges(e.r, r)) { *m = e.m; return true; }
        return false;
    }
    void put(int na, int ni, const grins_racipe_ranges &r, double m)
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : tab)
            if (e.na == na && e.ni == ni && same_ranges(e.r, r)) return;
        tab.push_back(Entry{r, na, ni, m});
    }
};

ClassMedianCache &class_cache()
{
    static ClassMedianCache *c = new ClassMedianCache();
    return *c;
}

double class_median(int na, int ni, const grins_racipe_ranges &r, double m0)
{
    double m = 0.0;
    if (class_cache().find(na, ni, r, &m)) return m;
    std::vector<double> v = level_samples(na, ni, r, m0);
    m = median_sorted(v);
    class_cache().put(na, ni, r, m);
    return m;
}

// The in-degree classes (a activating, b inhibiting inputs) of h's regulated
// nodes whose medians under r are not cached yet (the unregulated class
// (0, 0) first when it is missing).
std::vector<std::pair<int, int>> missing_classes(const grins_racipe *h, const grins_racipe_ranges &r)
{
    std::vector<std::pair<int, int>> out;
    double m = 0.0;
    if (!class_cache().find(0, 0, r, &m)) out.push_back({0, 0});
    if (r.median_mode != GRINS_MEDIAN_PER_INDEGREE) return out;
    for (int j = 0; j < h->N; ++j) {
        const std::pair<int, int> c{h->n_act_in[j], h->n_inh_in[j]};
        if (c.first == 0 && c.second == 0) continue;
        if (std::find(out.begin(), out.end(), c) != out.end()) continue;
        if (!class_cache().find(c.first, c.second, r, &m)) out.push_back(c);
    }
    return out;
}

// Computes the missing class medians of h under r, the regulated classes in
// parallel (each class's samples come from its own Philox stream, so the
// result does not depend on the order or the threads).
void warm_class_medians(const grins_racipe *h, const grins_racipe_ranges &r)
{
    std::vector<std::pair<int, int>> miss = missing_classes(h, r);
    if (miss.empty()) return;
    const double M0 = class_median(0, 0, r, 0.0);
    if (miss.front() == std::pair<int, int>{0, 0}) miss.erase(miss.begin());
    if (miss.empty()) return;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t T = std::min<size_t>(miss.size(), std::min<unsigned>(8u, std::max(1u, hw / 2)));
    std::atomic<size_t> next{0};
    auto work = [&]() {
        for (size_t i = next++; i < miss.size(); i = next++) class_median(miss[i].first, miss[i].second, r, M0);
    };
    std::vector<std::thread> team;
    for (size_t t = 1; t < T; ++t) team.emplace_back(work);
    work();
    for (auto &t : team) t.join();
}

// Rows of a per-parameter table: the constraints stated with
// grins_param_range in grins_racipe.h.
grins_status check_param_table(const grins_racipe *h, const grins_racipe_ranges &r)
{
    const int N = h->N, E = h->E;
    const bool strat = r.lhs_sets > 0 || r.sobol != GRINS_SOBOL_OFF;
    for (int d = 0; d < 2 * N + 3 * E; ++d) {
        const grins_param_range &p = r.param_ranges[d];
        const bool cont = d < 2 * N || (d >= 2 * N + E && d < 2 * N + 2 * E);
        if (!(std::isfinite(p.lo) && std::isfinite(p.hi) && p.lo > 0.0 && p.lo <= p.hi) || p.reserved != 0)
            return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d needs 0 < lo <= hi and reserved 0", d);
        if (!cont && p.dist != GRINS_DIST_TABLE1)
            return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d (threshold or Hill coefficient) takes dist 0", d);
        if (p.dist < GRINS_DIST_TABLE1 || p.dist > GRINS_DIST_LOGNORMAL)
            return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d has unknown distribution %d", d, p.dist);
        if (strat && p.dist > GRINS_DIST_LOGUNIFORM)
            return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d: stratified sets take Table 1 and log-uniform draws only", d);
        if (d >= 2 * N + E && d < 2 * N + 2 * E) {
            const bool act = h->sign[d - 2 * N - E] > 0;
            if (act ? p.lo < 1.0 : p.hi > 1.0)
                return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d: fold change on the wrong side of 1", d);
        }
        if (d >= 2 * N + 2 * E && (p.lo != std::floor(p.lo) || p.hi != std::floor(p.hi) || p.hi > 255.0))
            return fail(GRINS_E_INVALID_ARG, "param_ranges: row %d: Hill coefficients are integers in [1, 255]", d);
    }
    return GRINS_OK;
}

// A continuous parameter from row p (G, k or an activating lambda), or an
// inhibiting lambda (inverse range under Table 1).
double row_draw(const grins_param_range &p, bool inh, uint64_t x)
{
    if (inh && p.dist == GRINS_DIST_TABLE1) return 1.0 / span_map(1.0 / p.hi, 1.0 / p.lo, unit_double(x));
    return dist_draw(p.dist, p.lo, p.hi, x);
}

// Per-node medians of a per-parameter table (the definition stated with
// grins_racipe_node_medians): M0_j from node j's rows, then M_j with one
// factor per in-edge of j.
void table_medians(const grins_racipe *h, const grins_racipe_ranges &r, std::vector<double> &M)
{
    const int N = h->N, E = h->E, K = r.median_samples;
    const grins_param_range *P = r.param_ranges;
    std::vector<double> M0((size_t)N), v((size_t)K);
    for (int j = 0; j < N; ++j) {
        const MedianStream ms{(1ull << 63) + 2ull * (uint64_t)j};
        for (int s = 0; s < K; ++s)
            v[(size_t)s] = row_draw(P[j], false, ms.draw(s, 0)) / row_draw(P[N + j], false, ms.draw(s, 1));
        M0[(size_t)j] = median_sorted(v);
    }
    M = M0;
    if (r.median_mode != GRINS_MEDIAN_PER_INDEGREE) return;
    for (int j = 0; j < N; ++j) {
        std::vector<int> in;
        for (int e = 0; e < E; ++e)
            if (h->dst[e] == j) in.push_back(e);
        if (in.empty()) continue;
        const MedianStream ms{(1ull << 63) + 2ull * (uint64_t)j + 1ull};
        for (int s = 0; s < K; ++s) {
            double level = row_draw(P[j], false, ms.draw(s, 0)) / row_draw(P[N + j], false, ms.draw(s, 1));
            for (size_t q = 0; q < in.size(); ++q) {
                const int e = in[q], src = h->src[e];
                const bool act = h->sign[e] > 0;
                const uint64_t d = 2 + 5 * (uint64_t)q;
                const double Gs = row_draw(P[src], false, ms.draw(s, d));
                const double ks = row_draw(P[N + src], false, ms.draw(s, d + 1));
                const grins_param_range &pt = P[2 * N + e], &pl = P[2 * N + E + e], &pn = P[2 * N + 2 * E + e];
                const double T = span_map(pt.lo, pt.hi, unit_double(ms.draw(s, d + 2))) * M0[(size_t)src];
                const double lam = row_draw(pl, !act, ms.draw(s, d + 3));
                const int n = unit_int(ms.draw(s, d + 4), (int32_t)pn.lo, (int32_t)pn.hi - (int32_t)pn.lo + 1);
                level = level * hill_factor(act, Gs / ks, T, (double)n, lam);
            }
            v[(size_t)s] = level;
        }
        M[(size_t)j] = median_sorted(v);
    }
}

grins_status ensure_medians(grins_racipe *h, const grins_racipe_ranges &r)
{
    if (r.param_ranges) {
        grins_status st = check_param_table(h, r);
        if (st != GRINS_OK) return st;
        const size_t D = (size_t)(2 * h->N + 3 * h->E);
        const bool same_rows = h->median_table.size() == D &&
                               std::memcmp(h->median_table.data(), r.param_ranges, D * sizeof(grins_param_range)) == 0;
        if (h->median_valid && same_rows && same_ranges(h->median_ranges, r)) return GRINS_OK;
        table_medians(h, r, h->node_median);
        h->median_table.assign(r.param_ranges, r.param_ranges + D);
        h->median_ranges = r;
        h->median_valid = true;
        return GRINS_OK;
    }
    if (h->median_valid && h->median_table.empty() && same_ranges(h->median_ranges, r)) return GRINS_OK;
    h->median_table.clear();
    warm_class_medians(h, r);
    const double M0 = class_median(0, 0, r, 0.0);
    h->node_median.assign(h->N, M0);
    if (r.median_mode == GRINS_MEDIAN_PER_INDEGREE) {
        for (int j = 0; j < h->N; ++j) {
            const int na = h->n_act_in[j], ni = h->n_inh_in[j];
            if (na == 0 && ni == 0) continue;
            h->node_median[j] = class_median(na, ni, r, M0);
        }
    }
    h->median_ranges = r;
    h->median_valid = true;
    return GRINS_OK;
}

bool on_handle_device(const grins_racipe *h)
{
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && cur == h->device;
}

}  // namespace

extern "C" grins_status grins_racipe_node_medians(grins_racipe_t h, const grins_racipe_ranges *r,
                                                  double *out)
{
    AbiRange nvtx_range_("grins_racipe_node_medians");
    g_last_error.clear();
    if (!h || !out) return fail(GRINS_E_INVALID_ARG, "node_medians: NULL argument");
    grins_racipe_ranges rr;
    if (r) rr = *r; else grins_racipe_default_ranges(&rr);
    grins_status s = check_ranges(rr);
    if (s != GRINS_OK) return s;
    std::lock_guard<std::mutex> lock(h->median_mu);
    s = ensure_medians(h, rr);
    if (s != GRINS_OK) return s;
    std::copy(h->node_median.begin(), h->node_median.end(), out);
    return GRINS_OK;
}

// Sobol direction numbers of the first D dimensions, scrambled when asked,
// followed by the D digital shifts (zero unscrambled): the definitions
// stated with GRINS_SOBOL_* in grins_racipe.h.
static grins_status sobol_table(const grins_racipe_ranges &r, int D, uint64_t seed, std::vector<uint32_t> &out)
{
    if (r.sobol_dims < D || !r.sobol_poly || !r.sobol_m || r.sobol_m_cols < 1)
        return fail(GRINS_E_INVALID_ARG, "sample_params: Sobol tables need %d dimensions (have %d) and m columns",
                    D, r.sobol_dims);
    out.assign((size_t)D * 33, 0u);
    for (int d = 0; d < D; ++d) {
        uint64_t m[33];                                 // m[k], k = 1..32
        if (d == 0) {
            for (int k = 1; k <= 32; ++k) m[k] = 1;
        } else {
            const uint64_t p = (uint64_t)r.sobol_poly[d];
            int deg = 63;
            while (deg >= 0 && !((p >> deg) & 1ull)) --deg;
            if (deg < 1 || deg > 32 || deg > r.sobol_m_cols || !(p & 1ull))
                return fail(GRINS_E_INVALID_ARG, "sample_params: Sobol polynomial of dimension %d is invalid", d);
            for (int k = 1; k <= deg; ++k) {
                const int64_t mk = r.sobol_m[(size_t)d * r.sobol_m_cols + (k - 1)];
                if (mk < 1 || !(mk & 1) || mk >= (int64_t(1) << k))
                    return fail(GRINS_E_INVALID_ARG, "sample_params: Sobol m_%d of dimension %d is invalid", k, d);
                m[k] = (uint64_t)mk;
            }
            for (int k = deg + 1; k <= 32; ++k) {
                uint64_t v = m[k - deg] ^ (m[k - deg] << deg);
                for (int i = 1; i < deg; ++i)
                    if ((p >> (deg - i)) & 1ull) v ^= m[k - i] << i;
                m[k] = v;
            }
        }
        uint32_t *V = out.data() + (size_t)d * 32;
        for (int b = 0; b < 32; ++b) V[b] = (uint32_t)(m[b + 1] << (31 - b));
        if (r.sobol != GRINS_SOBOL_SCRAMBLED) continue;
        uint32_t M[33];                                 // row masks of the scramble, digit j = 1..32
        for (int j = 1; j <= 32; ++j) {
            uint64_t c[4] = {(uint64_t)d, (uint64_t)j, 0, 0};
            philox_host(c, seed, kTagSobol);
            const int bit = 32 - j;
            M[j] = (1u << bit) | (j >= 2 ? ((uint32_t)c[0] & (0xFFFFFFFFu << (bit + 1))) : 0u);
        }
        for (int b = 0; b < 32; ++b) {
            uint32_t y = 0;
            for (int j = 1; j <= 32; ++j)
                y |= (uint32_t)(__builtin_popcount(V[b] & M[j]) & 1) << (32 - j);
            V[b] = y;
        }
        uint64_t c[4] = {(uint64_t)d, 0, 0, 0};
        philox_host(c, seed, kTagSobol);
        out[(size_t)D * 32 + d] = (uint32_t)c[0];
    }
    return GRINS_OK;
}

// ------------------------------------------------------------------ sample
extern "C" grins_status grins_racipe_sample_params(grins_racipe_t h, const grins_racipe_ranges *r,
                                                   uint64_t seed, int64_t set0, int64_t n_sets,
                                                   int32_t n_ics, void *d_params, double *d_ic_unit,
                                                   void *stream)
{
    AbiRange nvtx_range_("grins_racipe_sample_params");
    g_last_error.clear();
    if (!h) return fail(GRINS_E_INVALID_ARG, "sample_params: NULL handle");
    if (set0 < 0 || n_sets < 0 || n_ics < 0)
        return fail(GRINS_E_INVALID_ARG, "sample_params: negative set0, n_sets or n_ics");
    if (n_sets > 0 && !d_params) return fail(GRINS_E_INVALID_ARG, "sample_params: d_params is NULL");
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "sample_params: current device is not the handle's");
    grins_racipe_ranges rr;
    if (r) rr = *r; else grins_racipe_default_ranges(&rr);
    grins_status s = check_ranges(rr);
    if (s != GRINS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the median of each edge's source under these ranges; the handle's
    // device copy when it holds exactly these values, else a staged copy
    std::vector<double> em((size_t)h->E);
    bool own_medians = false;
    {
        std::lock_guard<std::mutex> lock(h->median_mu);
        s = ensure_medians(h, rr);
        if (s != GRINS_OK) return s;
        for (int e = 0; e < h->E; ++e) em[(size_t)e] = h->node_median[h->src[e]];
        if (!h->edge_median_set && h->E > 0) {
            CUDA_TRY(cudaMemcpyAsync(h->d_edge_median, em.data(), sizeof(double) * h->E, cudaMemcpyHostToDevice, st),
                     "sample_params: median upload");
            CUDA_TRY(cudaStreamSynchronize(st), "sample_params: median upload");
            h->edge_median_host = em;
            h->edge_median_set = true;
        }
        own_medians = h->E > 0 && std::memcmp(em.data(), h->edge_median_host.data(), sizeof(double) * h->E) != 0;
    }
    SampleArgs a{};
    a.L = h->layout;
    a.edge_sign = h->d_edge_sign;
    a.edge_median = h->d_edge_median;
    a.seed = seed; a.set0 = set0; a.n_sets = n_sets;
    a.G_min = rr.G_min; a.G_span = rr.G_max - rr.G_min;
    a.k_min = rr.k_min; a.k_span = rr.k_max - rr.k_min;
    a.la_min = rr.lam_act_min; a.la_span = rr.lam_act_max - rr.lam_act_min;
    a.vi_min = 1.0 / rr.lam_inh_max;
    a.vi_span = 1.0 / rr.lam_inh_min - 1.0 / rr.lam_inh_max;
    a.thr_lo = rr.thr_lo; a.thr_span = rr.thr_hi - rr.thr_lo;
    a.n_min = rr.n_min; a.n_count = rr.n_max - rr.n_min + 1;
    a.dist_G = rr.dist_G; a.dist_k = rr.dist_k; a.dist_la = rr.dist_lam_act; a.dist_li = rr.dist_lam_inh;
    a.G_hi = rr.G_max; a.k_hi = rr.k_max; a.la_hi = rr.lam_act_max;
    a.lhs_sets = rr.lhs_sets;
    if (rr.lhs_sets > 0 && set0 + n_sets > rr.lhs_sets)
        return fail(GRINS_E_INVALID_ARG, "sample_params: sets [%lld, %lld) outside the Latin hypercube's %lld",
                    (long long)set0, (long long)(set0 + n_sets), (long long)rr.lhs_sets);
    a.li_min = rr.lam_inh_min; a.li_max = rr.lam_inh_max;
    a.params = static_cast<unsigned char *>(d_params);
    // tables the kernel reads besides the parameters: Sobol direction
    // numbers, per-parameter rows and, when they are not the handle's,
    // the edge medians, staged in one stream-ordered buffer
    const int D = 2 * h->N + 3 * h->E;
    std::vector<uint32_t> tab;
    if (rr.sobol != GRINS_SOBOL_OFF && n_sets > 0) {
        if (set0 + n_sets > (int64_t(1) << 32))
            return fail(GRINS_E_INVALID_ARG, "sample_params: Sobol sets beyond 2^32");
        s = sobol_table(rr, D, seed, tab);
        if (s != GRINS_OK) return s;
    }
    const size_t tab_bytes = (sizeof(uint32_t) * tab.size() + 15) / 16 * 16;
    const size_t row_bytes = rr.param_ranges ? sizeof(grins_param_range) * (size_t)D : 0;
    const size_t med_bytes = own_medians ? sizeof(double) * (size_t)h->E : 0;
    if (n_sets > 0 && tab_bytes + row_bytes + med_bytes > 0) {
        std::vector<unsigned char> blob(tab_bytes + row_bytes + med_bytes, 0);
        if (!tab.empty()) std::memcpy(blob.data(), tab.data(), sizeof(uint32_t) * tab.size());
        if (row_bytes) std::memcpy(blob.data() + tab_bytes, rr.param_ranges, row_bytes);
        if (med_bytes) std::memcpy(blob.data() + tab_bytes + row_bytes, em.data(), med_bytes);
        void *d_blob = nullptr;
        CUDA_TRY(dev_malloc_async(&d_blob, blob.size(), st), "sample_params: table buffer");
        cudaError_t e = cudaMemcpyAsync(d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
        unsigned char *base = static_cast<unsigned char *>(d_blob);
        if (!tab.empty()) {
            a.sobol_v = reinterpret_cast<const uint32_t *>(base);
            a.sobol_dims = D;
        }
        if (row_bytes) a.prange = reinterpret_cast<const grins_param_range *>(base + tab_bytes);
        if (med_bytes) a.edge_median = reinterpret_cast<const double *>(base + tab_bytes + row_bytes);
        if (e == cudaSuccess) e = launch_sample_params(a, st);
        const cudaError_t ef = cudaFreeAsync(d_blob, st);
        CUDA_TRY(e, "sample_params: launch");
        CUDA_TRY(ef, "sample_params: table buffer");
    } else {
        CUDA_TRY(launch_sample_params(a, st), "sample_params: launch");
    }
    if (d_ic_unit && n_ics > 0) {
        if (!rr.ic_ranges) {
            CUDA_TRY(launch_sample_ics(h->N, seed, n_ics, d_ic_unit, nullptr, st), "sample_params: IC launch");
        } else {
            for (int i = 0; i < h->N; ++i) {
                const grins_param_range &p = rr.ic_ranges[i];
                const bool logd = p.dist == GRINS_DIST_LOGUNIFORM || p.dist == GRINS_DIST_LOGNORMAL;
                if (p.dist < GRINS_DIST_TABLE1 || p.dist > GRINS_DIST_LOGNORMAL || p.reserved != 0 ||
                    !(p.lo >= 0.0 && p.lo <= p.hi && p.hi <= 1.0) || (logd && !(p.lo > 0.0)))
                    return fail(GRINS_E_INVALID_ARG, "ic_ranges: row %d needs 0 <= lo <= hi <= 1 (lo > 0 for log "
                                "distributions), a known dist and reserved 0", i);
            }
            void *d_rows = nullptr;
            const size_t bytes = sizeof(grins_param_range) * (size_t)h->N;
            CUDA_TRY(dev_malloc_async(&d_rows, bytes, st), "sample_params: IC rows");
            cudaError_t e = cudaMemcpyAsync(d_rows, rr.ic_ranges, bytes, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = launch_sample_ics(h->N, seed, n_ics, d_ic_unit, static_cast<const grins_param_range *>(d_rows), st);
            const cudaError_t ef = cudaFreeAsync(d_rows, st);
            CUDA_TRY(e, "sample_params: IC launch");
            CUDA_TRY(ef, "sample_params: IC rows");
        }
    }
    return GRINS_OK;
}

// --------------------------------------------------------------- integrate
static PolishArgs polish_args(const grins_racipe *h, const grins_solver_opts *o, const void *d_params,
                              int64_t n_sets, int32_t n_ics, double *d_states, uint8_t *d_status,
                              float *d_err_est)
{
    PolishArgs p{};
    p.topo = DevTopo{h->N, h->E, h->d_off, h->d_src, h->d_edge, h->d_sign};
    p.L = h->layout;
    p.params = static_cast<const unsigned char *>(d_params);
    p.n_solves = n_sets * (int64_t)n_ics;
    p.n_ics = n_ics;
    p.states = d_states;
    p.status = d_status;
    p.err_est = d_err_est;
    p.tol = o->polish_tol;
    p.max_move = o->polish_max_move;
    p.iters = o->polish_iters;
    p.check = h->d_queue + 2;
    p.cancel = o->cancel;
    return p;
}

static GrpTopo grp_topo(const grins_racipe *h) { return h->grp.topo(); }

// The FP64 integrator for h: the register-record kernel compiled for this
// network in FP64 (power-table edge terms) when the register layout exists,
// else the generic FP64 kernel (grp_jit null).  compile = false only looks
// up a kernel an earlier call compiled.
// A compiled register-record kernel for g, kind and variant if an earlier
// call compiled it, else the same with the re-pass flag toggled (a kernel
// compiled for the re-pass runs exactly as one without it when it is given
// no list).
static const void *lookup_either(const GrpTopo &g, int kind, int variant)
{
    const void *k = grp_jit_lookup(g, kind, variant);
    return k ? k : grp_jit_lookup(g, kind, variant ^ kJitTail);
}

static void pick_fp64_kernel(const grins_racipe *h, IntegrateArgs *a, bool compile, std::string *why,
                             bool tail = false, int kind = kJitRegisters64)
{
    a->grp = h->grp.topo();
    a->grp_jit = nullptr;
    std::string w = h->rr.L > 0 ? "" : "no register layout";
    if (h->rr.L > 0) {
        const GrpTopo g = h->rr.topo();
        const int variant = a->method | (a->n_t > 0 ? kJitSeries : 0) | (tail ? kJitTail : 0) |
                            (a->cancel ? kJitCancel : 0);
        // a lookup also takes the re-pass variant, which runs the same without a list
        const void *k = compile ? grp_jit_kernel(g, kind, &w, variant) : lookup_either(g, kind, variant);
        if (k) { a->grp = g; a->grp_jit = k; }
    }
    if (why) *why = w;
}

// Tolerance tightening near steady state: below a residual of 10 ss_tol the
// squared error norm is scaled by 1 / ss_tighten^2 (tolerances times
// ss_tighten).  Also fills the FP32 copies of the tolerance arguments, so
// it follows the assignment of rtol, atol, t_end and ss_tol.
static void set_tighten(IntegrateArgs *a, const grins_solver_opts *o)
{
    a->ss_near = 10.0 * o->ss_tol;
    a->ss_gain = 1.0 / (o->ss_tighten * o->ss_tighten);
    a->f_rtol = (float)a->rtol; a->f_atol = (float)a->atol; a->f_t_end = (float)a->t_end;
    a->f_ss_tol = (float)a->ss_tol; a->f_ss_near = (float)a->ss_near; a->f_ss_gain = (float)a->ss_gain;
    a->max_steps32 = (int32_t)std::min<int64_t>(o->max_steps, INT32_MAX);
    a->method = o->method;
}

// The FP32 lane-group kernel for h: sets a->grp and a->grp_jit to the
// kernel compiled for this network -- records in registers when the
// register layout exists, else records in shared memory (GRINS_JIT_KIND=grp
// asks for the latter) -- or leaves the run-time-layout kernel (grp_jit
// null).  compile = false only looks up kernels an earlier call compiled.
static bool pick_fp32_kernel(const grins_racipe *h, IntegrateArgs *a, bool compile, std::string *why,
                             bool tail = false)
{
    a->grp = h->grp.topo();
    a->grp_jit = nullptr;
    const char *ev = std::getenv("GRINS_JIT_KIND");
    const bool want_shared = ev && std::string(ev) == "grp";
    std::string w;
    if (!want_shared && h->rr.L > 0) {
        const GrpTopo g = h->rr.topo();
        const int variant = a->method | (a->n_t > 0 ? kJitSeries : 0) | (tail ? kJitTail : 0) |
                            (a->cancel ? kJitCancel : 0);
        const void *k = compile ? grp_jit_kernel(g, kJitRegisters, &w, variant)
                                : lookup_either(g, kJitRegisters, variant);
        if (k) { a->grp = g; a->grp_jit = k; if (why) *why = w; return true; }
    }
    if (h->grp.L > 0 && a->method == 0) {
        const void *k = compile ? grp_jit_kernel(a->grp, kJitShared, &w) : grp_jit_lookup(a->grp, kJitShared);
        if (k) a->grp_jit = k;
    }
    if (why) *why = w;
    return false;
}

static bool polish_opts_ok(const grins_solver_opts *o)
{
    return o->polish_tol > 0 && o->polish_iters >= 0 && o->polish_iters <= 64 && o->polish_max_move > 0;
}

extern "C" grins_status grins_racipe_polish(grins_racipe_t h, const grins_solver_opts *o,
                                            const void *d_params, int64_t n_sets, int32_t n_ics,
                                            double *d_states, uint8_t *d_status, float *d_err_est,
                                            void *stream)
{
    AbiRange nvtx_range_("grins_racipe_polish");
    g_last_error.clear();
    if (!h || !o) return fail(GRINS_E_INVALID_ARG, "polish: NULL handle or options");
    if (n_sets < 0 || n_ics < 1) return fail(GRINS_E_INVALID_ARG, "polish: bad sizes");
    if (n_sets > 0 && (!d_params || !d_states || !d_status))
        return fail(GRINS_E_INVALID_ARG, "polish: NULL required device buffer");
    if (!polish_opts_ok(o)) return fail(GRINS_E_INVALID_ARG, "polish: bad polish options");
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "polish: current device is not the handle's");
    if (n_sets == 0) return GRINS_OK;
    // units handed out from a counter (work per unit varies with its
    // converged solves: a fixed share left warps idle at the end)
    PolishArgs pa = polish_args(h, o, d_params, n_sets, n_ics, d_states, d_status, d_err_est);
    pa.queue = h->d_queue + 4;
    CUDA_TRY(cudaMemsetAsync(pa.queue, 0, sizeof(unsigned long long), (cudaStream_t)stream), "polish: counter");
    CUDA_TRY(launch_polish(pa, (cudaStream_t)stream, h->num_sms), "polish: launch");
    return GRINS_OK;
}

static bool tail_opts_ok(const grins_solver_opts *o)
{
    if (!(o->tail_rtol >= 0) || !std::isfinite(o->tail_rtol)) return false;
    if (o->tail_rtol == 0) return true;
    if (o->tail_precision != GRINS_TAIL_DD && o->tail_precision != GRINS_TAIL_FP64) return false;
    return o->tail_start >= 1 && std::isfinite(o->tail_start) && o->tail_rho >= 0 && std::isfinite(o->tail_rho) &&
           o->tail_late >= 0 && std::isfinite(o->tail_late) && o->tail_work >= 0;
}

static int slots_for(int n_ics)
{
    int s = (48 + n_ics - 1) / n_ics;
    return std::max(2, std::min(32, s));
}

extern "C" grins_status grins_racipe_integrate(grins_racipe_t h, const grins_solver_opts *o,
                                               const void *d_params, int64_t n_sets,
                                               const double *d_ic_unit, int32_t n_ics,
                                               double *d_states, uint8_t *d_status, double *d_t_final,
                                               float *d_err_est, int32_t *d_n_steps, double *d_series,
                                               void *stream)
{
    AbiRange nvtx_range_("grins_racipe_integrate");
    g_last_error.clear();
    if (!h || !o) return fail(GRINS_E_INVALID_ARG, "integrate: NULL handle or options");
    if (n_sets < 0) return fail(GRINS_E_INVALID_ARG, "integrate: n_sets < 0");
    if (n_ics < 1) return fail(GRINS_E_INVALID_ARG, "integrate: n_ics < 1");
    if (n_sets > 0 && (!d_params || !d_ic_unit || !d_states || !d_status))
        return fail(GRINS_E_INVALID_ARG, "integrate: NULL required device buffer");
    if (o->precision != GRINS_FP32 && o->precision != GRINS_FP64)
        return fail(GRINS_E_INVALID_ARG, "integrate: unknown precision %d", o->precision);
    if (!(o->rtol > 0) || !(o->atol > 0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
        return fail(GRINS_E_INVALID_ARG, "integrate: rtol and atol must be positive");
    if (!std::isfinite(o->t0) || !std::isfinite(o->t_end) || !(o->t_end > o->t0))
        return fail(GRINS_E_INVALID_ARG, "integrate: need finite t0 < t_end");
    if (!(o->ss_tol >= 0)) return fail(GRINS_E_INVALID_ARG, "integrate: ss_tol < 0");
    if (!(o->ss_tighten > 0 && o->ss_tighten <= 1)) return fail(GRINS_E_INVALID_ARG, "integrate: need 0 < ss_tighten <= 1");
    if (o->method != GRINS_METHOD_DOPRI5 && o->method != GRINS_METHOD_TSIT5)
        return fail(GRINS_E_INVALID_ARG, "integrate: unknown method %d", o->method);
    if (o->max_steps < 1) return fail(GRINS_E_INVALID_ARG, "integrate: max_steps < 1");
    if (o->n_t < 0 || (o->n_t > 0 && !o->t_grid)) return fail(GRINS_E_INVALID_ARG, "integrate: bad time grid");
    if ((o->n_t > 0) != (d_series != nullptr) && n_sets > 0)
        return fail(GRINS_E_INVALID_ARG, "integrate: d_series must be given exactly when n_t > 0");
    for (int g = 0; g < o->n_t; ++g) {
        const double tg = o->t_grid[g];
        if (!(tg >= o->t0 && tg <= o->t_end) || (g > 0 && !(tg > o->t_grid[g - 1])))
            return fail(GRINS_E_INVALID_ARG, "integrate: t_grid must increase strictly inside [t0, t_end]");
    }
    if (o->polish && !polish_opts_ok(o))
        return fail(GRINS_E_INVALID_ARG, "integrate: bad polish options");
    if (!tail_opts_ok(o)) return fail(GRINS_E_INVALID_ARG, "integrate: bad borderline re-pass options");
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "integrate: current device is not the handle's");
    if (n_sets == 0) return GRINS_OK;
    cudaStream_t st = (cudaStream_t)stream;

    if (o->n_t > h->grid_cap) {
        CUDA_TRY(cudaStreamSynchronize(st), "integrate: grid buffer");
        cudaFree(h->d_grid);
        h->d_grid = nullptr;
        h->grid_cap = 0;
        CUDA_TRY(dev_malloc(&h->d_grid, sizeof(double) * o->n_t), "integrate: grid buffer");
        h->grid_cap = o->n_t;
    }
    if (o->n_t > 0) {
        CUDA_TRY(cudaMemcpyAsync(h->d_grid, o->t_grid, sizeof(double) * o->n_t, cudaMemcpyHostToDevice, st),
                 "integrate: grid upload");
    }

    IntegrateArgs a{};
    a.topo = DevTopo{h->N, h->E, h->d_off, h->d_src, h->d_edge, h->d_sign};
    a.L = h->layout;
    a.params = static_cast<const unsigned char *>(d_params);
    a.n_sets = n_sets;
    a.ic_unit = d_ic_unit;
    a.n_ics = n_ics;
    a.rtol = o->rtol; a.atol = o->atol; a.t0 = o->t0; a.t_end = o->t_end; a.ss_tol = o->ss_tol;
    set_tighten(&a, o);
    a.max_steps = o->max_steps;
    a.t_grid = h->d_grid;
    a.n_t = o->n_t;
    a.states = d_states; a.status = d_status; a.t_final = d_t_final; a.n_steps = d_n_steps;
    a.series = o->n_t > 0 ? d_series : nullptr;
    a.queue = h->d_queue;
    a.check = h->d_queue + 2;
    a.slots = slots_for(n_ics);
    a.smem_limit = (int32_t)h->smem_optin;
    a.grp = grp_topo(h);
    a.cancel = o->cancel;
    IntegrateArgs a64{};             // the borderline re-pass, when it runs
    bool tail = false;
    IntegrateArgs::TailItem *tail_sorted = nullptr;   // its list, longest first
    if (o->precision == GRINS_FP32) {
        // grins_racipe_integrator describes the FP32 kernel: only its launches record it
        const bool want_tail = o->tail_rtol > 0 && o->n_t == 0;
        // the re-pass kernel's compile starts on the host pool while this
        // thread compiles the FP32 one (a first call waits for one, not both)
        if (want_tail && h->rr.L > 0)
            grp_jit_prefetch(h->rr.topo(), o->tail_precision == GRINS_TAIL_FP64 ? kJitRegisters64 : kJitRegistersDD,
                             a.method | kJitTail | (a.cancel ? kJitCancel : 0));
        const bool rr = pick_fp32_kernel(h, &a, true, &h->jit_why, want_tail);
        h->jit_used = a.grp_jit != nullptr;
        h->used_L = a.grp.L; h->used_R = a.grp.R; h->used_P = a.grp.P;
        h->used_method = a.method;
        h->tail_ran = false;
        if (o->tail_rtol <= 0) h->tail_why = "off";
        else if (o->n_t > 0) h->tail_why = "not run (time series requested)";
        else if (!rr) h->tail_why = "not run (no FP32 kernel compiled for the network)";
        else {
            a64 = a;
            std::string w64;
            pick_fp64_kernel(h, &a64, true, &w64, true,
                             o->tail_precision == GRINS_TAIL_FP64 ? kJitRegisters64 : kJitRegistersDD);
            if (!a64.grp_jit) h->tail_why = "not run (no re-pass kernel compiled for the network: " + w64 + ")";
            else tail = true;
        }
        if (tail) {
            const int64_t n_solves = n_sets * (int64_t)n_ics;
            if (n_solves > h->tail_cap) {
                CUDA_TRY(cudaStreamSynchronize(st), "integrate: re-pass buffer");
                cudaFree(h->d_tail);
                h->d_tail = nullptr;
                h->tail_cap = 0;
                CUDA_TRY(dev_malloc(&h->d_tail, 16 + 2 * sizeof(IntegrateArgs::TailItem) * (size_t)n_solves),
                         "integrate: re-pass buffer");
                h->tail_cap = n_solves;
            }
            auto *cnt = reinterpret_cast<unsigned long long *>(h->d_tail);
            auto *items = reinterpret_cast<IntegrateArgs::TailItem *>(h->d_tail + 16);
            tail_sorted = items + n_solves;
            CUDA_TRY(cudaMemsetAsync(cnt, 0, 16, st), "integrate: re-pass counters");
            a.tail_items = items;
            a.tail_n = cnt;
            a.f_tail_chk = (float)(o->tail_start * o->ss_tol);
            a.f_tail_rho = (float)(o->tail_rho * o->ss_tol);
            a.f_tail_late = (float)o->tail_late;
            a.tail_work = o->tail_work;
            a64.tail_items = tail_sorted;
            a64.tail_n = cnt;
            a64.rtol = o->tail_rtol;
            a64.atol = o->atol * (o->tail_rtol / o->rtol);
            a64.ss_near = 0.0;
            a64.ss_gain = 1.0;
            a64.f_rtol = (float)a64.rtol; a64.f_atol = (float)a64.atol;
            a64.f_ss_near = 0.0f; a64.f_ss_gain = 1.0f;
            h->tail_ran = true;
            char buf[160];
            std::snprintf(buf, sizeof(buf), "%s (kernel compiled for the network) from the checkpoint below %g "
                          "ss_tol at rtol %g", o->tail_precision == GRINS_TAIL_FP64 ? "FP64" : "double-float",
                          o->tail_start, o->tail_rtol);
            h->tail_why = buf;
        }
    } else {
        pick_fp64_kernel(h, &a, true, &h->jit_why64);
        h->jit_used64 = a.grp_jit != nullptr;
        h->ran64 = true;
    }
    if (a.method != GRINS_METHOD_DOPRI5 && !a.grp_jit)
        return fail(GRINS_E_INVALID_ARG, "integrate: the Tsitouras pair runs only on the kernel compiled for the "
                    "network, which is not available here");

    CUDA_TRY(cudaMemsetAsync(h->d_queue, 0, 2 * sizeof(unsigned long long), st), "integrate: queue reset");
    cudaError_t le;
    if (o->precision == GRINS_FP32) le = launch_integrate_fp32(a, st, h->num_sms);
    else le = launch_integrate_fp64(a, st, h->num_sms);
    if (le == cudaErrorInvalidConfiguration)
        return fail(GRINS_E_BUDGET, "integrate: the network needs more shared memory per block than the device has");
    if (le != cudaSuccess) return cuda_fail(le, "integrate: launch");
    if (o->pass_event)
        CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o->pass_event), st), "integrate: pass event");
    // With the re-pass and the polish both to run, the polish of every
    // solve the FP32 pass did not list (their statuses are final) runs on a
    // second stream beside the re-pass -- the re-pass is FP32 issue work, the
    // polish FP64 work, and the re-pass's last long solves leave SMs idle --
    // and a list-mode polish of the listed solves follows the re-pass.
    // The re-pass is launched before the forked polish becomes ready, so that
    // its blocks take their SM slots first; the polish's blocks fill what is
    // left and take over as the re-pass drains, drawing units from a counter.
    const bool overlap = tail && o->polish;
    if (overlap && !h->side) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "integrate: polish stream");
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "integrate: polish events");
        CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "integrate: polish events");
    }
    if (tail) {
        CUDA_TRY(launch_tail_order(a.tail_items, tail_sorted, a.tail_n, n_sets * (long long)n_ics, a.tail_work, st),
                 "integrate: re-pass order");
        CUDA_TRY(cudaMemsetAsync(h->d_queue, 0, 2 * sizeof(unsigned long long), st), "integrate: queue reset");
        if (overlap) {
            CUDA_TRY(cudaMemsetAsync(h->d_queue + 4, 0, 2 * sizeof(unsigned long long), st),
                     "integrate: polish counters");
            CUDA_TRY(cudaEventRecord(h->ev_fork, st), "integrate: fork");
            a64.tail_mark = 1;
        }
        le = launch_grp_jit(a64.grp_jit, a64, st, h->num_sms);
        if (le != cudaSuccess) return cuda_fail(le, "integrate: re-pass launch");
    }

    if (overlap) {
        PolishArgs pm = polish_args(h, o, d_params, n_sets, n_ics, d_states, d_status, d_err_est);
        pm.queue = h->d_queue + 4;
        CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0), "integrate: fork");
        CUDA_TRY(launch_polish(pm, h->side, h->num_sms), "integrate: polish launch");
        CUDA_TRY(cudaEventRecord(h->ev_join, h->side), "integrate: join");
        // the list-mode polish clears the listed solves' marks: it waits for
        // the polish beside the re-pass, which must not see a cleared mark
        CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0), "integrate: join");
        PolishArgs pl = polish_args(h, o, d_params, n_sets, n_ics, d_states, d_status, d_err_est);
        pl.items = tail_sorted;
        pl.n_items = a.tail_n;
        pl.queue = h->d_queue + 5;
        CUDA_TRY(launch_polish(pl, st, h->num_sms), "integrate: re-pass polish launch");
    } else if (o->polish) {
        PolishArgs pa = polish_args(h, o, d_params, n_sets, n_ics, d_states, d_status, d_err_est);
        pa.queue = h->d_queue + 4;
        CUDA_TRY(cudaMemsetAsync(pa.queue, 0, sizeof(unsigned long long), st), "integrate: polish counter");
        CUDA_TRY(launch_polish(pa, st, h->num_sms), "integrate: polish launch");
    } else if (d_err_est) {
        CUDA_TRY(cudaMemsetAsync(d_err_est, 0xff, sizeof(float) * n_sets * n_ics, st), "integrate: err_est");
    }
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_tail_stats(grins_racipe_t h, void *stream, int64_t *n_solves,
                                                int64_t *n_attempts)
{
    g_last_error.clear();
    if (!h || !n_solves || !n_attempts) return fail(GRINS_E_INVALID_ARG, "tail_stats: NULL argument");
    *n_solves = 0;
    *n_attempts = 0;
    if (!h->tail_ran || !h->d_tail) return GRINS_OK;
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "tail_stats: current device is not the handle's");
    unsigned long long w[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(w, h->d_tail, sizeof(w), cudaMemcpyDeviceToHost, (cudaStream_t)stream),
             "tail_stats: copy");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "tail_stats: synchronise");
    *n_solves = (int64_t)w[0];
    *n_attempts = (int64_t)w[1];
    return GRINS_OK;
}

// ------------------------------------------------------------------ rates
extern "C" grins_status grins_unit_rates(double *rates, void *stream)
{
    g_last_error.clear();
    if (!rates) return fail(GRINS_E_INVALID_ARG, "unit_rates: NULL argument");
    int dev = 0, n_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev), "unit_rates: device");
    CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "unit_rates: SM count");
    long long *d_cycles = nullptr;
    double *d_sink = nullptr;
    cudaError_t e = dev_malloc(&d_cycles, sizeof(long long) * n_sm);
    if (e == cudaSuccess) e = dev_malloc(&d_sink, sizeof(double) * n_sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cycles, 0, sizeof(long long) * n_sm, (cudaStream_t)stream);
    if (e == cudaSuccess) e = grins::measure_unit_rates(rates, (cudaStream_t)stream, d_cycles, d_sink, n_sm);
    const cudaError_t s = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(d_cycles);
    cudaFree(d_sink);
    if (e == cudaSuccess) e = s;
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? GRINS_E_NOMEM : GRINS_E_CUDA, "unit_rates: %s",
                    cudaGetErrorString(e));
    return GRINS_OK;
}

// ------------------------------------------------------------------ unique
extern "C" grins_status grins_racipe_unique_states(grins_racipe_t h, const void *d_params,
                                                   const double *d_states, const uint8_t *d_status,
                                                   int64_t n_sets, int32_t n_ics, double tol,
                                                   int32_t *d_state_id, int32_t *d_n_unique, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_unique_states");
    g_last_error.clear();
    if (!h) return fail(GRINS_E_INVALID_ARG, "unique_states: NULL handle");
    if (n_sets < 0 || n_ics < 1 || n_ics > 4096) return fail(GRINS_E_INVALID_ARG, "unique_states: bad sizes");
    if (!(tol >= 0) || !std::isfinite(tol)) return fail(GRINS_E_INVALID_ARG, "unique_states: tol must be >= 0");
    if (n_sets > 0 && (!d_params || !d_states || !d_status || !d_state_id || !d_n_unique))
        return fail(GRINS_E_INVALID_ARG, "unique_states: NULL device buffer");
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "unique_states: current device is not the handle's");
    UniqueArgs a{};
    a.L = h->layout;
    a.params = static_cast<const unsigned char *>(d_params);
    a.states = d_states; a.status = d_status;
    a.n_sets = n_sets; a.n_ics = n_ics; a.tol = tol;
    a.state_id = d_state_id; a.n_unique = d_n_unique;
    CUDA_TRY(launch_unique(a, (cudaStream_t)stream, h->num_sms), "unique_states: launch");
    return GRINS_OK;
}

// ------------------------------------------------------------------ levels
static grins_status level_args(grins_racipe_t h, const char *who, const void *d_params, const double *d_states,
                               const uint8_t *d_status, int64_t n_sets, int32_t n_ics, int32_t n_bins,
                               LevelArgs *a)
{
    if (!h) return fail(GRINS_E_INVALID_ARG, "%s: NULL handle", who);
    if (n_sets < 0 || n_ics < 1 || n_ics > 4096) return fail(GRINS_E_INVALID_ARG, "%s: bad sizes", who);
    if (n_bins < 2 || n_bins > 4096) return fail(GRINS_E_INVALID_ARG, "%s: n_bins outside [2, 4096]", who);
    if (n_sets > 0 && (!d_params || !d_states || !d_status))
        return fail(GRINS_E_INVALID_ARG, "%s: NULL device buffer", who);
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "%s: current device is not the handle's", who);
    *a = LevelArgs{};
    a->L = h->layout;
    a->params = static_cast<const unsigned char *>(d_params);
    a->states = d_states; a->status = d_status;
    a->n_sets = n_sets; a->n_ics = n_ics; a->n_bins = n_bins;
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_gk_histogram(grins_racipe_t h, const void *d_params, const double *d_states,
                                                  const uint8_t *d_status, int64_t n_sets, int32_t n_ics,
                                                  int32_t n_bins, unsigned long long *d_counts, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_gk_histogram");
    g_last_error.clear();
    LevelArgs a;
    const grins_status rc = level_args(h, "gk_histogram", d_params, d_states, d_status, n_sets, n_ics, n_bins, &a);
    if (rc != GRINS_OK) return rc;
    if (!d_counts) return fail(GRINS_E_INVALID_ARG, "gk_histogram: NULL counts");
    a.counts = d_counts;
    CUDA_TRY(launch_gk_histogram(a, (cudaStream_t)stream, h->num_sms), "gk_histogram: launch");
    return GRINS_OK;
}

// Boundary bins of a histogram of normalised values: binomially smoothed
// counts (Pascal's row 2m, exact in 64 bits), compressed into runs of equal
// counts; peaks and valleys among the runs; valleys taken from the highest
// down merge the groups of peaks on their two sides (union-find, each group
// keeping its highest peak); a merge whose absorbed group's peak is at
// least twice the valley and at least 1/64 of the highest count makes the
// valley's middle bin a boundary; the lowest valleys are kept first.
extern "C" grins_status grins_level_boundaries(const unsigned long long *h_counts, int32_t n_bins,
                                               int32_t half_width, int32_t max_boundaries, int32_t *h_bins,
                                               int32_t *n_out)
{
    g_last_error.clear();
    if (!h_counts || !h_bins || !n_out) return fail(GRINS_E_INVALID_ARG, "level_boundaries: NULL pointer");
    if (n_bins < 2 || n_bins > 4096) return fail(GRINS_E_INVALID_ARG, "level_boundaries: n_bins outside [2, 4096]");
    if (half_width < 0 || half_width > 8)
        return fail(GRINS_E_INVALID_ARG, "level_boundaries: half_width outside [0, 8]");
    if (max_boundaries < 1 || max_boundaries > kMaxLevelBounds)
        return fail(GRINS_E_INVALID_ARG, "level_boundaries: max_boundaries outside [1, %d]", kMaxLevelBounds);
    const int B = n_bins, m = half_width;
    std::vector<unsigned long long> wt(1, 1ull);                  // row 2m of Pascal's triangle
    for (int r = 1; r <= 2 * m; ++r) {
        std::vector<unsigned long long> nx(r + 1, 1ull);
        for (int j = 1; j < r; ++j) nx[j] = wt[j - 1] + wt[j];
        wt.swap(nx);
    }
    std::vector<unsigned long long> sm(B, 0ull);
    for (int b = 0; b < B; ++b)
        for (int j = -m; j <= m; ++j)
            if (b + j >= 0 && b + j < B) sm[b] += wt[j + m] * h_counts[b + j];
    const unsigned long long top = *std::max_element(sm.begin(), sm.end());
    struct Run { int b0, b1; unsigned long long v; };
    std::vector<Run> run;
    for (int b = 0; b < B; ++b) {
        if (!run.empty() && run.back().v == sm[b]) run.back().b1 = b;
        else run.push_back({b, b, sm[b]});
    }
    const int R = (int)run.size();
    std::vector<char> peak(R, 0);
    std::vector<int> valleys;
    for (int r = 0; r < R && R > 1; ++r) {
        const bool below_l = r == 0 || run[r - 1].v < run[r].v, below_r = r == R - 1 || run[r + 1].v < run[r].v;
        if (below_l && below_r) peak[r] = 1;
        if (r > 0 && r < R - 1 && run[r - 1].v > run[r].v && run[r + 1].v > run[r].v) valleys.push_back(r);
    }
    std::vector<int> parent(R);
    for (int r = 0; r < R; ++r) parent[r] = r;
    auto root = [&](int r) { while (parent[r] != r) r = parent[r] = parent[parent[r]]; return r; };
    std::vector<int> best(R);                                     // a group's highest peak run (first among equals)
    for (int r = 0; r < R; ++r) best[r] = r;
    std::sort(valleys.begin(), valleys.end(), [&](int a, int b) {
        return run[a].v != run[b].v ? run[a].v > run[b].v : run[a].b0 < run[b].b0;
    });
    std::vector<std::pair<unsigned long long, int>> cut;          // (valley count, boundary bin)
    for (int v : valleys) {
        int pl = v - 1, pr = v + 1;
        while (!peak[pl]) --pl;
        while (!peak[pr]) ++pr;
        const int gl = root(pl), gr = root(pr);
        const unsigned long long hl = run[best[gl]].v, hr = run[best[gr]].v;
        // absorbed: the lower highest peak; equal peaks: the one further right
        const bool left_absorbed = hl < hr || (hl == hr && best[gl] > best[gr]);
        const int young = left_absorbed ? gl : gr, old = left_absorbed ? gr : gl;
        const unsigned long long h = run[best[young]].v, d = run[v].v;
        if (2 * d <= h && 64 * h >= top) cut.push_back({d, (run[v].b0 + run[v].b1) / 2});
        parent[young] = old;
    }
    std::sort(cut.begin(), cut.end());
    if ((int)cut.size() > max_boundaries) cut.resize(max_boundaries);
    std::vector<int> bins;
    for (const auto &p : cut) bins.push_back(p.second);
    std::sort(bins.begin(), bins.end());
    for (size_t t = 0; t < bins.size(); ++t) h_bins[t] = bins[t];
    *n_out = (int32_t)bins.size();
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_level_states(grins_racipe_t h, const void *d_params, const double *d_states,
                                                  const uint8_t *d_status, int64_t n_sets, int32_t n_ics,
                                                  int32_t n_bins, const int32_t *h_bounds, int32_t n_bounds,
                                                  unsigned long long *d_labels, int32_t *d_n_states,
                                                  unsigned long long *d_multi_hist, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_level_states");
    g_last_error.clear();
    LevelArgs a;
    const grins_status rc = level_args(h, "level_states", d_params, d_states, d_status, n_sets, n_ics, n_bins, &a);
    if (rc != GRINS_OK) return rc;
    if (n_bounds < 0 || n_bounds > kMaxLevelBounds || (n_bounds > 0 && !h_bounds))
        return fail(GRINS_E_INVALID_ARG, "level_states: n_bounds outside [0, %d] or NULL bounds", kMaxLevelBounds);
    for (int t = 0; t < n_bounds; ++t)
        if (h_bounds[t] < 0 || h_bounds[t] >= n_bins || (t > 0 && h_bounds[t] <= h_bounds[t - 1]))
            return fail(GRINS_E_INVALID_ARG, "level_states: boundaries must increase within [0, n_bins)");
    if (n_sets > 0 && (!d_labels || !d_n_states || !d_multi_hist))
        return fail(GRINS_E_INVALID_ARG, "level_states: NULL output buffer");
    int width = 0;
    while ((1 << width) < n_bounds + 1) ++width;
    if ((long long)h->N * width > 64)
        return fail(GRINS_E_BUDGET, "level_states: %d nodes x %d bits exceed a 64-bit label", h->N, width);
    a.n_bounds = n_bounds;
    for (int t = 0; t < n_bounds; ++t) a.bounds[t] = h_bounds[t];
    a.width = width;
    a.labels = d_labels; a.n_states = d_n_states; a.multi_hist = d_multi_hist;
    CUDA_TRY(launch_level_states(a, (cudaStream_t)stream, h->num_sms), "level_states: launch");
    return GRINS_OK;
}

// ------------------------------------------------------------------- Ising
extern "C" grins_status grins_ising_run(grins_racipe_t h, int32_t mode, int32_t enc01, uint64_t seed,
                                        int64_t n_traj, const unsigned long long *d_init, int32_t max_steps,
                                        unsigned long long *d_final, int32_t *d_steps, uint8_t *d_status,
                                        void *stream)
{
    AbiRange nvtx_range_("grins_ising_run");
    g_last_error.clear();
    if (!h) return fail(GRINS_E_INVALID_ARG, "ising_run: NULL handle");
    if (mode != GRINS_ISING_SYNC && mode != GRINS_ISING_ASYNC) return fail(GRINS_E_INVALID_ARG, "ising_run: unknown mode %d", mode);
    if (n_traj < 0 || max_steps < 0) return fail(GRINS_E_INVALID_ARG, "ising_run: negative size");
    if (n_traj > 0 && (!d_final || !d_steps || !d_status)) return fail(GRINS_E_INVALID_ARG, "ising_run: NULL output buffer");
    if (!on_handle_device(h)) return fail(GRINS_E_INVALID_ARG, "ising_run: current device is not the handle's");
    IsingArgs a{};
    a.N = h->N; a.mode = mode; a.enc01 = enc01 ? 1 : 0; a.max_steps = max_steps;
    a.seed = seed; a.n_traj = n_traj; a.init = d_init;
    a.final_state = d_final; a.steps = d_steps; a.status = d_status;
    for (int e = 0; e < h->E; ++e) {
        const int i = h->dst[e];
        if (h->sign[e] > 0) { a.act[i] |= 1ull << h->src[e]; ++a.n_act[i]; }
        else { a.inh[i] |= 1ull << h->src[e]; ++a.n_inh[i]; }
    }
    CUDA_TRY(launch_ising(a, (cudaStream_t)stream, h->num_sms), "ising_run: launch");
    return GRINS_OK;
}

// ------------------------------------------------------------------- plans
// A plan integrates many networks (jobs) in one batched launch of the
// lane-group kernel, followed by each job's polish and dedupe, all captured
// once into a CUDA graph that grins_racipe_plan_run replays.
struct grins_racipe_plan {
    int device = 0, num_sms = 1, smem_limit = 0;
    grins_solver_opts opts{};
    std::vector<grins_racipe_job> jobs;
    std::vector<IntegrateArgs> args;
    IntegrateArgs *d_args = nullptr;
    double *d_cum = nullptr;
    unsigned long long *d_counters = nullptr;   // per job: queue, spare, check code, check info
    BatchArgs batch{};
    int warps = 4, slot_extra = 1;
    int mode = 0;                          // 0: one persistent launch (run-time layouts); 1: per-job compiled
                                           // kernels on branches; 2: one persistent launch of a kernel compiled
                                           // for every job's layout
    const void *ct_kern = nullptr;         // mode 2: the plan kernel
    int ct_warps = 4;                      // mode 2: warps per block
    int ct_minb = 3;                       // mode 2: resident blocks per SM (register cap of every body)
    std::vector<int32_t> body_of;          // mode 2: each job's body
    int ct_bodies = 0;
    IntegrateArgs *d_ct_args = nullptr;    // mode 2: per-job arguments with the register layouts
    int32_t *d_body_of = nullptr;
    PlanArgs ct{};
    std::string ct_why;
    bool prefetched = false;               // mode 1: the per-job compiles were started
    std::vector<IntegrateArgs> jargs;      // mode 1: per-job arguments (compiled kernel and its layout)
    std::vector<size_t> order;             // mode 1: jobs by decreasing work
    std::vector<cudaStream_t> side;        // mode 1: branch streams
    std::vector<cudaEvent_t> events;       // mode 1: fork event, then one join event per branch
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string info;
};

static void plan_free(grins_racipe_plan *p)
{
    cudaFree(p->d_ct_args); cudaFree(p->d_body_of);
    p->d_ct_args = nullptr; p->d_body_of = nullptr;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (cudaStream_t x : p->side) cudaStreamDestroy(x);
    for (cudaEvent_t x : p->events) cudaEventDestroy(x);
    p->side.clear();
    p->events.clear();
    cudaFree(p->d_args); cudaFree(p->d_cum); cudaFree(p->d_counters);
    p->exec = nullptr; p->graph = nullptr; p->cap_stream = nullptr;
    p->d_args = nullptr; p->d_cum = nullptr; p->d_counters = nullptr;
}

// Per-job integrator arguments for a slot rule (extra slots per domain) and,
// when `sample` > 1, only the first 1/sample of each job's sets.
static void plan_args(grins_racipe_plan *p, int slot_extra, int sample)
{
    p->args.assign(p->jobs.size(), IntegrateArgs{});
    int wb = 0;
    for (size_t b = 0; b < p->jobs.size(); ++b) {
        const grins_racipe_job &j = p->jobs[b];
        const grins_racipe *h = j.net;
        const grins_solver_opts *o = &p->opts;
        IntegrateArgs &a = p->args[b];
        a.topo = DevTopo{h->N, h->E, h->d_off, h->d_src, h->d_edge, h->d_sign};
        a.L = h->layout;
        a.params = static_cast<const unsigned char *>(j.d_params);
        a.n_sets = sample > 1 ? (j.n_sets + sample - 1) / sample : j.n_sets;
        a.ic_unit = j.d_ic_unit;
        a.n_ics = j.n_ics;
        a.rtol = o->rtol; a.atol = o->atol; a.t0 = o->t0; a.t_end = o->t_end; a.ss_tol = o->ss_tol;
    set_tighten(&a, o);
        a.max_steps = o->max_steps;
        a.t_grid = nullptr;
        a.n_t = 0;
        a.states = j.d_states; a.status = j.d_status; a.t_final = j.d_t_final; a.n_steps = j.d_n_steps;
        a.series = nullptr;
        a.queue = p->d_counters + 4 * b;
        a.check = p->d_counters + 4 * b + 2;
        a.smem_limit = p->smem_limit;
        a.grp = grp_topo(h);
        a.grp_jit = nullptr;
        a.cancel = o->cancel;
        const int ndom = grp_domains(a.grp.L);
        const int groups = kWarp / a.grp.L / ndom;
        int sd = (groups + j.n_ics - 1) / j.n_ics + slot_extra;
        sd = std::max(1, std::min(16, sd));
        a.slots = sd * ndom;
        wb = std::max(wb, GrpLayout{a.grp.L, a.grp.R, a.grp.P, a.slots}.warp_bytes());
    }
    p->batch.warp_bytes = wb;
}

static grins_status plan_upload(grins_racipe_plan *p, cudaStream_t st)
{
    CUDA_TRY(cudaMemcpyAsync(p->d_args, p->args.data(), sizeof(IntegrateArgs) * p->args.size(),
                             cudaMemcpyHostToDevice, st), "plan: argument upload");
    CUDA_TRY(cudaStreamSynchronize(st), "plan: argument upload");
    return GRINS_OK;
}

// Polish and dedupe of job b on stream st.
static grins_status plan_job_tail(grins_racipe_plan *p, size_t b, cudaStream_t st)
{
    const grins_racipe_job &j = p->jobs[b];
    if (j.n_sets == 0) return GRINS_OK;
    if (p->opts.polish) {
        PolishArgs pa = polish_args(j.net, &p->opts, j.d_params, j.n_sets, j.n_ics, j.d_states, j.d_status,
                                    j.d_err_est);
        pa.check = p->d_counters + 4 * b + 2;
        pa.queue = p->d_counters + 4 * b;              // the job's integrate is done with it
        CUDA_TRY(cudaMemsetAsync(pa.queue, 0, sizeof(unsigned long long), st), "plan: polish counter");
        CUDA_TRY(launch_polish(pa, st, p->num_sms), "plan: polish launch");
    } else if (j.d_err_est) {
        CUDA_TRY(cudaMemsetAsync(j.d_err_est, 0xff, sizeof(float) * j.n_sets * j.n_ics, st), "plan: err_est");
    }
    if (j.d_state_id) {
        UniqueArgs u{};
        u.L = j.net->layout;
        u.params = static_cast<const unsigned char *>(j.d_params);
        u.states = j.d_states; u.status = j.d_status;
        u.n_sets = j.n_sets; u.n_ics = j.n_ics; u.tol = j.dedupe_tol;
        u.state_id = j.d_state_id; u.n_unique = j.d_n_unique;
        CUDA_TRY(launch_unique(u, st, p->num_sms), "plan: dedupe launch");
    }
    return GRINS_OK;
}

// The plan's work on stream st: reset the counters, then either the
// persistent batched integration followed by every job's polish and dedupe,
// or, per job on a branch stream forked from st, its compiled integrator,
// polish and dedupe, the branches joined back into st.
static grins_status plan_enqueue(grins_racipe_plan *p, cudaStream_t st, bool integrate_only)
{
    CUDA_TRY(cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned long long) * 4 * p->jobs.size(), st),
             "plan: counter reset");
    if (p->mode == 0 || p->mode == 2) {
        const cudaError_t e = p->mode == 2 ? launch_plan_ct(p->ct_kern, p->ct, st, p->num_sms, p->smem_limit)
                                           : launch_integrate_batch(p->batch, p->warps, st, p->num_sms, p->smem_limit);
        if (e == cudaErrorInvalidConfiguration)
            return fail(GRINS_E_BUDGET, "plan: the persistent launch needs more shared memory per block than the "
                        "device has");
        if (e != cudaSuccess) return cuda_fail(e, "plan: persistent launch");
        if (integrate_only) return GRINS_OK;
        // the jobs' polish and dedupe, dealt out to the branch streams
        const int K = (int)p->side.size();
        CUDA_TRY(cudaEventRecord(p->events[0], st), "plan: fork");
        for (int k = 0; k < K; ++k) CUDA_TRY(cudaStreamWaitEvent(p->side[k], p->events[0], 0), "plan: fork");
        for (size_t q = 0; q < p->order.size(); ++q) {
            const grins_status s = plan_job_tail(p, p->order[q], p->side[q % K]);
            if (s != GRINS_OK) return s;
        }
        for (int k = 0; k < K; ++k) {
            CUDA_TRY(cudaEventRecord(p->events[1 + k], p->side[k]), "plan: join");
            CUDA_TRY(cudaStreamWaitEvent(st, p->events[1 + k], 0), "plan: join");
        }
        return GRINS_OK;
    }
    const int K = (int)p->side.size();
    CUDA_TRY(cudaEventRecord(p->events[0], st), "plan: fork");
    for (int k = 0; k < K; ++k) CUDA_TRY(cudaStreamWaitEvent(p->side[k], p->events[0], 0), "plan: fork");
    for (size_t q = 0; q < p->order.size(); ++q) {
        const size_t b = p->order[q];
        cudaStream_t sb = p->side[q % K];
        if (p->jargs[b].n_sets > 0) {
            const cudaError_t e = launch_integrate_fp32(p->jargs[b], sb, p->num_sms);
            if (e == cudaErrorInvalidConfiguration)
                return fail(GRINS_E_BUDGET, "plan: job %zu needs more shared memory per block than the device has", b);
            if (e != cudaSuccess) return cuda_fail(e, "plan: job launch");
        }
        if (!integrate_only) {
            const grins_status s = plan_job_tail(p, b, sb);
            if (s != GRINS_OK) return s;
        }
    }
    for (int k = 0; k < K; ++k) {
        CUDA_TRY(cudaEventRecord(p->events[1 + k], p->side[k]), "plan: join");
        CUDA_TRY(cudaStreamWaitEvent(st, p->events[1 + k], 0), "plan: join");
    }
    return GRINS_OK;
}

// Mode 2 setup (after plan_args): the distinct register layouts of the
// jobs' networks, the plan kernel compiled for them (once), and per-job
// arguments pointing at each network's register layout, uploaded with the
// job -> body map.  GRINS_E_BUDGET when a network has no register layout or
// the kernel cannot be compiled.
static grins_status plan_setup_branches(grins_racipe_plan *p, bool prefetch);

static grins_status plan_setup_ct(grins_racipe_plan *p, cudaStream_t st)
{
    const size_t n = p->jobs.size();
    const grins_status sb = plan_setup_branches(p, false);
    if (sb != GRINS_OK) return sb;
    std::vector<GrpTopo> lays;
    std::vector<int32_t> body(n);
    int gather = 0;
    for (size_t b = 0; b < n; ++b) {
        const grins_racipe *h = p->jobs[b].net;
        if (h->rr.L <= 0) return fail(GRINS_E_BUDGET, "plan: job %zu's network has no register layout", b);
        const GrpTopo g = h->rr.topo();
        int found = -1;
        for (size_t i = 0; i < lays.size() && found < 0; ++i) {
            const GrpTopo &x = lays[i];
            bool same = x.L == g.L && x.R == g.R && x.P == g.P;
            for (int r = 0; same && r < g.R; ++r)
                same = x.row_off[r] == g.row_off[r] && x.row_deg[r] == g.row_deg[r] && x.link_to[r] == g.link_to[r];
            if (same) found = (int)i;
        }
        if (found < 0) { found = (int)lays.size(); lays.push_back(g); }
        body[b] = found;
        gather = std::max(gather, rr_warp_bytes(g.R, 1, 4));
    }
    p->ct_kern = grp_jit_plan_kernel(lays.data(), (int)lays.size(), p->ct_warps, p->ct_minb,
                                     p->opts.cancel != nullptr, &p->ct_why);
    if (!p->ct_kern) return fail(GRINS_E_BUDGET, "plan: no compiled plan kernel (%s)", p->ct_why.c_str());
    p->ct_bodies = (int)lays.size();
    std::vector<IntegrateArgs> a = p->args;
    for (size_t b = 0; b < n; ++b) {
        a[b].grp = p->jobs[b].net->rr.topo();
        a[b].grp_jit = nullptr;
    }
    if (!p->d_ct_args) {
        CUDA_TRY(dev_malloc(&p->d_ct_args, sizeof(IntegrateArgs) * n), "plan: arguments");
        CUDA_TRY(dev_malloc(&p->d_body_of, sizeof(int32_t) * n), "plan: body map");
    }
    CUDA_TRY(cudaMemcpyAsync(p->d_ct_args, a.data(), sizeof(IntegrateArgs) * n, cudaMemcpyHostToDevice, st),
             "plan: argument upload");
    CUDA_TRY(cudaMemcpyAsync(p->d_body_of, body.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st),
             "plan: body map upload");
    CUDA_TRY(cudaStreamSynchronize(st), "plan: argument upload");
    p->body_of = body;
    gather = (gather + 127) / 128 * 128;
    p->ct = PlanArgs{p->d_ct_args, p->d_cum, p->d_body_of, (int32_t)n, gather,
                     gather + (int)((sizeof(IntegrateArgs) + 127) / 128 * 128)};
    return GRINS_OK;
}

// Mode 1 setup: branch streams and events, the job order, and per-job
// arguments (from p->args) with the kernel compiled for each job's network;
// the compiles run in parallel on the host pool.
static grins_status plan_setup_branches(grins_racipe_plan *p, bool prefetch);

static grins_status plan_setup_jobs(grins_racipe_plan *p)
{
    const size_t n = p->jobs.size();
    const grins_status s = plan_setup_branches(p, true);
    if (s != GRINS_OK) return s;
    p->jargs = p->args;
    for (size_t b = 0; b < n; ++b) pick_fp32_kernel(p->jobs[b].net, &p->jargs[b], true, nullptr);
    return GRINS_OK;
}

// Branch streams and events, and the jobs by decreasing work (once per
// plan); with `prefetch` the compiles of every job's kernel are started on
// the host pool.
static grins_status plan_setup_branches(grins_racipe_plan *p, bool prefetch)
{
    const size_t n = p->jobs.size();
    if (p->side.empty()) {
        const int K = (int)std::min<size_t>(16, n);
        p->side.assign(K, nullptr);
        p->events.assign(K + 1, nullptr);
        for (auto &x : p->side) CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "plan: branch streams");
        for (auto &x : p->events) CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "plan: events");
        p->order.resize(n);
        for (size_t b = 0; b < n; ++b) p->order[b] = b;
        std::stable_sort(p->order.begin(), p->order.end(), [p](size_t x, size_t y) {
            auto work = [p](size_t b) {
                const grins_racipe_job &j = p->jobs[b];
                return (double)j.n_sets * j.n_ics * (j.net->E + j.net->N);
            };
            return work(x) > work(y);
        });
    }
    if (prefetch && !p->prefetched) {
        p->prefetched = true;
        for (size_t b = 0; b < n; ++b) {          // start every compile before waiting for any
            const grins_racipe *h = p->jobs[b].net;
            if (h->rr.L > 0) grp_jit_prefetch(h->rr.topo(), kJitRegisters, p->opts.cancel ? kJitCancel : 0);
            else grp_jit_prefetch(h->grp.topo(), kJitShared);
        }
    }
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_plan_create(const grins_solver_opts *o, const grins_racipe_job *jobs,
                                                 int32_t n_jobs, int32_t autotune, void *stream,
                                                 grins_racipe_plan_t *out)
{
    AbiRange nvtx_range_("grins_racipe_plan_create");
    g_last_error.clear();
    if (!o || !out || (n_jobs > 0 && !jobs)) return fail(GRINS_E_INVALID_ARG, "plan_create: NULL argument");
    *out = nullptr;
    if (n_jobs < 1) return fail(GRINS_E_INVALID_ARG, "plan_create: n_jobs < 1");
    if (o->precision != GRINS_FP32) return fail(GRINS_E_INVALID_ARG, "plan_create: plans integrate in FP32");
    if (!(o->rtol > 0) || !(o->atol > 0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
        return fail(GRINS_E_INVALID_ARG, "plan_create: rtol and atol must be positive");
    if (!std::isfinite(o->t0) || !std::isfinite(o->t_end) || !(o->t_end > o->t0))
        return fail(GRINS_E_INVALID_ARG, "plan_create: need finite t0 < t_end");
    if (!(o->ss_tol >= 0) || o->max_steps < 1) return fail(GRINS_E_INVALID_ARG, "plan_create: bad ss_tol or max_steps");
    if (!(o->ss_tighten > 0 && o->ss_tighten <= 1)) return fail(GRINS_E_INVALID_ARG, "plan_create: need 0 < ss_tighten <= 1");
    if (o->method != GRINS_METHOD_DOPRI5) return fail(GRINS_E_INVALID_ARG, "plan_create: plans run Dormand-Prince only");
    if (o->n_t != 0) return fail(GRINS_E_INVALID_ARG, "plan_create: plans do not write time series");
    if (o->polish && !polish_opts_ok(o)) return fail(GRINS_E_INVALID_ARG, "plan_create: bad polish options");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev), "plan_create: current device");
    for (int b = 0; b < n_jobs; ++b) {
        const grins_racipe_job &j = jobs[b];
        if (!j.net) return fail(GRINS_E_INVALID_ARG, "plan_create: job %d has no network", b);
        if (j.net->device != dev) return fail(GRINS_E_INVALID_ARG, "plan_create: job %d's network is on another device", b);
        if (j.n_sets < 0 || j.n_ics < 1) return fail(GRINS_E_INVALID_ARG, "plan_create: job %d has bad sizes", b);
        if (j.n_sets > 0 && (!j.d_params || !j.d_ic_unit || !j.d_states || !j.d_status))
            return fail(GRINS_E_INVALID_ARG, "plan_create: job %d lacks a required device buffer", b);
        if ((j.d_state_id == nullptr) != (j.d_n_unique == nullptr))
            return fail(GRINS_E_INVALID_ARG, "plan_create: job %d: give both dedupe outputs or neither", b);
        if (j.d_state_id && (!(j.dedupe_tol >= 0) || !std::isfinite(j.dedupe_tol) || j.n_ics > 4096))
            return fail(GRINS_E_INVALID_ARG, "plan_create: job %d: bad dedupe tolerance or n_ics", b);
        if (j.net->grp.L <= 0 || j.net->grp.R > 8)
            return fail(GRINS_E_BUDGET, "plan_create: job %d's network has no lane-group layout of at most 8 rows", b);
    }
    grins_racipe_plan *p = new (std::nothrow) grins_racipe_plan();
    if (!p) return fail(GRINS_E_NOMEM, "plan_create: host allocation failed");
    p->device = dev;
    p->num_sms = jobs[0].net->num_sms;
    p->smem_limit = (int)jobs[0].net->smem_optin;
    p->opts = *o;
    p->jobs.assign(jobs, jobs + n_jobs);
    // share of the work per job ~ solves x (edges + nodes)
    std::vector<double> cum(n_jobs);
    double tot = 0.0;
    for (int b = 0; b < n_jobs; ++b) {
        tot += (double)jobs[b].n_sets * jobs[b].n_ics * (jobs[b].net->E + jobs[b].net->N);
        cum[b] = tot;
    }
    for (int b = 0; b < n_jobs; ++b) cum[b] = tot > 0 ? cum[b] / tot : (b + 1.0) / n_jobs;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t ce = dev_malloc(&p->d_args, sizeof(IntegrateArgs) * n_jobs);
    if (ce == cudaSuccess) ce = dev_malloc(&p->d_cum, sizeof(double) * n_jobs);
    if (ce == cudaSuccess) ce = dev_malloc(&p->d_counters, sizeof(unsigned long long) * 4 * n_jobs);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_cum, cum.data(), sizeof(double) * n_jobs, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) { plan_free(p); delete p; return cuda_fail(ce, "plan_create: device buffers"); }
    p->batch.jobs = p->d_args;
    p->batch.cum_work = p->d_cum;
    p->batch.n_jobs = n_jobs;

    // autotuner: block size (warps per block) x slots per scheduling domain,
    // each timed on the first sixteenth of every job's sets
    char buf[512];
    std::string tried;
    if (autotune < 0 || autotune > 3) { plan_free(p); delete p; return fail(GRINS_E_INVALID_ARG, "plan_create: autotune must be 0, 1, 2 or 3"); }
    if (autotune == 1) {
        float best = -1.0f;
        int bw = 4, bx = 1;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int w : {2, 4}) {
            for (int x : {1, 2}) {
                plan_args(p, x, 16);
                p->warps = w;
                grins_status s = plan_upload(p, st);
                if (s != GRINS_OK) { plan_free(p); delete p; return s; }
                cudaEventRecord(e0, st);
                s = plan_enqueue(p, st, true);
                cudaEventRecord(e1, st);
                if (s == GRINS_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    std::snprintf(buf, sizeof(buf), "%s%d warps/%d extra slots: %.3f ms", tried.empty() ? "" : "; ",
                                  w, x, ms);
                    tried += buf;
                    if (best < 0 || ms < best) { best = ms; bw = w; bx = x; }
                } else if (s != GRINS_E_BUDGET) {
                    cudaEventDestroy(e0); cudaEventDestroy(e1);
                    plan_free(p); delete p;
                    return s != GRINS_OK ? s : fail(GRINS_E_CUDA, "plan_create: autotune run failed");
                }
                g_last_error.clear();
            }
        }
        // the per-job form: every network's compiled kernel on graph branches
        plan_args(p, 1, 16);
        grins_status s = plan_setup_jobs(p);
        if (s != GRINS_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); plan_free(p); delete p; return s; }
        p->mode = 1;
        cudaEventRecord(e0, st);
        s = plan_enqueue(p, st, true);
        cudaEventRecord(e1, st);
        bool per_job = false;
        float per_job_ms = -1.0f;
        if (s == GRINS_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            std::snprintf(buf, sizeof(buf), "; per-network compiled kernels: %.3f ms", ms);
            tried += buf;
            per_job_ms = ms;
            per_job = best < 0 || ms < best;
        } else if (s != GRINS_E_BUDGET) {
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            plan_free(p); delete p;
            return s != GRINS_OK ? s : fail(GRINS_E_CUDA, "plan_create: autotune run failed");
        }
        g_last_error.clear();
        // one launch of the kernel compiled for every job's layout: blocks of
        // 4 or 2 warps, 8, 12 or 16 resident warps per SM (the register cap
        // of every body; a block size with the same cap reuses the bodies)
        float ct_ms = -1.0f;
        int ct_best = 3, ct_best_w = 4;
        plan_args(p, 1, 16);
        const int ct_cfg[6][2] = {{4, 2}, {4, 3}, {4, 4}, {2, 4}, {2, 6}, {2, 8}};
        for (const auto &cfg : ct_cfg) {
            const int mb = cfg[1];
            p->ct_warps = cfg[0];
            p->ct_minb = mb;
            s = plan_setup_ct(p, st);
            if (s == GRINS_OK) {
                p->mode = 2;
                cudaEventRecord(e0, st);
                s = plan_enqueue(p, st, true);
                cudaEventRecord(e1, st);
                float ms = -1.0f;
                if (s == GRINS_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                    cudaEventElapsedTime(&ms, e0, e1);
                    std::snprintf(buf, sizeof(buf), "; one compiled launch (%d layouts, %d warps x %d blocks per SM): "
                                  "%.3f ms", p->ct_bodies, p->ct_warps, mb, ms);
                    tried += buf;
                    if (ct_ms < 0 || ms < ct_ms) { ct_ms = ms; ct_best = mb; ct_best_w = cfg[0]; }
                }
            }
            if (s != GRINS_OK && s != GRINS_E_BUDGET) {
                cudaEventDestroy(e0); cudaEventDestroy(e1);
                plan_free(p); delete p;
                return s;
            }
            g_last_error.clear();
        }
        p->ct_minb = ct_best;
        p->ct_warps = ct_best_w;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best < 0 && !per_job && ct_ms < 0) { plan_free(p); delete p; return fail(GRINS_E_BUDGET, "plan_create: no configuration fits"); }
        p->mode = per_job ? 1 : 0;
        if (ct_ms >= 0 && (ct_ms < best || best < 0) && (!per_job || ct_ms < per_job_ms)) p->mode = 2;
        p->warps = bw;
        p->slot_extra = bx;
    }
    if (autotune == 2) p->mode = 1;
    if (autotune == 3) p->mode = 2;
    plan_args(p, p->slot_extra, 1);
    grins_status s = plan_setup_branches(p, false);
    if (p->mode == 1 && s == GRINS_OK) s = plan_setup_jobs(p);
    if (p->mode == 2 && s == GRINS_OK) s = plan_setup_ct(p, st);
    if (s == GRINS_OK) s = plan_upload(p, st);
    if (s != GRINS_OK) { plan_free(p); delete p; return s; }

    // capture the plan's work once into a graph
    ce = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) { plan_free(p); delete p; return cuda_fail(ce, "plan_create: graph capture"); }
    s = plan_enqueue(p, p->cap_stream, false);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(p->cap_stream, &g);
    p->graph = g;
    if (s != GRINS_OK) { plan_free(p); delete p; return s; }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (ce != cudaSuccess) { plan_free(p); delete p; return cuda_fail(ce, "plan_create: graph instantiation"); }
    if (p->mode == 2)
        std::snprintf(buf, sizeof(buf), "one persistent launch of a kernel compiled for the jobs' %d register "
                      "layouts, %d jobs, %d warps per block, %d blocks per SM%s", p->ct_bodies, n_jobs, p->ct_warps,
                      p->ct_minb, autotune == 1 ? "; autotuned: " : "");
    else if (p->mode == 1)
        std::snprintf(buf, sizeof(buf), "per-network compiled lane-group DP5(4) kernels, %d jobs on %d graph "
                      "branches%s", n_jobs, (int)p->side.size(), autotune == 1 ? "; autotuned: " : "");
    else
        std::snprintf(buf, sizeof(buf), "batched lane-group DP5(4), %d jobs, %d warps per block, %d extra slots "
                      "per domain, %d-byte warp region%s", n_jobs, p->warps, p->slot_extra, p->batch.warp_bytes,
                      autotune == 1 ? "; autotuned: " : "");
    p->info = buf;
    p->info += tried;
    *out = p;
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_plan_run(grins_racipe_plan_t p, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_plan_run");
    g_last_error.clear();
    if (!p) return fail(GRINS_E_INVALID_ARG, "plan_run: NULL plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return fail(GRINS_E_INVALID_ARG, "plan_run: current device is not the plan's");
    CUDA_TRY(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "plan_run: graph launch");
    return GRINS_OK;
}

extern "C" const char *grins_racipe_plan_info(grins_racipe_plan_t p)
{
    return p ? p->info.c_str() : "";
}

extern "C" grins_status grins_racipe_plan_destroy(grins_racipe_plan_t p)
{
    if (!p) return fail(GRINS_E_INVALID_ARG, "plan_destroy: NULL plan");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    plan_free(p);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
    return GRINS_OK;
}

// ------------------------------------------------------------------ server
// Continuous batching of ensemble requests.  A worker thread admits queued
// requests in arrival order while the in-flight count and the HBM budget
// allow, gives each its own stream, device buffers (from a private
// stream-ordered memory pool) and work counters, and enqueues sample ->
// FP32 integrate -> FP64 polish -> dedupe.  Requests admitted while others
// run execute concurrently (each launch's grid covers only its own work).
// Results stay in device memory until the request is released.
namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerRequest {
    int64_t id = 0;
    grins_racipe *net = nullptr;
    grins_racipe_ranges ranges{};
    // the request's own copies of the tables `ranges` points to (the
    // caller's may be gone by the time the worker samples)
    std::vector<int64_t> sobol_poly, sobol_m;
    std::vector<grins_param_range> param_rows, ic_rows;
    uint64_t seed = 0;
    int64_t n_sets = 0;
    int32_t n_ics = 0;
    grins_solver_opts opts{};
    double dedupe_tol = 1e-2;
    int state = 0;                 // GRINS_REQ_*
    grins_status err = GRINS_OK;
    std::string msg;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t bytes = 0;
    int slot = -1;
    bool jit_wait = false;         // admitted once its compile is done (or jit_max_wait_s passed)
    bool prep = false;             // admitted once the server's prep thread has its class medians
    bool cancel = false;           // grins_racipe_server_cancel was called while it ran
    GrpTopo jit_topo{};
    int jit_kind = 0;
    unsigned char *mem = nullptr;
    unsigned char *params = nullptr;
    double *ic = nullptr, *states = nullptr, *t_final = nullptr;
    uint8_t *status = nullptr;
    float *err_est = nullptr;
    int32_t *n_steps = nullptr, *state_id = nullptr, *n_unique = nullptr;
    unsigned long long *words = nullptr;
    cudaEvent_t done = nullptr;
};

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct grins_racipe_server {
    int device = 0, num_sms = 1, max_inflight = 8;
    int64_t budget = 0, used = 0;
    bool jit = true;
    double jit_min_work = 2e6, jit_max_wait_s = 1.0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<char> slot_busy;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<int64_t> pending;
    std::map<int64_t, std::unique_ptr<ServerRequest>> reqs;
    std::set<grins_racipe *> busy_nets;
    std::thread worker;
    // host preparation off the submitting thread: the half-functional class
    // medians a request's network needs and the cache does not hold yet
    std::thread prep_worker;
    std::deque<int64_t> prep_q;
    std::condition_variable prep_cv;
    bool stop = false;
    int64_t next_id = 1;
    std::string fatal;
    // one cancel flag per in-flight slot, in pinned host memory mapped for
    // the device: the kernels of the slot's request poll it
    volatile int32_t *cancel_host = nullptr;
    const volatile int32_t *cancel_dev = nullptr;
};

namespace {

// Bytes of device memory a request holds from admission to release.
// A request's compiled register-record kernel polls its slot's cancel flag.
int server_variant(int kind) { return kind == kJitShared ? 0 : kJitCancel; }

int64_t request_bytes(const ServerRequest &r)
{
    const int64_t S = r.n_sets, I = r.n_ics, N = r.net->N;
    return align256(S * r.net->layout.stride) + align256(I * N * 8) + align256(S * I * N * 8) +
           align256(S * I) + align256(S * I * 8) + align256(S * I * 4) * 3 + align256(S * 4) + 256;
}

// Enqueues the request's work on its stream (called by the worker with the
// server lock held).
grins_status server_launch(grins_racipe_server *sv, ServerRequest &r)
{
    cudaStream_t st = sv->streams[r.slot];
    const int64_t S = r.n_sets, I = r.n_ics, N = r.net->N;
    CUDA_TRY(dev_malloc_pool(reinterpret_cast<void **>(&r.mem), (size_t)r.bytes, sv->pool, st),
             "server: request buffers");
    unsigned char *q = r.mem;
    auto take = [&](int64_t b) { unsigned char *x = q; q += align256(b); return x; };
    r.params = take(S * r.net->layout.stride);
    r.ic = reinterpret_cast<double *>(take(I * N * 8));
    r.states = reinterpret_cast<double *>(take(S * I * N * 8));
    r.status = take(S * I);
    r.t_final = reinterpret_cast<double *>(take(S * I * 8));
    r.err_est = reinterpret_cast<float *>(take(S * I * 4));
    r.n_steps = reinterpret_cast<int32_t *>(take(S * I * 4));
    r.state_id = reinterpret_cast<int32_t *>(take(S * I * 4));
    r.n_unique = reinterpret_cast<int32_t *>(take(S * 4));
    r.words = reinterpret_cast<unsigned long long *>(take(32));
    grins_status s = grins_racipe_sample_params(r.net, &r.ranges, r.seed, 0, S, I, r.params, r.ic, st);
    if (s != GRINS_OK) return s;
    const grins_racipe *h = r.net;
    const grins_solver_opts *o = &r.opts;
    IntegrateArgs a{};
    a.topo = DevTopo{h->N, h->E, h->d_off, h->d_src, h->d_edge, h->d_sign};
    a.L = h->layout;
    a.params = r.params;
    a.n_sets = S;
    a.ic_unit = r.ic;
    a.n_ics = I;
    a.rtol = o->rtol; a.atol = o->atol; a.t0 = o->t0; a.t_end = o->t_end; a.ss_tol = o->ss_tol;
    set_tighten(&a, o);
    a.max_steps = o->max_steps;
    a.states = r.states; a.status = r.status; a.t_final = r.t_final; a.n_steps = r.n_steps;
    a.queue = r.words;
    a.check = r.words + 2;
    a.slots = slots_for(I);
    a.smem_limit = (int32_t)h->smem_optin;
    a.grp = grp_topo(h);
    a.cancel = sv->cancel_dev + r.slot;       // the slot's flag (reset at admission), not the options' pointer
    if (o->precision == GRINS_FP32) pick_fp32_kernel(h, &a, false, nullptr);   // never compiles here
    else pick_fp64_kernel(h, &a, false, nullptr);
    CUDA_TRY(cudaMemsetAsync(r.words, 0, 32, st), "server: counter reset");
    cudaError_t le = o->precision == GRINS_FP32 ? launch_integrate_fp32(a, st, h->num_sms)
                                                : launch_integrate_fp64(a, st, h->num_sms);
    if (le == cudaErrorInvalidConfiguration)
        return fail(GRINS_E_BUDGET, "server: the network needs more shared memory per block than the device has");
    if (le != cudaSuccess) return cuda_fail(le, "server: integrate launch");
    if (o->polish) {
        PolishArgs pa = polish_args(h, o, r.params, S, I, r.states, r.status, r.err_est);
        pa.check = r.words + 2;
        pa.cancel = a.cancel;
        pa.queue = r.words;                             // the integrate before it on this stream is done with it
        CUDA_TRY(cudaMemsetAsync(pa.queue, 0, sizeof(unsigned long long), st), "server: polish counter");
        CUDA_TRY(launch_polish(pa, st, h->num_sms), "server: polish launch");
    } else {
        CUDA_TRY(cudaMemsetAsync(r.err_est, 0xff, sizeof(float) * S * I, st), "server: err_est");
    }
    s = grins_racipe_unique_states(r.net, r.params, r.states, r.status, S, I, r.dedupe_tol, r.state_id,
                                   r.n_unique, st);
    if (s != GRINS_OK) return s;
    CUDA_TRY(cudaEventRecord(r.done, st), "server: completion event");
    return GRINS_OK;
}

void server_loop(grins_racipe_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        bool progress = false;
        // completions
        for (auto &kv : sv->reqs) {
            ServerRequest &r = *kv.second;
            if (r.state != GRINS_REQ_RUNNING) continue;
            const cudaError_t q = cudaEventQuery(r.done);
            if (q == cudaErrorNotReady) continue;
            r.t_done = now_s();
            r.state = q == cudaSuccess ? (r.cancel ? GRINS_REQ_CANCELLED : GRINS_REQ_DONE) : GRINS_REQ_FAILED;
            if (q != cudaSuccess) { r.err = GRINS_E_CUDA; r.msg = cudaGetErrorString(q); }
            else if (r.cancel) { r.err = GRINS_E_CANCELLED; r.msg = "cancelled while running"; }
            sv->slot_busy[r.slot] = 0;
            sv->busy_nets.erase(r.net);
            progress = true;
        }
        if (progress) sv->cv_done.notify_all();
        // admissions, in arrival order; a request whose network is busy with
        // an earlier request waits without blocking the others
        for (auto it = sv->pending.begin(); it != sv->pending.end();) {
            ServerRequest &r = *sv->reqs[*it];
            int slot = -1;
            for (int i = 0; i < sv->max_inflight && slot < 0; ++i)
                if (!sv->slot_busy[i]) slot = i;
            if (slot < 0) break;
            if (sv->busy_nets.count(r.net)) { ++it; continue; }
            if (r.prep) { ++it; continue; }
            if (r.jit_wait) {
                if (grp_jit_prefetch(r.jit_topo, r.jit_kind, server_variant(r.jit_kind)) == 0 &&
                    now_s() - r.t_submit < sv->jit_max_wait_s) {
                    ++it;
                    continue;
                }
                r.jit_wait = false;
            }
            if (sv->used + r.bytes > sv->budget && sv->used > 0) break;   // head waits for memory
            r.slot = slot;
            sv->slot_busy[slot] = 1;
            sv->busy_nets.insert(r.net);
            sv->used += r.bytes;
            r.t_admit = now_s();
            r.state = GRINS_REQ_RUNNING;
            sv->cancel_host[slot] = 0;                // a cancel from here on reaches the kernels
            sv->pending.erase(it);
            // the launch sequence runs without the lock: a CUDA call can
            // stall behind other threads' driver work, and submissions,
            // waits and cancels must not wait for it (a running request
            // cannot be released, and only this thread admits or completes)
            lock.unlock();
            cudaSetDevice(r.net->device);
            grins_status s = GRINS_OK;
            if (cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess)
                s = fail(GRINS_E_CUDA, "server: completion event");
            if (s == GRINS_OK) s = server_launch(sv, r);
            const std::string msg = s != GRINS_OK ? std::string(grins_last_error()) : std::string();
            lock.lock();
            if (s != GRINS_OK) {
                r.state = GRINS_REQ_FAILED;
                r.err = s;
                r.msg = msg;
                r.t_done = now_s();
                sv->slot_busy[slot] = 0;
                sv->busy_nets.erase(r.net);
                sv->cv_done.notify_all();
            }
            progress = true;
            it = sv->pending.begin();                 // others may have queued meanwhile
        }
        if (!progress) sv->cv.wait_for(lock, std::chrono::microseconds(100));
    }
}

// The prep thread: computes the missing class medians of queued requests,
// one request at a time (the classes of one in parallel), then lets the
// worker admit it.
void server_prep_loop(grins_racipe_server *sv)
{
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        if (sv->prep_q.empty()) {
            sv->prep_cv.wait(lock);
            continue;
        }
        const int64_t id = sv->prep_q.front();
        sv->prep_q.pop_front();
        auto it = sv->reqs.find(id);
        if (it == sv->reqs.end() || !it->second->prep) continue;
        grins_racipe *net = it->second->net;
        const grins_racipe_ranges rr = it->second->ranges;
        lock.unlock();
        warm_class_medians(net, rr);
        lock.lock();
        auto jt = sv->reqs.find(id);
        if (jt != sv->reqs.end()) jt->second->prep = false;
        sv->cv.notify_all();
    }
}

}  // namespace

extern "C" void grins_server_default_config(grins_server_config *c)
{
    if (!c) return;
    c->max_inflight = 8;
    c->hbm_budget_bytes = (int64_t)32 << 30;
    c->jit = 1;
    c->jit_min_work = 2e6;
    c->jit_max_wait_s = 1.0;
}

extern "C" grins_status grins_racipe_server_create(const grins_server_config *c, grins_racipe_server_t *out)
{
    g_last_error.clear();
    if (!out) return fail(GRINS_E_INVALID_ARG, "server_create: out is NULL");
    *out = nullptr;
    grins_server_config cfg;
    if (c) cfg = *c; else grins_server_default_config(&cfg);
    if (cfg.max_inflight < 1 || cfg.max_inflight > 64 || cfg.hbm_budget_bytes <= 0)
        return fail(GRINS_E_INVALID_ARG, "server_create: need 1 <= max_inflight <= 64 and a positive budget");
    if (!(cfg.jit_min_work >= 0) || !(cfg.jit_max_wait_s >= 0))
        return fail(GRINS_E_INVALID_ARG, "server_create: jit_min_work and jit_max_wait_s must be >= 0");
    auto sv = std::unique_ptr<grins_racipe_server>(new (std::nothrow) grins_racipe_server());
    if (!sv) return fail(GRINS_E_NOMEM, "server_create: host allocation failed");
    CUDA_TRY(cudaGetDevice(&sv->device), "server_create: current device");
    CUDA_TRY(cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device), "server_create");
    sv->max_inflight = cfg.max_inflight;
    sv->budget = cfg.hbm_budget_bytes;
    sv->jit = cfg.jit != 0;
    sv->jit_min_work = cfg.jit_min_work;
    sv->jit_max_wait_s = cfg.jit_max_wait_s;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = sv->device;
    CUDA_TRY(cudaMemPoolCreate(&sv->pool, &props), "server_create: memory pool");
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    sv->streams.assign(sv->max_inflight, nullptr);
    sv->slot_busy.assign(sv->max_inflight, 0);
    for (auto &st : sv->streams) {
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto &x : sv->streams) if (x) cudaStreamDestroy(x);
            cudaMemPoolDestroy(sv->pool);
            return cuda_fail(e, "server_create: streams");
        }
    }
    {
        int32_t *hf = nullptr;
        void *df = nullptr;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&hf), sizeof(int32_t) * sv->max_inflight,
                                      cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&df, hf, 0);
        if (e != cudaSuccess) {
            if (hf) cudaFreeHost(hf);
            for (auto &x : sv->streams) cudaStreamDestroy(x);
            cudaMemPoolDestroy(sv->pool);
            return cuda_fail(e, "server_create: cancel flags");
        }
        for (int i = 0; i < sv->max_inflight; ++i) hf[i] = 0;
        sv->cancel_host = hf;
        sv->cancel_dev = static_cast<const volatile int32_t *>(df);
    }
    grins_racipe_server *raw = sv.release();
    raw->worker = std::thread(server_loop, raw);
    raw->prep_worker = std::thread(server_prep_loop, raw);
    *out = raw;
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_server_submit(grins_racipe_server_t sv, grins_racipe_t net,
                                                   const grins_racipe_ranges *r, uint64_t seed, int64_t n_sets,
                                                   int32_t n_ics, const grins_solver_opts *o, double dedupe_tol,
                                                   int64_t *request_id)
{
    AbiRange nvtx_range_("grins_racipe_server_submit");
    g_last_error.clear();
    if (!sv || !net || !o || !request_id) return fail(GRINS_E_INVALID_ARG, "server_submit: NULL argument");
    if (n_sets < 1 || n_ics < 1 || n_ics > 4096) return fail(GRINS_E_INVALID_ARG, "server_submit: bad sizes");
    if (net->device != sv->device) return fail(GRINS_E_INVALID_ARG, "server_submit: network on another device");
    if (o->n_t != 0) return fail(GRINS_E_INVALID_ARG, "server_submit: requests do not write time series");
    if (o->precision != GRINS_FP32 && o->precision != GRINS_FP64)
        return fail(GRINS_E_INVALID_ARG, "server_submit: unknown precision");
    if (!(o->rtol > 0) || !(o->atol > 0) || !(o->t_end > o->t0) || o->max_steps < 1 || !(o->ss_tol >= 0) ||
        !(o->ss_tighten > 0 && o->ss_tighten <= 1) ||
        (o->polish && !polish_opts_ok(o)))
        return fail(GRINS_E_INVALID_ARG, "server_submit: bad solver options");
    if (o->method != GRINS_METHOD_DOPRI5)
        return fail(GRINS_E_INVALID_ARG, "server_submit: the server runs Dormand-Prince only");
    if (!(dedupe_tol >= 0)) return fail(GRINS_E_INVALID_ARG, "server_submit: dedupe_tol < 0");
    grins_racipe_ranges rr;
    if (r) rr = *r; else grins_racipe_default_ranges(&rr);
    grins_status s = check_ranges(rr);
    if (s != GRINS_OK) return s;
    // the half-functional median table is host work.  Class medians the
    // process-wide cache lacks (tens of milliseconds per class) are computed
    // by the server's prep thread, and the request waits in the queue for
    // them; otherwise (all cached, or a per-parameter table, whose rows are
    // checked here) the table is filled in this thread -- in microseconds
    // when cached
    const bool prep = !rr.param_ranges && !missing_classes(net, rr).empty();
    if (!prep) {
        std::lock_guard<std::mutex> lock(net->median_mu);
        s = ensure_medians(net, rr);
    }
    if (s != GRINS_OK) return s;
    auto req = std::unique_ptr<ServerRequest>(new (std::nothrow) ServerRequest());
    if (!req) return fail(GRINS_E_NOMEM, "server_submit: host allocation failed");
    req->net = net; req->ranges = rr; req->seed = seed; req->n_sets = n_sets; req->n_ics = n_ics;
    if (rr.sobol != GRINS_SOBOL_OFF && rr.sobol_poly && rr.sobol_m && rr.sobol_dims > 0 && rr.sobol_m_cols > 0) {
        req->sobol_poly.assign(rr.sobol_poly, rr.sobol_poly + rr.sobol_dims);
        req->sobol_m.assign(rr.sobol_m, rr.sobol_m + (size_t)rr.sobol_dims * (size_t)rr.sobol_m_cols);
        req->ranges.sobol_poly = req->sobol_poly.data();
        req->ranges.sobol_m = req->sobol_m.data();
    }
    if (rr.param_ranges) {
        req->param_rows.assign(rr.param_ranges, rr.param_ranges + 2 * net->N + 3 * net->E);
        req->ranges.param_ranges = req->param_rows.data();
    }
    if (rr.ic_ranges) {
        req->ic_rows.assign(rr.ic_ranges, rr.ic_ranges + net->N);
        req->ranges.ic_ranges = req->ic_rows.data();
    }
    req->opts = *o; req->dedupe_tol = dedupe_tol;
    req->bytes = request_bytes(*req);
    if (req->bytes > sv->budget)
        return fail(GRINS_E_BUDGET, "server_submit: the request needs %lld bytes, above the %lld-byte budget",
                    (long long)req->bytes, (long long)sv->budget);
    // large FP32 requests start the compile of their network's integrator
    // now, so that it overlaps the queueing; the worker admits them once it
    // is done (the kernel the integrate call would pick: records in
    // registers when that layout exists, else records in shared memory)
    if (sv->jit && (double)n_sets * n_ics * std::max(net->E, 1) >= sv->jit_min_work) {
        const char *ev = std::getenv("GRINS_JIT_KIND");
        const bool want_shared = ev && std::string(ev) == "grp";
        if (o->precision == GRINS_FP64) {
            if (net->rr.L > 0) { req->jit_topo = net->rr.topo(); req->jit_kind = kJitRegisters64; }
        } else if (!want_shared && net->rr.L > 0) {
            req->jit_topo = net->rr.topo(); req->jit_kind = kJitRegisters;
        } else {
            req->jit_topo = net->grp.topo(); req->jit_kind = kJitShared;
        }
        req->jit_wait = grp_jit_prefetch(req->jit_topo, req->jit_kind, server_variant(req->jit_kind)) == 0;
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    req->id = sv->next_id++;
    req->t_submit = now_s();
    req->state = GRINS_REQ_QUEUED;
    req->prep = prep;
    *request_id = req->id;
    sv->pending.push_back(req->id);
    if (prep) {
        sv->prep_q.push_back(req->id);
        sv->prep_cv.notify_one();
    }
    sv->reqs.emplace(req->id, std::move(req));
    sv->cv.notify_all();
    return GRINS_OK;
}

static void fill_info(const ServerRequest &r, grins_request_info *info)
{
    info->state = r.state;
    info->error = r.err;
    info->n_sets = r.n_sets;
    info->n_ics = r.n_ics;
    info->bytes = r.bytes;
    const double t_out = r.t_admit > 0 ? r.t_admit : (r.state >= GRINS_REQ_DONE ? r.t_done : now_s());
    info->queued_s = t_out - r.t_submit;
    info->latency_s = r.state >= GRINS_REQ_DONE ? r.t_done - r.t_submit : -1.0;
}

extern "C" grins_status grins_racipe_server_wait(grins_racipe_server_t sv, int64_t id, double timeout_s,
                                                 grins_request_info *info)
{
    g_last_error.clear();
    if (!sv) return fail(GRINS_E_INVALID_ARG, "server_wait: NULL server");
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return fail(GRINS_E_INVALID_ARG, "server_wait: unknown request %lld", (long long)id);
    ServerRequest &r = *it->second;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((long long)(std::max(0.0, timeout_s) * 1e6));
    while (r.state < GRINS_REQ_DONE) {
        if (timeout_s >= 0 && sv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) break;
        if (timeout_s < 0) sv->cv_done.wait(lock);
    }
    if (info) fill_info(r, info);
    if (r.state == GRINS_REQ_FAILED)
        return fail(r.err, "server_wait: request %lld failed: %s", (long long)id, r.msg.c_str());
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_server_copy_results(grins_racipe_server_t sv, int64_t id, double *d_states,
                                                         uint8_t *d_status, int32_t *d_n_unique,
                                                         int32_t *d_state_id, int32_t *d_n_steps, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_server_copy_results");
    g_last_error.clear();
    if (!sv) return fail(GRINS_E_INVALID_ARG, "server_copy_results: NULL server");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return fail(GRINS_E_INVALID_ARG, "server_copy_results: unknown request");
    ServerRequest &r = *it->second;
    if (r.state != GRINS_REQ_DONE && !(r.state == GRINS_REQ_CANCELLED && r.mem))
        return fail(GRINS_E_INVALID_ARG, "server_copy_results: request not done (or cancelled before it ran)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t S = r.n_sets, I = r.n_ics, N = r.net->N;
    if (d_states) CUDA_TRY(cudaMemcpyAsync(d_states, r.states, S * I * N * 8, cudaMemcpyDeviceToDevice, st), "copy");
    if (d_status) CUDA_TRY(cudaMemcpyAsync(d_status, r.status, S * I, cudaMemcpyDeviceToDevice, st), "copy");
    if (d_n_unique) CUDA_TRY(cudaMemcpyAsync(d_n_unique, r.n_unique, S * 4, cudaMemcpyDeviceToDevice, st), "copy");
    if (d_state_id) CUDA_TRY(cudaMemcpyAsync(d_state_id, r.state_id, S * I * 4, cudaMemcpyDeviceToDevice, st), "copy");
    if (d_n_steps) CUDA_TRY(cudaMemcpyAsync(d_n_steps, r.n_steps, S * I * 4, cudaMemcpyDeviceToDevice, st), "copy");
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_server_cancel(grins_racipe_server_t sv, int64_t id)
{
    g_last_error.clear();
    if (!sv) return fail(GRINS_E_INVALID_ARG, "server_cancel: NULL server");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return fail(GRINS_E_INVALID_ARG, "server_cancel: unknown request");
    ServerRequest &r = *it->second;
    if (r.state == GRINS_REQ_QUEUED) {
        // never admitted: no buffers, no slot
        for (auto p = sv->pending.begin(); p != sv->pending.end(); ++p)
            if (*p == id) { sv->pending.erase(p); break; }
        r.state = GRINS_REQ_CANCELLED;
        r.err = GRINS_E_CANCELLED;
        r.msg = "cancelled before it ran";
        r.t_done = now_s();
        sv->cv_done.notify_all();
        sv->cv.notify_all();
    } else if (r.state == GRINS_REQ_RUNNING && !r.cancel) {
        r.cancel = true;
        sv->cancel_host[r.slot] = 1;            // the slot's kernels stop taking work
    }
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_server_release(grins_racipe_server_t sv, int64_t id)
{
    g_last_error.clear();
    if (!sv) return fail(GRINS_E_INVALID_ARG, "server_release: NULL server");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return fail(GRINS_E_INVALID_ARG, "server_release: unknown request");
    ServerRequest &r = *it->second;
    if (r.state == GRINS_REQ_QUEUED || r.state == GRINS_REQ_RUNNING)
        return fail(GRINS_E_INVALID_ARG, "server_release: request %lld is not finished", (long long)id);
    if (r.mem) {
        cudaFreeAsync(r.mem, sv->streams[r.slot]);
        sv->used -= r.bytes;
    }
    if (r.done) cudaEventDestroy(r.done);
    sv->reqs.erase(it);
    sv->cv.notify_all();
    return GRINS_OK;
}

extern "C" grins_status grins_racipe_server_destroy(grins_racipe_server_t sv)
{
    if (!sv) return fail(GRINS_E_INVALID_ARG, "server_destroy: NULL server");
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
        sv->prep_cv.notify_all();
    }
    sv->worker.join();
    sv->prep_worker.join();
    cudaSetDevice(sv->device);
    for (auto &st : sv->streams) cudaStreamSynchronize(st);
    for (auto &kv : sv->reqs) {
        if (kv.second->mem) cudaFreeAsync(kv.second->mem, sv->streams[kv.second->slot]);
        if (kv.second->done) cudaEventDestroy(kv.second->done);
    }
    for (auto &st : sv->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    cudaMemPoolDestroy(sv->pool);
    cudaFreeHost(const_cast<int32_t *>(sv->cancel_host));
    delete sv;
    return GRINS_OK;
}

#ifdef GRINS_CHECKED
// Checked builds only: first index/alignment violation recorded by the
// handle's kernels (0 = none); *info receives the offending index.
extern "C" int grins_debug_check_status(grins_racipe_t h, long long *info)
{
    unsigned long long w[2] = {0, 0};
    if (!h || cudaMemcpy(w, h->d_queue + 2, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (info) *info = (long long)w[1];
    return (int)w[0];
}
#endif

// ------------------------------------------------- integrate, no allocation
// grins_racipe_integrate_static: the integrate entry point for callers that
// cannot allocate device memory.  Its scratch -- the work-queue counter, the
// check words and the device copy of the time grid -- lives in the fixed
// array below instead of the handle's workspace, and nothing is allocated
// per call.  Every device that loads the library holds this array until the
// process exits.
namespace {

// Words at the head of the array: 0 the work-queue counter, 1 reserved (kept
// zero; the check words sit at a fixed offset), 2-3 the first index/alignment
// violation of a checked build (code, offending index).
constexpr int kStaticWords = 4;
constexpr size_t kStaticBytes = kStaticWords * sizeof(unsigned long long) +
                                (size_t)GRINS_STATIC_MAX_GRID * sizeof(double);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
struct StaticAddr {
    unsigned long long ctx_id = 0;     // the context the address belongs to (0: not looked up)
    unsigned char *addr = nullptr;
};
StaticAddr g_static_addr[kStaticMaxDevices];

// Unique id of the current CUDA context (cuCtxGetId through the runtime's
// driver entry points; ids are never reused within a process), so that the
// address looked up in a context is not used in a later one, for example
// after cudaDeviceReset.  0 when the driver cannot say.
unsigned long long current_context_id()
{
    using GetCur = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of g_static_scratch on the current device, looked up once
// per device and context (host code must not use the symbol itself: it
// names a host-side shadow, not device memory).  The first lookup in a
// context may load the library's device code there (lazy module loading).
grins_status static_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kStaticMaxDevices)
        return fail(GRINS_E_INVALID_ARG, "integrate_static: device %d outside [0, %d)", device, kStaticMaxDevices);
    // the handle's allocations already made this device's context current;
    // with no context id (0) the address is looked up again on every call
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticAddr &a = g_static_addr[device];
    if (!a.addr || ctx == 0 || a.ctx_id != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "integrate_static: cudaGetSymbolAddress");
        a.addr = static_cast<unsigned char *>(p);
        a.ctx_id = ctx;
    }
    *out = a.addr;
    return GRINS_OK;
}

}  // namespace

#ifdef GRINS_CHECKED
// Checked builds only: the first index/alignment violation recorded by a
// grins_racipe_integrate_static call on the current device (its kernels
// write their check words into the static array, not the handle's).
extern "C" int grins_debug_static_check_status(long long *info)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    unsigned char *scratch = nullptr;
    if (static_scratch(dev, &scratch) != GRINS_OK) return -1;
    unsigned long long w[2] = {0, 0};
    if (cudaMemcpy(w, scratch + 2 * sizeof(unsigned long long), sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    if (info) *info = (long long)w[1];
    return (int)w[0];
}
#endif

extern "C" grins_status grins_racipe_integrate_static(grins_racipe_t h, const grins_solver_opts *o,
                                                      const void *d_params, int64_t n_sets,
                                                      const double *d_ic_unit, int32_t n_ics,
                                                      double *d_states, uint8_t *d_status,
                                                      double *d_t_final, float *d_err_est,
                                                      int32_t *d_n_steps, double *d_series, void *stream)
{
    AbiRange nvtx_range_("grins_racipe_integrate_static");
    g_last_error.clear();
    if (!h || !o) return fail(GRINS_E_INVALID_ARG, "integrate_static: NULL handle or options");
    if (n_sets < 0) return fail(GRINS_E_INVALID_ARG, "integrate_static: n_sets < 0");
    if (n_ics < 1) return fail(GRINS_E_INVALID_ARG, "integrate_static: n_ics < 1");
    if (n_sets > 0 && (!d_params || !d_ic_unit || !d_states || !d_status))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: NULL required device buffer");
    if (o->precision != GRINS_FP32 && o->precision != GRINS_FP64)
        return fail(GRINS_E_INVALID_ARG, "integrate_static: unknown precision %d", o->precision);
    if (!(o->rtol > 0) || !(o->atol > 0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: rtol and atol must be positive");
    if (!std::isfinite(o->t0) || !std::isfinite(o->t_end) || !(o->t_end > o->t0))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: need finite t0 < t_end");
    if (!(o->ss_tol >= 0)) return fail(GRINS_E_INVALID_ARG, "integrate_static: ss_tol < 0");
    if (!(o->ss_tighten > 0 && o->ss_tighten <= 1))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: need 0 < ss_tighten <= 1");
    if (o->method != GRINS_METHOD_DOPRI5 && o->method != GRINS_METHOD_TSIT5)
        return fail(GRINS_E_INVALID_ARG, "integrate_static: unknown method %d", o->method);
    if (o->max_steps < 1) return fail(GRINS_E_INVALID_ARG, "integrate_static: max_steps < 1");
    if (o->n_t < 0 || (o->n_t > 0 && !o->t_grid))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: bad time grid");
    if (o->n_t > GRINS_STATIC_MAX_GRID)
        return fail(GRINS_E_BUDGET, "integrate_static: n_t = %d exceeds the fixed scratch limit of %d grid times",
                    o->n_t, GRINS_STATIC_MAX_GRID);
    if ((o->n_t > 0) != (d_series != nullptr) && n_sets > 0)
        return fail(GRINS_E_INVALID_ARG, "integrate_static: d_series must be given exactly when n_t > 0");
    for (int g = 0; g < o->n_t; ++g) {
        const double tg = o->t_grid[g];
        if (!(tg >= o->t0 && tg <= o->t_end) || (g > 0 && !(tg > o->t_grid[g - 1])))
            return fail(GRINS_E_INVALID_ARG, "integrate_static: t_grid must increase strictly inside [t0, t_end]");
    }
    if (o->polish && !polish_opts_ok(o))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: bad polish options");
    if (!on_handle_device(h))
        return fail(GRINS_E_INVALID_ARG, "integrate_static: current device is not the handle's");
    unsigned char *scratch = nullptr;
    grins_status s = static_scratch(h->device, &scratch);
    if (s != GRINS_OK) return s;
    if (n_sets == 0) return GRINS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *words = reinterpret_cast<unsigned long long *>(scratch);
    double *grid = reinterpret_cast<double *>(scratch + kStaticWords * sizeof(unsigned long long));
    if (o->n_t > 0) {
        CUDA_TRY(cudaMemcpyAsync(grid, o->t_grid, sizeof(double) * o->n_t, cudaMemcpyHostToDevice, st),
                 "integrate_static: grid upload");
    }

    IntegrateArgs a{};
    a.topo = DevTopo{h->N, h->E, h->d_off, h->d_src, h->d_edge, h->d_sign};
    a.L = h->layout;
    a.params = static_cast<const unsigned char *>(d_params);
    a.n_sets = n_sets;
    a.ic_unit = d_ic_unit;
    a.n_ics = n_ics;
    a.rtol = o->rtol; a.atol = o->atol; a.t0 = o->t0; a.t_end = o->t_end; a.ss_tol = o->ss_tol;
    set_tighten(&a, o);
    a.max_steps = o->max_steps;
    a.t_grid = grid;
    a.n_t = o->n_t;
    a.states = d_states; a.status = d_status; a.t_final = d_t_final; a.n_steps = d_n_steps;
    a.series = o->n_t > 0 ? d_series : nullptr;
    a.queue = words;
    a.check = words + 2;
    a.slots = slots_for(n_ics);
    a.smem_limit = (int32_t)h->smem_optin;
    a.grp = grp_topo(h);
    a.cancel = o->cancel;
    if (o->precision == GRINS_FP32) pick_fp32_kernel(h, &a, false, nullptr);   // only kernels an earlier call loaded
    else pick_fp64_kernel(h, &a, false, nullptr);
    if (a.method != GRINS_METHOD_DOPRI5 && !a.grp_jit)
        return fail(GRINS_E_INVALID_ARG, "integrate_static: the Tsitouras pair needs the network's compiled kernel, "
                    "loaded by an earlier grins_racipe_integrate call");

    // the array keeps the previous call's counters: clear them first
    CUDA_TRY(cudaMemsetAsync(words, 0, kStaticWords * sizeof(unsigned long long), st),
             "integrate_static: scratch reset");
    cudaError_t le;
    if (o->precision == GRINS_FP32) le = launch_integrate_fp32(a, st, h->num_sms);
    else le = launch_integrate_fp64(a, st, h->num_sms);
    if (le == cudaErrorInvalidConfiguration)
        return fail(GRINS_E_BUDGET, "integrate_static: the network needs more shared memory per block than the device has");
    if (le != cudaSuccess) return cuda_fail(le, "integrate_static: launch");

    if (o->polish) {
        PolishArgs p = polish_args(h, o, d_params, n_sets, n_ics, d_states, d_status, d_err_est);
        p.check = words + 2;
        CUDA_TRY(launch_polish(p, st, h->num_sms), "integrate_static: polish launch");
    } else if (d_err_est) {
        CUDA_TRY(cudaMemsetAsync(d_err_est, 0xff, sizeof(float) * n_sets * n_ics, st), "integrate_static: err_est");
    }
    return GRINS_OK;
}
