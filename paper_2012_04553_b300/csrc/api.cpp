// C ABI (include/pm.h): argument checking, plan ownership, device buffers,
// the plan-family autotuner, launches and the host half of the morph
// transform.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.hpp"

namespace pm {

pm_status build_graph(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                      const uint8_t *labels, int device, void *stream, pm_graph **out);
pm_status prepare_csr(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                      int64_t *rowptr, int32_t *col, int32_t *new_id, int64_t *lowdeg);

namespace {
thread_local std::string g_last_error;
std::mutex g_alloc_mu;
pm_alloc_fn g_alloc = nullptr;
pm_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

// Host-side fault injection (environment variable PM_FAULT, read at each
// call): "alloc" fails every device allocation, "load" every graph load,
// "plan" every plan, so error paths are exercised without a GPU fault.
bool fault_injected(const char *what) {
    const char *f = std::getenv("PM_FAULT");
    return f && std::strcmp(f, what) == 0;
}

void *dev_alloc(size_t bytes, int device) {
    if (fault_injected("alloc")) return nullptr;
    if (bytes == 0) bytes = 256;
    pm_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (a) return a(bytes, device, ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *ptr, size_t bytes, int device) {
    if (!ptr) return;
    if (bytes == 0) bytes = 256;
    pm_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f) f(ptr, bytes, device, ctx);
    else cudaFree(ptr);
}

}  // namespace pm

using namespace pm;

namespace {

// A device copy of a list of plans.
struct PlanTable {
    std::vector<DevPlan> plans;
    DevPlan *d = nullptr;
    size_t cap = 0;         // plans the device buffer holds
    int max_enum = 2;
    bool dirty = true;
};

}  // namespace

struct pm_query_plan {
    const pm_graph *g = nullptr;
    pm_op op = PM_OP_COUNT;
    MorphPlan morph;
    // per matched pattern: its rooted plans [rooted_begin[j], rooted_begin[j+1])
    // and its free plan free_plans[j]
    std::vector<DevPlan> rooted;
    std::vector<int> rooted_begin;
    std::vector<DevPlan> free_plans;
    std::vector<int> choice;        // per matched pattern: 0 rooted, 1 free, -1 undecided
    std::vector<int> split_code;    // per matched pattern: task granularity (0: split / 4, 1: as compiled, 2: x 4)
    int forced = -1;                // pm_plan_select: -1 = autotuned per pattern
    int launch_mode = PM_LAUNCH_PER_PATTERN;
    PlanTable active;               // pm_count / pm_support
    PlanTable rooted_table;         // pm_count_roots
    uint64_t *d_counters = nullptr;
    Control *d_ctl = nullptr;
    // MNI
    int n_bitsets = 0;
    int64_t words = 0;
    uint32_t *d_bitsets = nullptr;
    std::vector<int32_t> col_off, col_src;   // per query column: sources (bitset ids)
    std::vector<int> query_col_base;         // first query column of each query
    int32_t *d_col_off = nullptr, *d_col_src = nullptr;
    unsigned long long *d_popc = nullptr;
    std::vector<int> dom_base;               // per matched pattern
    Deferred *d_defer = nullptr;             // deferred-chunk list and its piece scan
    uint32_t *d_piece_off = nullptr;
    uint32_t defer_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the last matching launch
    bool timed = false;
    // per matched pattern: events around its launch sequence in the last
    // pm_count (per-pattern launch mode), and whether they were recorded
    std::vector<cudaEvent_t> pat_ev;
    std::vector<char> pat_recorded;
    int64_t launches = 0;                    // library kernels launched by the last count
    std::vector<uint64_t> pat_bytes;         // algorithmic bytes per matched pattern (instrumented count)
    unsigned long long *d_stats = nullptr;
    uint8_t *d_timed_out = nullptr;          // pm_count_each: expired matched patterns
    uint32_t *d_wedge = nullptr;             // wedge-kernel counters: blocks x n, kept zero
    int wedge_nblocks = 0;
    uint2 *d_lists = nullptr;                // heavy-root wedge kernel: entry lists
    int64_t list_cap = 0, heavy_from = 0;
    size_t bytes_lists = 0;
    bool wedge_ready = false;
    unsigned int *d_plan_done = nullptr;     // per-plan progress (single launch, per-pattern deadlines)
    size_t plan_done_cap = 0;
    cudaGraphExec_t graph_each = nullptr;    // pm_plan_capture_each: pm_count_each as a CUDA graph
    int32_t *d_spill = nullptr;              // clique-kernel spill sets (per warp)
    int64_t spill_len = 0;
    size_t bytes_counters = 0, bytes_bitsets = 0, bytes_cols = 0, bytes_wedge = 0, bytes_spill = 0;
    bool spill_ready = false;
    bool device_ready = false;
    // decomposition kernels (decomp.cu): formula of each matched pattern
    // (-1: none), the active (formula, counter) pairs and their passes
    std::vector<int> decomp_f;
    std::vector<int32_t> decomp_targets;
    int decomp_passes_active = 0;
    int32_t *d_targets = nullptr;
    size_t bytes_targets = 0;
    int32_t *d_tslot = nullptr;              // triangle count per CSR slot
    size_t bytes_tslot = 0;
    uint32_t *d_dW = nullptr;                // 2-path counters (path blocks x n, kept zero)
    int32_t *d_dtouched = nullptr;
    size_t bytes_dW = 0;
    int dpath_blocks = 0;
    uint64_t *d_basis = nullptr;
    uint32_t *d_k4e = nullptr;               // 4-cliques per edge (CSR slot of the lower endpoint)
    size_t bytes_k4e = 0;
    uint32_t *d_local = nullptr;             // neighbourhood bitmap overflow (large out-degrees)
    size_t bytes_local = 0;
    int local_blocks = 0;
    bool local_ready = false;
    // neighbourhood-graph pass (wheel.cu): list offsets, common-neighbour
    // lists, scan scratch, hub rank index, mirror positions, counters
    struct {
        int64_t *toff = nullptr;
        int32_t *T = nullptr;
        int64_t *bsum = nullptr;
        int32_t *rank = nullptr;
        int32_t *mpos = nullptr;
        uint32_t *gcnt = nullptr;
        uint32_t *kW = nullptr;
        unsigned long long *kE = nullptr;
        int32_t *ktouched = nullptr;
        size_t b_toff = 0, b_T = 0, b_bsum = 0, b_rank = 0, b_mpos = 0, b_gcnt = 0, b_kW = 0, b_kE = 0;
        int64_t gcnt_words = 0;
        int w4_blocks = 0, k23_blocks = 0;
        uint32_t *k5g = nullptr;
        size_t b_k5g = 0;
        int64_t k5g_words = 0;
        int k5e_blocks = 0;
    } wh;
    // CUDA graph of a whole pm_count (pm_plan_capture): replayed by pm_count
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t *h_pinned = nullptr;            // counters (2 per matched) then the Control block
};

namespace {

// A kernel set the control block's fault word: 1 = common-neighbour lists
// whose lengths differ from the per-edge triangle counts, 2 = an index out
// of range caught by the PM_DEBUG build's bounds checks (the access was
// skipped).  Both are internal errors; the results are not returned.
pm_status list_fault(const char *who, int fault) {
    set_error(std::string(who) + (fault == 2 ? ": a kernel bounds check failed (PM_DEBUG build)"
                                             : ": common-neighbour lists disagree with the per-edge triangle counts"));
    return PM_ECUDA;
}

void free_wheel(pm_query_plan *p, int dev) {
    auto &w = p->wh;
    dev_free(w.toff, w.b_toff, dev);
    dev_free(w.T, w.b_T, dev);
    dev_free(w.bsum, w.b_bsum, dev);
    dev_free(w.rank, w.b_rank, dev);
    dev_free(w.mpos, w.b_mpos, dev);
    dev_free(w.gcnt, w.b_gcnt, dev);
    dev_free(w.kW, w.b_kW, dev);
    dev_free(w.kE, w.b_kE, dev);
    dev_free(w.ktouched, w.b_kW, dev);
    dev_free(w.k5g, w.b_k5g, dev);
    p->wh = {};
}

struct DeviceGuard {
    int prev = 0;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        ok = cudaSetDevice(dev) == cudaSuccess;
        // a failed runtime call made earlier on this thread (outside this
        // call) must not be read back as this call's launch error
        if (ok) cudaGetLastError();
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

pm_status cuda_fail(const char *what, cudaError_t e) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return PM_ECUDA;
}

pm_status to_pat(const pm_pattern &q, bool graph_labeled, Pat *out) {
    if (q.k < 2 || q.k > PM_MAX_K) {
        set_error("pattern: k must be in [2, 8]");
        return PM_EINVAL;
    }
    const int npairs = q.k * (q.k - 1) / 2;
    if (npairs < 32 && (q.edge_mask >> npairs)) {
        set_error("pattern: edge_mask has bits beyond the k*(k-1)/2 pairs");
        return PM_EINVAL;
    }
    if (q.induced != PM_EDGE_INDUCED && q.induced != PM_VERTEX_INDUCED) {
        set_error("pattern: induced must be PM_EDGE_INDUCED or PM_VERTEX_INDUCED");
        return PM_EINVAL;
    }
    for (int u = 0; u < q.k; u++) {
        if (q.label[u] < -1) {
            set_error("pattern: label must be -1 (any) or a label value in [0, 127]");
            return PM_EINVAL;
        }
    }
    Pat p = Pat::from_mask(q.k, q.edge_mask, q.label, q.induced == PM_VERTEX_INDUCED);
    if (!p.connected()) {
        set_error("pattern: not connected (Section 2 requires connected patterns)");
        return PM_EINVAL;
    }
    if (p.labeled() && !graph_labeled) {
        set_error("pattern: labeled pattern on an unlabeled graph");
        return PM_EINVAL;
    }
    *out = p;
    return PM_OK;
}

void free_table(PlanTable &t, int dev) {
    dev_free(t.d, sizeof(DevPlan) * std::max<size_t>(t.cap, 1), dev);
    t.d = nullptr;
    t.cap = 0;
    t.dirty = true;
}

pm_status upload_table(PlanTable &t, int dev) {
    if (!t.dirty) return PM_OK;
    // set-operation plans first: the matching kernel takes a prefix of the table
    std::stable_partition(t.plans.begin(), t.plans.end(),
                          [](const DevPlan &dp) { return dp.kind == PLAN_SETOPS; });
    t.max_enum = 2;
    for (const DevPlan &dp : t.plans) t.max_enum = std::max(t.max_enum, int(dp.n_enum));
    if (t.plans.size() > t.cap || !t.d) {
        dev_free(t.d, sizeof(DevPlan) * std::max<size_t>(t.cap, 1), dev);
        t.cap = std::max<size_t>(t.plans.size(), 1);
        t.d = (DevPlan *)dev_alloc(sizeof(DevPlan) * t.cap, dev);
        if (!t.d) {
            t.cap = 0;
            set_error("device allocation failed (plan table)");
            return PM_ENOMEM;
        }
    }
    if (!t.plans.empty()) {
        cudaError_t e = cudaMemcpy(t.d, t.plans.data(), sizeof(DevPlan) * t.plans.size(),
                                   cudaMemcpyHostToDevice);
        if (e) return cuda_fail("plan table upload", e);
    }
    t.dirty = false;
    return PM_OK;
}

void free_plan_device(pm_query_plan *p) {
    const int dev = p->g ? p->g->device : 0;
    free_table(p->active, dev);
    free_table(p->rooted_table, dev);
    dev_free(p->d_counters, p->bytes_counters, dev);
    dev_free(p->d_ctl, sizeof(Control), dev);
    dev_free(p->d_bitsets, p->bytes_bitsets, dev);
    dev_free(p->d_col_off, p->bytes_cols, dev);
    dev_free(p->d_col_src, p->bytes_cols, dev);
    dev_free(p->d_popc, p->bytes_cols, dev);
    dev_free(p->d_stats, std::max<size_t>(256, sizeof(unsigned long long) * (p->morph.matched.size() + 1)), dev);
    dev_free(p->d_timed_out, std::max<size_t>(p->morph.matched.size(), 1), dev);
    p->d_timed_out = nullptr;
    dev_free(p->d_wedge, p->bytes_wedge, dev);
    p->d_wedge = nullptr;
    p->bytes_wedge = 0;
    dev_free(p->d_lists, p->bytes_lists, dev);
    p->d_lists = nullptr;
    p->bytes_lists = 0;
    p->wedge_ready = false;
    dev_free(p->d_spill, p->bytes_spill, dev);
    p->d_spill = nullptr;
    p->bytes_spill = 0;
    p->spill_ready = false;
    dev_free(p->d_plan_done, sizeof(unsigned int) * 3 * p->plan_done_cap, dev);
    p->d_plan_done = nullptr;
    p->plan_done_cap = 0;
    dev_free(p->d_targets, p->bytes_targets, dev);
    dev_free(p->d_tslot, p->bytes_tslot, dev);
    dev_free(p->d_dW, p->bytes_dW, dev);
    dev_free(p->d_dtouched, p->bytes_dW, dev);
    dev_free(p->d_basis, sizeof(uint64_t) * 2 * DB_COUNT, dev);
    dev_free(p->d_k4e, p->bytes_k4e, dev);
    dev_free(p->d_local, p->bytes_local, dev);
    free_wheel(p, dev);
    p->d_k4e = nullptr;
    p->bytes_k4e = 0;
    p->d_local = nullptr;
    p->bytes_local = 0;
    p->local_ready = false;
    p->d_targets = nullptr;
    p->bytes_targets = 0;
    p->d_tslot = nullptr;
    p->bytes_tslot = 0;
    p->d_dW = nullptr;
    p->d_dtouched = nullptr;
    p->bytes_dW = 0;
    p->d_basis = nullptr;
    dev_free(p->d_defer, sizeof(Deferred) * std::max<uint32_t>(p->defer_cap, 1), dev);
    dev_free(p->d_piece_off, sizeof(uint32_t) * std::max<uint32_t>(p->defer_cap, 1), dev);
    p->d_counters = nullptr;
    p->d_ctl = nullptr;
    p->d_bitsets = nullptr;
    p->d_col_off = p->d_col_src = nullptr;
    p->d_popc = nullptr;
    p->d_stats = nullptr;
    p->d_defer = nullptr;
    p->d_piece_off = nullptr;
    p->defer_cap = 0;
    p->device_ready = false;
}

// Root list in internal ids with its oriented-edge offsets, on the device.
struct RootTasks {
    int32_t *d_roots = nullptr;
    int64_t *d_off = nullptr;
    size_t b_roots = 0, b_off = 0;
    int device = 0;
    ~RootTasks() {
        dev_free(d_roots, b_roots, device);
        dev_free(d_off, b_off, device);
    }
};

DevTasks all_tasks(const pm_graph *g) {
    DevTasks t{};
    t.roots = nullptr;
    for (int s = 0; s < 3; s++) {
        t.off[s] = g->d_off[s];
        t.ntasks[s] = g->ntasks[s];
    }
    t.nroots = g->n;
    return t;
}

pm_status root_tasks(const pm_graph *g, const int32_t *roots, int64_t nroots, cudaStream_t s,
                     RootTasks &rt, DevTasks *out) {
    std::vector<int32_t> ids(nroots);
    std::vector<int64_t> off(nroots + 1, 0);
    for (int64_t i = 0; i < nroots; i++) {
        if (roots[i] < 0 || roots[i] >= g->n) {
            set_error("pm_count_roots: root id outside [0, n)");
            return PM_EINVAL;
        }
        ids[i] = g->new_id[roots[i]];
        off[i + 1] = off[i] + g->lowdeg[ids[i]];
    }
    rt.device = g->device;
    rt.b_roots = sizeof(int32_t) * std::max<int64_t>(nroots, 1);
    rt.b_off = sizeof(int64_t) * (nroots + 1);
    rt.d_roots = (int32_t *)dev_alloc(rt.b_roots, g->device);
    rt.d_off = (int64_t *)dev_alloc(rt.b_off, g->device);
    if (!rt.d_roots || !rt.d_off) {
        set_error("pm_count_roots: device allocation failed");
        return PM_ENOMEM;
    }
    cudaError_t e1 = nroots ? cudaMemcpyAsync(rt.d_roots, ids.data(), sizeof(int32_t) * nroots,
                                              cudaMemcpyHostToDevice, s) : cudaSuccess;
    cudaError_t e2 = cudaMemcpyAsync(rt.d_off, off.data(), rt.b_off, cudaMemcpyHostToDevice, s);
    if (e1 || e2) return cuda_fail("pm_count_roots: upload", e1 ? e1 : e2);
    DevTasks t{};
    t.roots = rt.d_roots;
    t.off[0] = rt.d_off;
    t.ntasks[0] = off[nroots];
    t.nroots = nroots;
    *out = t;
    return PM_OK;
}

void u128_from_words(const uint64_t *w, unsigned __int128 *v) {
    *v = (unsigned __int128)w[0] | ((unsigned __int128)w[1] << 64);
}

// Device buffers of a plan, made on first use (pm_plan itself is host-only).
pm_status ensure_device(pm_query_plan *p) {
    const pm_graph *g = p->g;
    if (!g) {
        set_error("plan was made without a graph; it cannot run");
        return PM_EINVAL;
    }
    if (p->device_ready) return PM_OK;
    const size_t nm = p->morph.matched.size();
    p->bytes_counters = sizeof(uint64_t) * 2 * std::max<size_t>(nm, 1);
    p->d_counters = (uint64_t *)dev_alloc(p->bytes_counters, g->device);
    p->d_ctl = (Control *)dev_alloc(sizeof(Control), g->device);
    // deferral list: room for every first-pass chunk of the largest table,
    // up to 2^26 entries (768 MiB); beyond that, oversized chunks run unsplit
    const int64_t per_plan = (std::max(g->ntasks[2], int64_t(1)) + 31) / 32;
    const int64_t nplans = int64_t(std::max(p->rooted.size(), p->free_plans.size()));
    p->defer_cap = uint32_t(std::min<int64_t>(std::max<int64_t>(per_plan * nplans, 1024),
                                              int64_t(1) << 26));
    p->d_defer = (Deferred *)dev_alloc(sizeof(Deferred) * p->defer_cap, g->device);
    p->d_piece_off = (uint32_t *)dev_alloc(sizeof(uint32_t) * p->defer_cap, g->device);
    if (!p->d_counters || !p->d_ctl || !p->d_defer || !p->d_piece_off) {
        set_error("device allocation failed (plan buffers)");
        free_plan_device(p);
        return PM_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    if (p->op == PM_OP_SUPPORT) {
        p->words = (g->n + 31) / 32;
        p->bytes_bitsets = sizeof(uint32_t) * size_t(p->words) * std::max(p->n_bitsets, 1);
        p->bytes_cols = sizeof(int64_t) * std::max(p->col_off.size(), p->col_src.size()) + 64;
        p->d_bitsets = (uint32_t *)dev_alloc(p->bytes_bitsets, g->device);
        p->d_col_off = (int32_t *)dev_alloc(p->bytes_cols, g->device);
        p->d_col_src = (int32_t *)dev_alloc(p->bytes_cols, g->device);
        p->d_popc = (unsigned long long *)dev_alloc(p->bytes_cols, g->device);
        if (!p->d_bitsets || !p->d_col_off || !p->d_col_src || !p->d_popc) {
            set_error("device allocation failed (MNI bitsets)");
            free_plan_device(p);
            return PM_ENOMEM;
        }
        e = cudaMemcpy(p->d_col_off, p->col_off.data(), sizeof(int32_t) * p->col_off.size(),
                       cudaMemcpyHostToDevice);
        if (!e && !p->col_src.empty())
            e = cudaMemcpy(p->d_col_src, p->col_src.data(), sizeof(int32_t) * p->col_src.size(),
                           cudaMemcpyHostToDevice);
    }
    if (!e && (!p->ev0 || !p->ev1)) {
        e = cudaEventCreate(&p->ev0);
        if (!e) e = cudaEventCreate(&p->ev1);
    }
    if (!e && p->pat_ev.empty()) {
        p->pat_ev.assign(2 * nm, nullptr);
        p->pat_recorded.assign(nm, 0);
        for (size_t i = 0; i < 2 * nm && !e; i++) e = cudaEventCreate(&p->pat_ev[i]);
    }
    if (e) {
        free_plan_device(p);
        return cuda_fail("plan set-up", e);
    }
    p->device_ready = true;
    return PM_OK;
}

int64_t echunks_for(const std::vector<DevPlan> &plans, const DevTasks &t) {
    int64_t most = 0;
    for (const DevPlan &dp : plans)
        if (dp.kind == PLAN_SETOPS) most = std::max(most, t.ntasks[dp.task_space]);
    return (most + 31) / 32;
}

// Scratch of the wedge kernels: entry lists of the heavy-root kernel (two
// per block, largest degree each) and, when some roots are light, the light
// kernel's dense per-block counters (zeroed once; the kernel leaves them
// zero).  Roots of rank >= n - H are heavy, H = PM_WEDGE_HEAVY (default
// 16384; rows are addressed with 32-bit cursors, so a graph with 2^32 or
// more adjacency entries has no heavy roots).
pm_status ensure_wedge(pm_query_plan *p, cudaStream_t s) {
    if (p->wedge_ready) return PM_OK;
    const pm_graph *g = p->g;
    p->wedge_nblocks = wedge_blocks(g->device);
    int64_t heavy = 16384;
    if (const char *env = std::getenv("PM_WEDGE_HEAVY")) heavy = std::max<int64_t>(0, std::atoll(env));
    if (2 * g->m >= (int64_t(1) << 32)) heavy = 0;
    p->heavy_from = std::max<int64_t>(0, g->n - heavy);
    p->list_cap = std::max<int64_t>(1, g->max_degree);
    if (p->heavy_from < g->n) {
        p->bytes_lists = sizeof(uint2) * 2 * size_t(p->list_cap) * size_t(p->wedge_nblocks);
        p->d_lists = (uint2 *)dev_alloc(p->bytes_lists, g->device);
        if (!p->d_lists) {
            p->bytes_lists = 0;
            set_error("device allocation failed (wedge entry lists)");
            return PM_ENOMEM;
        }
    }
    if (p->heavy_from > 0) {
        p->bytes_wedge = sizeof(uint32_t) * size_t(g->n) * size_t(p->wedge_nblocks);
        p->d_wedge = (uint32_t *)dev_alloc(p->bytes_wedge, g->device);
        if (!p->d_wedge) {
            p->bytes_wedge = 0;
            set_error("device allocation failed (wedge counters)");
            return PM_ENOMEM;
        }
        cudaError_t e = cudaMemsetAsync(p->d_wedge, 0, p->bytes_wedge, s);
        if (e) return cuda_fail("wedge counters", e);
    }
    p->wedge_ready = true;
    return PM_OK;
}

// Spill sets of the clique kernel, sized by the graph's largest degree
// (none when every set fits the kernel's shared buffers).
pm_status ensure_clique(pm_query_plan *p) {
    if (p->spill_ready) return PM_OK;
    const pm_graph *g = p->g;
    p->spill_len = clique_spill_len(g->max_degree);
    if (p->spill_len > 0) {
        p->bytes_spill = sizeof(int32_t) * 2 * size_t(p->spill_len) * size_t(clique_warps(g->device));
        p->d_spill = (int32_t *)dev_alloc(p->bytes_spill, g->device);
        if (!p->d_spill) {
            p->bytes_spill = 0;
            set_error("device allocation failed (clique spill sets)");
            return PM_ENOMEM;
        }
    }
    p->spill_ready = true;
    return PM_OK;
}

// Scratch of the decomposition kernels for the active passes: the sums, the
// per-slot triangle counts and, for 2-path passes, per-block counters
// (zeroed once; the kernel leaves them zero) and touched lists.
pm_status ensure_decomp(pm_query_plan *p, cudaStream_t s) {
    const pm_graph *g = p->g;
    const int passes = p->decomp_passes_active;
    if (!p->d_basis) {
        p->d_basis = (uint64_t *)dev_alloc(sizeof(uint64_t) * 2 * DB_COUNT, g->device);
        if (!p->d_basis) {
            set_error("device allocation failed (decomposition sums)");
            return PM_ENOMEM;
        }
    }
    if (!p->d_tslot) {
        p->bytes_tslot = sizeof(int32_t) * size_t(std::max<int64_t>(2 * g->m, 1));
        p->d_tslot = (int32_t *)dev_alloc(p->bytes_tslot, g->device);
        if (!p->d_tslot) {
            p->bytes_tslot = 0;
            set_error("device allocation failed (triangle counts per edge)");
            return PM_ENOMEM;
        }
    }
    if ((passes & DP_PATHS) && !p->d_dW) {
        p->dpath_blocks = decomp_path_blocks(g->device);
        p->bytes_dW = sizeof(uint32_t) * size_t(g->n) * size_t(p->dpath_blocks);
        p->d_dW = (uint32_t *)dev_alloc(p->bytes_dW, g->device);
        p->d_dtouched = (int32_t *)dev_alloc(p->bytes_dW, g->device);
        if (!p->d_dW || !p->d_dtouched) {
            dev_free(p->d_dW, p->bytes_dW, g->device);
            dev_free(p->d_dtouched, p->bytes_dW, g->device);
            p->d_dW = nullptr;
            p->d_dtouched = nullptr;
            p->bytes_dW = 0;
            set_error("device allocation failed (2-path counters)");
            return PM_ENOMEM;
        }
        cudaError_t e = cudaMemsetAsync(p->d_dW, 0, p->bytes_dW, s);
        if (e) return cuda_fail("2-path counters", e);
    }
    if ((passes & DP_K4E) && !p->d_k4e) {
        p->bytes_k4e = sizeof(uint32_t) * size_t(std::max<int64_t>(2 * g->m, 1));
        p->d_k4e = (uint32_t *)dev_alloc(p->bytes_k4e, g->device);
        if (!p->d_k4e) {
            p->bytes_k4e = 0;
            set_error("device allocation failed (4-cliques per edge)");
            return PM_ENOMEM;
        }
    }
    if ((passes & DP_WHEEL) && !p->wh.T) {
        auto &w = p->wh;
        const int64_t nnz = 2 * g->m;
        auto fail = [&](const char *what) {
            free_wheel(p, g->device);
            set_error(std::string("device allocation failed (") + what + ")");
            return PM_ENOMEM;
        };
        w.b_toff = sizeof(int64_t) * size_t(nnz + 1);
        w.toff = (int64_t *)dev_alloc(w.b_toff, g->device);
        w.b_bsum = sizeof(int64_t) * size_t(std::max<int64_t>(tscan_blocks(nnz), 1));
        w.bsum = (int64_t *)dev_alloc(w.b_bsum, g->device);
        if (!w.toff || !w.bsum) return fail("common-neighbour list offsets");
        if (g->n_hubs > 0) {
            w.b_rank = sizeof(int32_t) * size_t(g->n_hubs) * size_t(g->hub_words);
            w.rank = (int32_t *)dev_alloc(w.b_rank, g->device);
            if (!w.rank) return fail("hub rank index");
        }
        // the lists' total length: one triangle pass (own control block, no
        // deadline) and the offset scan
        int64_t total = 0;
        if (nnz > 0) {
            Control *ctl = (Control *)dev_alloc(sizeof(Control), g->device);
            if (!ctl) return fail("control block");
            cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Control), s);
            DecompLaunch D{};
            D.g = g->dev();
            D.tasks = all_tasks(g);
            D.t = p->d_tslot;
            D.basis = p->d_basis;
            D.ctl = ctl;
            WheelArgs A{};
            A.g = D.g;
            A.t = p->d_tslot;
            A.toff = w.toff;
            A.bsum = w.bsum;
            int bad = e != cudaSuccess;
            if (!bad) bad = launch_decomp_triangles(D, s) || launch_list_offsets(A, s);
            if (!bad) e = cudaMemcpyAsync(&total, w.toff + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (!bad && !e) e = cudaStreamSynchronize(s);
            dev_free(ctl, sizeof(Control), g->device);
            if (bad) return PM_ECUDA;
            if (e) return cuda_fail("common-neighbour list sizes", e);
        }
        w.b_T = sizeof(int32_t) * size_t(std::max<int64_t>(total, 1));
        w.T = (int32_t *)dev_alloc(w.b_T, g->device);
        if (!w.T) return fail("common-neighbour lists");
    }
    if ((passes & DP_K23E) && !p->wh.kW) {
        auto &w = p->wh;
        w.k23_blocks = k23_blocks(g->device);
        w.b_mpos = sizeof(int32_t) * size_t(std::max<int64_t>(2 * g->m, 1));
        w.b_kW = sizeof(uint32_t) * size_t(g->n) * size_t(w.k23_blocks);
        w.b_kE = sizeof(unsigned long long) * size_t(g->n) * size_t(w.k23_blocks);
        w.mpos = (int32_t *)dev_alloc(w.b_mpos, g->device);
        w.kW = (uint32_t *)dev_alloc(w.b_kW, g->device);
        w.kE = (unsigned long long *)dev_alloc(w.b_kE, g->device);
        w.ktouched = (int32_t *)dev_alloc(w.b_kW, g->device);
        if (!w.mpos || !w.kW || !w.kE || !w.ktouched) {
            free_wheel(p, g->device);
            set_error("device allocation failed (K2,3 root counters)");
            return PM_ENOMEM;
        }
        cudaError_t e = cudaMemsetAsync(w.kW, 0, w.b_kW, s);
        if (!e) e = cudaMemsetAsync(w.kE, 0, w.b_kE, s);
        if (e) return cuda_fail("K2,3 root counters", e);
    }
    if ((passes & DP_K5E) && !p->wh.k5e_blocks) {
        auto &w = p->wh;
        w.k5e_blocks = k5e_blocks(g->device);
        w.k5g_words = k5e_global_words(g->max_updeg, g->max_degree);
        if (w.k5g_words) {
            // per warp (16 per block): 32-bit counters over the largest up-degree
            w.b_k5g = sizeof(uint32_t) * size_t(w.k5g_words) * size_t(w.k5e_blocks) * 16;
            w.k5g = (uint32_t *)dev_alloc(w.b_k5g, g->device);
            if (!w.k5g) {
                free_wheel(p, g->device);
                set_error("device allocation failed (K5 minus an edge counters)");
                return PM_ENOMEM;
            }
            cudaError_t e = cudaMemsetAsync(w.k5g, 0, w.b_k5g, s);
            if (e) return cuda_fail("K5 minus an edge counters", e);
        }
    }
    if ((passes & DP_W4) && !p->wh.w4_blocks) {
        auto &w = p->wh;
        w.w4_blocks = w4_blocks(g->device);
        w.gcnt_words = w4_global_words(g->max_degree);
        if (w.gcnt_words) {
            w.b_gcnt = sizeof(uint32_t) * size_t(w.gcnt_words) * size_t(w.w4_blocks);
            w.gcnt = (uint32_t *)dev_alloc(w.b_gcnt, g->device);
            if (!w.gcnt) {
                free_wheel(p, g->device);
                set_error("device allocation failed (4-wheel counters)");
                return PM_ENOMEM;
            }
        }
    }
    if ((passes & DP_LOCAL) && !p->local_ready) {
        p->local_blocks = local_blocks(g->device);
        const int64_t gw = local_grow_words(g->max_updeg);
        if (gw > 0) {
            // neighbourhoods too large for shared memory: per-block rows,
            // members and per-member sums in global memory
            p->bytes_local = size_t(p->local_blocks) *
                             (sizeof(uint32_t) * size_t(gw) + 2 * sizeof(int32_t) * size_t(g->max_updeg));
            p->d_local = (uint32_t *)dev_alloc(p->bytes_local, g->device);
            if (!p->d_local) {
                p->bytes_local = 0;
                set_error("device allocation failed (neighbourhood bitmaps)");
                return PM_ENOMEM;
            }
        }
        p->local_ready = true;
    }
    return PM_OK;
}

// Launch both matching passes for one plan table on the given tasks.
// gate_budget_ns > 0 (with gate_flags): every matched pattern gets its own
// deadline and its expiry is flagged per pattern (pm_count_each).
pm_status launch_table(pm_query_plan *p, const PlanTable &t, const DevTasks &tasks,
                       int sample_stride, bool domains, unsigned long long *stats,
                       cudaStream_t s, uint64_t gate_budget_ns = 0,
                       uint8_t *gate_flags = nullptr, bool record = false,
                       bool with_decomp = false) {
    // events around each matched pattern's launches (per-pattern mode only)
    if (record) std::fill(p->pat_recorded.begin(), p->pat_recorded.end(), 0);
    auto mark = [&](int counter, int end) {
        if (!record || counter < 0 || size_t(counter) >= p->pat_recorded.size()) return;
        cudaEventRecord(p->pat_ev[2 * size_t(counter) + size_t(end)], s);
        if (end) p->pat_recorded[size_t(counter)] = 1;
    };
    const pm_graph *g = p->g;
    MatchLaunch L{};
    L.g = g->dev();
    L.plans = t.d;
    L.nplans = int(t.plans.size());
    L.max_enum = t.max_enum;
    L.tasks = tasks;
    L.n_echunks = echunks_for(t.plans, tasks);
    L.sample_stride = sample_stride;
    L.counters = p->d_counters;
    L.bitsets = p->d_bitsets;
    L.words = p->words;
    L.ctl = p->d_ctl;
    L.defer = p->d_defer;
    L.defer_cap = p->defer_cap;
    L.piece_off = p->d_piece_off;
    L.stats = stats;
    int n_setops = 0;
    while (n_setops < L.nplans && t.plans[n_setops].kind == PLAN_SETOPS) n_setops++;
    if (n_setops > 0 && L.n_echunks > 0 && p->launch_mode == PM_LAUNCH_PER_PATTERN) {
        // one launch sequence per matched pattern (plans of a pattern are adjacent)
        int b = 0;
        while (b < n_setops) {
            int e = b + 1;
            while (e < n_setops && t.plans[e].counter == t.plans[b].counter) e++;
            MatchLaunch G = L;
            G.plans = t.d + b;
            G.nplans = e - b;
            std::vector<DevPlan> sub(t.plans.begin() + b, t.plans.begin() + e);
            G.n_echunks = echunks_for(sub, tasks);
            G.max_enum = 2;
            for (const DevPlan &dp : sub) G.max_enum = std::max(G.max_enum, int(dp.n_enum));
            if (gate_flags) {
                p->launches++;
                if (launch_pattern_gate(p->d_ctl, gate_flags, b > 0 ? t.plans[b - 1].counter : -1,
                                        gate_budget_ns, s))
                    return PM_ECUDA;
            } else if (b > 0 && (p->launches++, launch_rearm(p->d_ctl, s))) {
                return PM_ECUDA;
            }
            mark(t.plans[b].counter, 0);
            p->launches += 3;
            G.stats = stats ? stats + 1 + t.plans[b].counter : nullptr;   // bytes per matched pattern
            const int rc = domains ? launch_domains(G, s) : launch_count(G, s);
            if (rc) return PM_ECUDA;
            mark(t.plans[b].counter, 1);
            b = e;
        }
    } else if (n_setops > 0 && L.n_echunks > 0 && !gate_flags) {
        L.nplans = n_setops;
        p->launches += 3;
        L.stats = stats ? stats + 1 + t.plans[0].counter : nullptr;     // one launch: all on the first
        const int rc = domains ? launch_domains(L, s) : launch_count(L, s);
        if (rc) return PM_ECUDA;
    } else if (n_setops > 0 && L.n_echunks > 0) {
        // per-pattern deadlines in the shared launch: one persistent launch
        // (both passes over one queue) per pattern size, smallest first (the
        // plans are sorted so), each pattern with the budget from its
        // launch's start; plans whose work is cut are flagged from their
        // progress counters.  A size's deferred hub pieces are thus taken up
        // as soon as that size's first pass ends, not behind larger patterns.
        if (!p->d_plan_done || p->plan_done_cap < size_t(n_setops)) {
            dev_free(p->d_plan_done, sizeof(unsigned int) * 3 * p->plan_done_cap, g->device);
            p->plan_done_cap = size_t(n_setops);
            p->d_plan_done = (unsigned int *)dev_alloc(sizeof(unsigned int) * 3 * p->plan_done_cap,
                                                       g->device);
            if (!p->d_plan_done) {
                p->plan_done_cap = 0;
                set_error("device allocation failed (plan progress)");
                return PM_ENOMEM;
            }
        }
        int b = 0;
        while (b < n_setops) {
            const int kb = p->morph.matched[size_t(t.plans[b].counter)].k;
            int e = b + 1;
            while (e < n_setops && p->morph.matched[size_t(t.plans[e].counter)].k == kb) e++;
            MatchLaunch G = L;
            G.plans = t.d + b;
            G.nplans = e - b;
            std::vector<DevPlan> sub(t.plans.begin() + b, t.plans.begin() + e);
            G.n_echunks = echunks_for(sub, tasks);
            G.max_enum = 2;
            for (const DevPlan &dp : sub) G.max_enum = std::max(G.max_enum, int(dp.n_enum));
            if (G.n_echunks == 0) {
                b = e;
                continue;
            }
            cudaMemsetAsync(p->d_plan_done, 0, sizeof(unsigned int) * 3 * size_t(e - b), s);
            G.plan_done = p->d_plan_done;
            p->launches++;
            if (launch_pattern_gate(p->d_ctl, gate_flags, -1, gate_budget_ns, s)) return PM_ECUDA;
            p->launches += 3;
            G.stats = stats ? stats + 1 + t.plans[b].counter : nullptr;
            const int rc = domains ? launch_domains(G, s) : launch_count(G, s);
            if (rc) return PM_ECUDA;
            const int64_t stride = sample_stride > 1 ? sample_stride : 1;
            p->launches++;
            if (launch_plan_flags(p->d_ctl, G.plans, e - b, p->d_plan_done,
                                  (unsigned long long)((G.n_echunks + stride - 1) / stride), gate_flags, s))
                return PM_ECUDA;
            b = e;
        }
    }
    int last = n_setops > 0 && !(gate_flags && p->launch_mode == PM_LAUNCH_SINGLE)
                   ? t.plans[n_setops - 1].counter
                   : -1;
    for (size_t i = size_t(n_setops); i < t.plans.size(); i++) {
        const DevPlan &dp = t.plans[i];
        if (domains) {
            set_error("wedge-pair and clique plans count only");
            return PM_EINVAL;
        }
        pm_status st = dp.kind == PLAN_WEDGE_PAIRS ? ensure_wedge(p, s) : ensure_clique(p);
        if (st != PM_OK) return st;
        if (gate_flags && (p->launches++, launch_pattern_gate(p->d_ctl, gate_flags, last, gate_budget_ns, s)))
            return PM_ECUDA;
        mark(dp.counter, 0);
        p->launches += dp.kind == PLAN_WEDGE_PAIRS
                           ? int(p->heavy_from < L.g.n) + int(p->heavy_from > 0)
                           : 1;
        if (dp.kind == PLAN_WEDGE_PAIRS) {
            if (launch_wedge_pairs(L.g, tasks, p->heavy_from, dp.counter, p->d_counters, p->d_wedge,
                                   p->d_lists, p->list_cap, p->wedge_nblocks, sample_stride,
                                   p->d_ctl, s))
                return PM_ECUDA;
        } else if (launch_clique(L.g, tasks, dp.k, dp.counter, p->d_counters, p->d_spill,
                                 p->spill_len, sample_stride, p->d_ctl,
                                 stats ? stats + 1 + dp.counter : nullptr, s)) {
            return PM_ECUDA;
        }
        mark(dp.counter, 1);
        last = dp.counter;
    }
    if (with_decomp && !p->decomp_targets.empty()) {
        // the decomposable patterns together: the passes they need, then
        // one combine writing each one's count (timed as one group, on the
        // first of them)
        pm_status st = ensure_decomp(p, s);
        if (st != PM_OK) return st;
        if (gate_flags && (p->launches++, launch_pattern_gate(p->d_ctl, gate_flags, last, gate_budget_ns, s)))
            return PM_ECUDA;
        const int first = p->decomp_targets[1];
        const int nt = int(p->decomp_targets.size() / 2);
        mark(first, 0);
        DecompLaunch D{};
        D.g = L.g;
        D.tasks = tasks;
        D.passes = p->decomp_passes_active;
        D.t = p->d_tslot;
        D.k4e = p->d_k4e;
        D.local_blocks = p->local_blocks;
        D.local.g = L.g;
        D.local.low_off = tasks.off[TASKS_LOWER];
        D.local.basis = p->d_basis;
        D.local.ctl = p->d_ctl;
        D.local.max_s = p->g->max_updeg;
        D.local.grow_words = local_grow_words(p->g->max_updeg);
        if (p->d_local) {
            // per block: rows, then members, then per-member sums
            D.local.grows = p->d_local;
            D.local.gmem = reinterpret_cast<int32_t *>(p->d_local + size_t(p->local_blocks) * size_t(D.local.grow_words));
            D.local.gts = reinterpret_cast<uint32_t *>(D.local.gmem) + size_t(p->local_blocks) * size_t(D.local.max_s);
        }
        D.wheel.toff = p->wh.toff;
        D.wheel.T = p->wh.T;
        D.wheel.T_len = int64_t(p->wh.b_T / sizeof(int32_t));
        D.wheel.bsum = p->wh.bsum;
        D.wheel.hub_rank = p->wh.rank;
        D.wheel.n_hubs = p->wh.rank ? g->n_hubs : 0;
        D.wheel.mpos = p->wh.mpos;
        D.wheel.gcnt = p->wh.gcnt;
        D.wheel.gcnt_words = p->wh.gcnt_words;
        D.wheel.w4_blocks = p->wh.w4_blocks;
        D.wheel.kW = p->wh.kW;
        D.wheel.kE = p->wh.kE;
        D.wheel.k23_narrow = g->max_degree < 65536 ? 1 : 0;
        D.wheel.ktouched = p->wh.ktouched;
        D.wheel.k23_blocks = p->wh.k23_blocks;
        D.wheel.k5g = p->wh.k5g;
        D.wheel.k5g_words = p->wh.k5g_words;
        D.wheel.k5e_blocks = p->wh.k5e_blocks;
        D.wheel.g = L.g;
        D.W = p->d_dW;
        D.touched = p->d_dtouched;
        D.path_blocks = p->dpath_blocks;
        D.basis = p->d_basis;
        D.ctl = p->d_ctl;
        D.stats = stats ? stats + 1 + first : nullptr;
        p->launches += 3 + int((D.passes & DP_TRI2) != 0) + int((D.passes & DP_PATHS) != 0) +
                       2 * int((D.passes & DP_LOCAL) != 0) + 1 +
                       ((D.passes & DP_WHEEL) ? wheel_launches(D.wheel, D.passes) : 0);
        if (launch_decomp(D, s)) return PM_ECUDA;
        if (launch_decomp_combine(p->d_basis, p->d_targets, nt, p->d_counters, s)) return PM_ECUDA;
        mark(first, 1);
        if (gate_flags && (p->launches++, launch_flag_targets(p->d_ctl, gate_flags, p->d_targets, nt, s)))
            return PM_ECUDA;
        last = -1;
    }
    if (gate_flags && last >= 0 && (p->launches++, launch_pattern_gate(p->d_ctl, gate_flags, last, 0, s)))
        return PM_ECUDA;
    return PM_OK;
}

// After an expired deadline the wedge counters may be left non-zero.
void rezero_wedge(pm_query_plan *p, cudaStream_t s) {
    if (p->d_wedge) cudaMemsetAsync(p->d_wedge, 0, p->bytes_wedge, s);
    if (p->d_dW) cudaMemsetAsync(p->d_dW, 0, p->bytes_dW, s);
    if (p->wh.kW) cudaMemsetAsync(p->wh.kW, 0, p->wh.b_kW, s);
    if (p->wh.kE) cudaMemsetAsync(p->wh.kE, 0, p->wh.b_kE, s);
    if (p->wh.k5g) cudaMemsetAsync(p->wh.k5g, 0, p->wh.b_k5g, s);
}

// Task granularity: the second-level candidates a chunk keeps before the
// rest is deferred to other warps (hub roots), scaled by split code 0 (/4),
// 1 (as compiled) or 2 (x4).
void scale_split(DevPlan &dp, int code) {
    if (code == 0) dp.split = std::max(8, dp.split / 4);
    else if (code == 2) dp.split = std::min(1 << 20, dp.split * 4);
}

// The plans of matched pattern j in family f (0 rooted, 1 free), with the
// split code of the pattern (when tuned).
std::vector<DevPlan> family_plans(const pm_query_plan *p, size_t j, int f) {
    std::vector<DevPlan> v;
    if (f == PM_PLANS_FREE) v = {p->free_plans[j]};
    else v.assign(p->rooted.begin() + p->rooted_begin[j], p->rooted.begin() + p->rooted_begin[j + 1]);
    if (j < p->split_code.size())
        for (DevPlan &dp : v) scale_split(dp, p->split_code[j]);
    return v;
}

// Decomposable patterns of counting plans use the decomposition kernels
// unless a set-operation family is forced.
bool decomp_default(const pm_query_plan *p, size_t j) {
    return p->op == PM_OP_COUNT && p->decomp_f[j] >= 0 &&
           (p->forced == PM_PLANS_AUTO || p->forced == PM_PLANS_QUICK ||
            p->forced == PM_PLANS_DECOMP);
}

// Family without timing: decomposition where it applies, the rooted family
// where it runs the wedge kernel, else free.
int quick_family(const pm_query_plan *p, size_t j) {
    const bool wedge = p->rooted_begin[j + 1] - p->rooted_begin[j] == 1 &&
                       p->rooted[p->rooted_begin[j]].kind == PLAN_WEDGE_PAIRS;
    return decomp_default(p, j) ? PM_PLANS_DECOMP : (wedge ? PM_PLANS_ROOTED : PM_PLANS_FREE);
}

// Autotuner: for every matched pattern without a decision, time its rooted
// plans and its free plan (counting kernels) on the same sample of task
// chunks (every stride-th chunk, about 4096 chunks, 0.5 s deadline each) and
// keep the faster family.  Decisions are cached on the graph under the
// pattern's canonical key, so later plans on the same graph reuse them.
pm_status autotune(pm_query_plan *p, cudaStream_t s) {
    const pm_graph *g = p->g;
    const size_t nm = p->morph.matched.size();
    double budget_s = 30.0;
    if (const char *env = std::getenv("PM_AUTOTUNE_BUDGET_S")) budget_s = std::atof(env);
    const auto t_start = std::chrono::steady_clock::now();
    // smallest patterns first, so a spent budget leaves the largest untimed
    std::vector<size_t> order(nm);
    for (size_t j = 0; j < nm; j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const Pat &x = p->morph.matched[a], &y = p->morph.matched[b];
        return x.k != y.k ? x.k < y.k : x.n_edges() < y.n_edges();
    });
    for (size_t j : order) {
        if (p->choice[j] >= 0) continue;
        if (decomp_default(p, j)) {
            p->choice[j] = PM_PLANS_DECOMP;   // per plan: the decision depends on the operation
            continue;
        }
        const Key key = canonical(p->morph.matched[j]);
        {
            std::lock_guard<std::mutex> lk(g->tune_mu);
            auto it = g->tuned.find(key);
            if (it != g->tuned.end()) {
                p->choice[j] = it->second;
                auto sp = g->tuned_split.find(key);
                p->split_code[j] = sp != g->tuned_split.end() ? sp->second : 1;
                continue;
            }
        }
        if (budget_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > budget_s) {
            // sampling budget spent: the quick rule, not cached on the graph
            p->choice[j] = quick_family(p, j);
            p->split_code[j] = 1;
            continue;
        }
        const DevTasks tasks = all_tasks(g);
        float best = std::numeric_limits<float>::infinity();
        int best_f = PM_PLANS_ROOTED;
        // the sample: about 4096 chunks, or 8x (64x) sparser when every
        // family ran past its deadline on the denser one
        for (int sparse = 1; sparse <= 64 && !std::isfinite(best); sparse *= 8)
        for (int f = PM_PLANS_ROOTED; f <= PM_PLANS_FREE; f++) {
            PlanTable t;
            t.plans = family_plans(p, j, f);
            // The clique kernel is exact but not yet load-balanced: the tasks
            // between two hubs sit side by side in one chunk, so one warp can
            // run long after the rest.  Until that is fixed it is left to
            // explicit selection (pm_plan_select, pm_count_roots).
            if (t.plans.size() == 1 && t.plans[0].kind == PLAN_CLIQUE) continue;
            for (DevPlan &dp : t.plans) dp.counter = 0;
            // scratch allocation stays out of the timed region
            if (t.plans.size() == 1 && t.plans[0].kind == PLAN_WEDGE_PAIRS) {
                pm_status st = ensure_wedge(p, s);
                if (st != PM_OK) return st;
            }
            pm_status st = upload_table(t, g->device);
            if (st != PM_OK) return st;
            const int64_t ech = echunks_for(t.plans, tasks);
            const int stride = int(std::max<int64_t>(1, ech / 4096) * sparse);
            cudaError_t e = cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, s);
            if (!e && launch_arm(p->d_ctl, uint64_t(5e8), s)) e = cudaErrorLaunchFailure;
            if (!e) e = cudaEventRecord(p->ev0, s);
            if (!e && launch_table(p, t, tasks, stride, false, nullptr, s) != PM_OK)
                e = cudaErrorLaunchFailure;
            if (!e) e = cudaEventRecord(p->ev1, s);
            Control ctl{};
            if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            float ms = 0.f;
            if (!e) e = cudaEventElapsedTime(&ms, p->ev0, p->ev1);
            free_table(t, g->device);
            if (e) return cuda_fail("autotune", e);
            if (ctl.status == 1) {
                ms = std::numeric_limits<float>::infinity();
                rezero_wedge(p, s);
            } else {
                ms *= float(sparse);    // comparable with the denser sample
            }
            if (ms < best) { best = ms; best_f = f; }
        }
        // task granularity of the chosen family (set-operation plans only):
        // a quarter and four times the compiled split on the same sample
        int best_code = 1;
        std::vector<DevPlan> chosen = family_plans(p, j, best_f);
        bool setops = !chosen.empty();
        for (const DevPlan &dp : chosen) setops &= dp.kind == PLAN_SETOPS && dp.n_enum >= 3;
        if (setops && std::isfinite(best)) {
            for (int code : {0, 2}) {
                PlanTable t;
                t.plans = chosen;
                for (DevPlan &dp : t.plans) {
                    dp.counter = 0;
                    scale_split(dp, code);
                }
                pm_status st = upload_table(t, g->device);
                if (st != PM_OK) return st;
                const int64_t ech = echunks_for(t.plans, tasks);
                const int stride = int(std::max<int64_t>(1, ech / 4096));
                cudaError_t e = cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, s);
                if (!e && launch_arm(p->d_ctl, uint64_t(5e8), s)) e = cudaErrorLaunchFailure;
                if (!e) e = cudaEventRecord(p->ev0, s);
                if (!e && launch_table(p, t, tasks, stride, false, nullptr, s) != PM_OK)
                    e = cudaErrorLaunchFailure;
                if (!e) e = cudaEventRecord(p->ev1, s);
                Control ctl{};
                if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaStreamSynchronize(s);
                float ms = 0.f;
                if (!e) e = cudaEventElapsedTime(&ms, p->ev0, p->ev1);
                free_table(t, g->device);
                if (e) return cuda_fail("autotune (split)", e);
                if (ctl.status != 1 && ms < 0.9f * best) {
                    best = ms;
                    best_code = code;
                }
            }
        }
        p->choice[j] = best_f;
        p->split_code[j] = best_code;
        std::lock_guard<std::mutex> lk(g->tune_mu);
        g->tuned[key] = best_f;
        g->tuned_split[key] = best_code;
        g->tuned_ms[key] = best;
    }
    return PM_OK;
}

// The table pm_count / pm_support run: each matched pattern's chosen family.
pm_status prepare_active(pm_query_plan *p, cudaStream_t s) {
    const size_t nm = p->morph.matched.size();
    std::vector<int> want(nm);
    if (p->forced == PM_PLANS_QUICK) {
        for (size_t j = 0; j < nm; j++) want[j] = quick_family(p, j);
    } else if (p->forced == PM_PLANS_ROOTED || p->forced == PM_PLANS_FREE) {
        std::fill(want.begin(), want.end(), p->forced);
    } else {
        pm_status st = autotune(p, s);
        if (st != PM_OK) return st;
        want = p->choice;
    }
    std::vector<DevPlan> plans;
    std::vector<int32_t> targets;
    int passes = 0;
    for (size_t j = 0; j < nm; j++) {
        if (want[j] == PM_PLANS_DECOMP) {
            targets.push_back(p->decomp_f[j]);
            targets.push_back(int32_t(j));
            passes |= decomp_passes(p->decomp_f[j]);
            continue;
        }
        std::vector<DevPlan> v = family_plans(p, j, want[j]);
        plans.insert(plans.end(), v.begin(), v.end());
    }
    if (targets != p->decomp_targets || !p->d_targets) {
        const size_t bytes = sizeof(int32_t) * std::max<size_t>(targets.size(), 2);
        if (bytes > p->bytes_targets) {
            dev_free(p->d_targets, p->bytes_targets, p->g->device);
            p->d_targets = (int32_t *)dev_alloc(bytes, p->g->device);
            p->bytes_targets = p->d_targets ? bytes : 0;
            if (!p->d_targets) {
                set_error("device allocation failed (decomposition targets)");
                return PM_ENOMEM;
            }
        }
        if (!targets.empty()) {
            cudaError_t e = cudaMemcpy(p->d_targets, targets.data(), sizeof(int32_t) * targets.size(),
                                       cudaMemcpyHostToDevice);
            if (e) return cuda_fail("decomposition targets upload", e);
        }
        p->decomp_targets = targets;
    }
    p->decomp_passes_active = passes;
    std::stable_partition(plans.begin(), plans.end(),
                          [](const DevPlan &dp) { return dp.kind == PLAN_SETOPS; });
    // set-operation plans smallest pattern first, then by the autotuner's
    // sampled time (untimed last; a pattern's plans stay adjacent), so in
    // one shared launch with a deadline the cheap patterns finish first
    {
        std::vector<double> cost(nm, std::numeric_limits<double>::infinity());
        std::lock_guard<std::mutex> lk(p->g->tune_mu);
        for (size_t j = 0; j < nm; j++) {
            auto it = p->g->tuned_ms.find(canonical(p->morph.matched[j]));
            if (it != p->g->tuned_ms.end()) cost[j] = it->second;
        }
        auto setops_end = std::find_if(plans.begin(), plans.end(),
                                       [](const DevPlan &dp) { return dp.kind != PLAN_SETOPS; });
        std::stable_sort(plans.begin(), setops_end, [&](const DevPlan &a, const DevPlan &b) {
            const Pat &x = p->morph.matched[size_t(a.counter)], &y = p->morph.matched[size_t(b.counter)];
            if (x.k != y.k) return x.k < y.k;
            return cost[size_t(a.counter)] < cost[size_t(b.counter)];
        });
    }
    if (p->active.plans.size() != plans.size() ||
        std::memcmp(p->active.plans.data(), plans.data(), sizeof(DevPlan) * plans.size()) != 0) {
        p->active.plans = plans;
        p->active.dirty = true;
    }
    return upload_table(p->active, p->g->device);
}

// Cost of matching one pattern on a graph, for cost-based morph selection:
// the autotuner's sampled time of its faster plan family (cached per graph);
// a pattern whose sampled runs both hit the deadline costs 1e9 ms.
// Cost of a pattern not yet timed once the morph selection's sampling time
// is spent: no sampling, an estimate that only orders patterns by what
// drives matching cost on skewed graphs (size, and anti-edges for
// vertex-induced patterns, whose set differences do not shrink on hubs).
double estimated_cost(const Pat &q) {
    double ms = 1.0;
    for (int i = 3; i < q.k; i++) ms *= 10.0;
    return q.vi && !q.is_clique() ? 20.0 * ms : ms;
}

double pattern_cost(const pm_graph *g, const Pat &q, std::chrono::steady_clock::time_point deadline) {
    const bool spent = std::chrono::steady_clock::now() > deadline;
    const int f = decomp_formula(q);
    if (f >= 0) {
        // the decomposition passes this pattern needs, timed once per graph
        const int passes = decomp_passes(f);
        {
            std::lock_guard<std::mutex> lk(g->tune_mu);
            auto it = g->decomp_ms.find(passes);
            if (it != g->decomp_ms.end()) return it->second;
        }
        if (spent) return 1.0;      // decomposition passes: tens to hundreds of ms at scale 20
        pm_pattern r{};
        r.k = q.k;
        r.edge_mask = q.mask();
        for (int u = 0; u < PM_MAX_K; u++) r.label[u] = -1;
        r.induced = PM_EDGE_INDUCED;
        pm_query_plan *tmp = nullptr;
        double ms = 1e9;
        if (pm_plan(g, &r, 1, PM_OP_COUNT, PM_MORPH_NONE, &tmp) == PM_OK) {
            uint64_t c[2];
            float t = 0.f;
            if (pm_count(tmp, nullptr, 10.0, c, nullptr) == PM_OK &&
                pm_plan_pattern_ms(tmp, &t) == PM_OK)
                ms = t;
            pm_free_plan(tmp);
        }
        std::lock_guard<std::mutex> lk(g->tune_mu);
        g->decomp_ms[passes] = ms;
        return ms;
    }
    const Key key = canonical(q);
    {
        std::lock_guard<std::mutex> lk(g->tune_mu);
        auto it = g->tuned_ms.find(key);
        if (it != g->tuned_ms.end()) return std::isfinite(it->second) ? it->second : 1e9;
    }
    if (spent) return estimated_cost(q);
    pm_pattern r{};
    r.k = q.k;
    r.edge_mask = q.mask();
    for (int u = 0; u < PM_MAX_K; u++) r.label[u] = u < q.k ? q.lab[u] : -1;
    r.induced = q.vi ? PM_VERTEX_INDUCED : PM_EDGE_INDUCED;
    pm_query_plan *tmp = nullptr;
    if (pm_plan(g, &r, 1, PM_OP_COUNT, PM_MORPH_NONE, &tmp) != PM_OK) return 1e9;
    double ms = 1e9;
    if (pm_plan_autotune(tmp, nullptr, nullptr) == PM_OK) {
        std::lock_guard<std::mutex> lk(g->tune_mu);
        auto it = g->tuned_ms.find(canonical(tmp->morph.matched[0]));
        if (it != g->tuned_ms.end() && std::isfinite(it->second)) ms = it->second;
    }
    pm_free_plan(tmp);
    return ms;
}

pm_status run_count(pm_query_plan *p, void *stream, double timeout_s, const int32_t *roots,
                    int64_t nroots, bool use_roots, uint64_t *counts, uint64_t *matched,
                    uint64_t *alg_bytes = nullptr) {
    if (!p || !counts) {
        set_error("pm_count: null argument");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_COUNT) {
        set_error("pm_count: plan was made for PM_OP_SUPPORT");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    if (!g) {
        set_error("pm_count: plan was made without a graph");
        return PM_EINVAL;
    }
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    if (st != PM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RootTasks rt;
    DevTasks tasks;
    PlanTable *table;
    if (use_roots) {
        st = root_tasks(g, roots, nroots, s, rt, &tasks);
        if (st != PM_OK) return st;
        if (p->rooted_table.dirty) p->rooted_table.plans = p->rooted;   // (re)partitioned on upload
        st = upload_table(p->rooted_table, g->device);
        table = &p->rooted_table;
    } else {
        tasks = all_tasks(g);
        st = prepare_active(p, s);
        table = &p->active;
    }
    if (st != PM_OK) return st;
    const size_t nm = p->morph.matched.size();
    cudaError_t e = cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, s);
    if (e) return cuda_fail("pm_count: memset", e);
    const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
    p->launches = 1;
    if (launch_arm(p->d_ctl, budget, s)) return PM_ECUDA;
    const size_t stat_bytes = std::max<size_t>(256, sizeof(unsigned long long) * (nm + 1));
    if (alg_bytes && !p->d_stats) {
        p->d_stats = (unsigned long long *)dev_alloc(stat_bytes, g->device);
        if (!p->d_stats) return PM_ENOMEM;
    }
    if (alg_bytes) {
        e = cudaMemsetAsync(p->d_stats, 0, sizeof(unsigned long long) * (nm + 1), s);
        if (e) return cuda_fail("pm_count: memset", e);
    }
    cudaEventRecord(p->ev0, s);
    st = launch_table(p, *table, tasks, 1, false, alg_bytes ? p->d_stats : nullptr, s, 0, nullptr,
                      !use_roots && !alg_bytes, !use_roots);
    if (st != PM_OK) return st;
    cudaEventRecord(p->ev1, s);
    p->timed = true;
    if (alg_bytes) {
        std::vector<unsigned long long> v(nm + 1);
        e = cudaMemcpyAsync(v.data(), p->d_stats, sizeof(unsigned long long) * (nm + 1),
                            cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail("pm_count: stats readback", e);
        uint64_t total = 0;
        p->pat_bytes.assign(nm, 0);
        for (size_t j = 0; j < nm; j++) {
            p->pat_bytes[j] = v[j + 1];
            total += v[j + 1];
        }
        *alg_bytes = total + v[0];
    }
    std::vector<uint64_t> raw(2 * nm);
    Control ctl;
    e = cudaMemcpyAsync(raw.data(), p->d_counters, sizeof(uint64_t) * 2 * nm,
                        cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail("pm_count: kernel or readback", e);
    if (ctl.status == 1) {
        rezero_wedge(p, s);
        cudaStreamSynchronize(s);
        set_error("pm_count: deadline expired");
        return PM_ETIMEOUT;
    }
    if (ctl.fault) return list_fault("pm_count", ctl.fault);
    if (matched) std::memcpy(matched, raw.data(), sizeof(uint64_t) * 2 * nm);
    return pm_morph(p, raw.data(), counts);
}

// pm_count with a deadline per matched pattern and a status per query.
pm_status run_count_each(pm_query_plan *p, void *stream, double timeout_s, double total_s,
                         uint64_t *counts, int32_t *status) {
    if (!p || !counts || !status) {
        set_error("pm_count_each: null argument");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_COUNT || !p->g) {
        set_error("pm_count_each: needs a counting plan made on a graph");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    cudaStream_t s = (cudaStream_t)stream;
    if (st == PM_OK) st = prepare_active(p, s);
    if (st != PM_OK) return st;
    const size_t nm = p->morph.matched.size();
    if (!p->d_timed_out) {
        p->d_timed_out = (uint8_t *)dev_alloc(std::max<size_t>(nm, 1), g->device);
        if (!p->d_timed_out) return PM_ENOMEM;
    }
    if (p->graph_each) {
        // replay of pm_plan_capture_each (its deadlines are fixed in the graph)
        cudaError_t e = cudaGraphLaunch(p->graph_each, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail("pm_count_each (graph replay)", e);
        std::vector<uint8_t> flags(nm);
        std::memcpy(flags.data(), reinterpret_cast<uint8_t *>(p->h_pinned + 2 * nm) + sizeof(Control), nm);
        Control ctl;
        std::memcpy(&ctl, p->h_pinned + 2 * nm, sizeof(Control));
        if (ctl.fault) return list_fault("pm_count_each (graph replay)", ctl.fault);
        bool any = false;
        for (size_t j = 0; j < nm; j++) any |= flags[j] != 0;
        if (any) {
            rezero_wedge(p, s);
            cudaStreamSynchronize(s);
        }
        p->timed = true;
        st = pm_morph(p, p->h_pinned, counts);
        if (st != PM_OK) return st;
        for (size_t i = 0; i < p->morph.terms.size(); i++) {
            status[i] = PM_OK;
            for (const Term &t : p->morph.terms[i])
                if (flags[t.matched]) status[i] = PM_ETIMEOUT;
            if (status[i] != PM_OK) counts[2 * i] = counts[2 * i + 1] = 0;
        }
        return PM_OK;
    }
    const int saved_mode = p->launch_mode;
    cudaError_t e = cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, s);
    if (!e) e = cudaMemsetAsync(p->d_timed_out, 0, std::max<size_t>(nm, 1), s);
    if (e) {
        p->launch_mode = saved_mode;
        return cuda_fail("pm_count_each: memset", e);
    }
    const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
    p->launches = 1;
    if (launch_arm(p->d_ctl, total_s > 0 ? uint64_t(total_s * 1e9) : 0, s)) {
        p->launch_mode = saved_mode;
        return PM_ECUDA;
    }
    cudaEventRecord(p->ev0, s);
    st = launch_table(p, p->active, all_tasks(g), 1, false, nullptr, s, budget,
                      p->d_timed_out, true, true);
    p->launch_mode = saved_mode;
    if (st != PM_OK) return st;
    cudaEventRecord(p->ev1, s);
    p->timed = true;
    std::vector<uint64_t> raw(2 * nm);
    std::vector<uint8_t> flags(std::max<size_t>(nm, 1));
    e = cudaMemcpyAsync(raw.data(), p->d_counters, sizeof(uint64_t) * 2 * nm,
                        cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(flags.data(), p->d_timed_out, nm, cudaMemcpyDeviceToHost, s);
    Control ctl;
    if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail("pm_count_each: kernel or readback", e);
    if (ctl.fault) return list_fault("pm_count_each", ctl.fault);
    bool any = false;
    for (size_t j = 0; j < nm; j++) any |= flags[j] != 0;
    if (any) {
        rezero_wedge(p, s);
        cudaStreamSynchronize(s);
    }
    st = pm_morph(p, raw.data(), counts);
    if (st != PM_OK) return st;
    for (size_t i = 0; i < p->morph.terms.size(); i++) {
        status[i] = PM_OK;
        for (const Term &t : p->morph.terms[i])
            if (flags[t.matched]) status[i] = PM_ETIMEOUT;
        if (status[i] != PM_OK) counts[2 * i] = counts[2 * i + 1] = 0;
    }
    return PM_OK;
}

}  // namespace

// Validates a query set and returns the size of its alternative set under
// `mode` (morph selection only, no plan compilation): the serving loop's
// per-request count of matched patterns, for its deduplication statistic.
namespace pm {
pm_status matched_set_size(const pm_graph *g, const pm_pattern *queries, int32_t nq,
                           pm_morph_mode mode, int32_t *n_matched) {
    if (!queries || nq < 1 || !n_matched) {
        set_error("matched_set_size: null argument or empty query set");
        return PM_EINVAL;
    }
    std::vector<Pat> pats(nq);
    for (int32_t i = 0; i < nq; i++) {
        pm_status st = to_pat(queries[i], g ? g->labeled : true, &pats[i]);
        if (st != PM_OK) return st;
    }
    MorphPlan mp;
    std::string why;
    // cost-based selection needs device timings; the naive set stands in
    const pm_morph_mode m = mode == PM_MORPH_COST ? PM_MORPH_NAIVE : mode;
    pm_status st = morph_select(pats, PM_OP_COUNT, m, mp, &why, nullptr);
    if (st != PM_OK) {
        set_error("matched_set_size: " + why);
        return st;
    }
    *n_matched = int32_t(mp.matched.size());
    return PM_OK;
}
}  // namespace pm

extern "C" {

pm_status pm_count_each(pm_query_plan *p, void *stream, double timeout_per_pattern_s,
                        double timeout_total_s, uint64_t *counts, int32_t *status) {
    return run_count_each(p, stream, timeout_per_pattern_s, timeout_total_s, counts, status);
}

pm_status pm_set_allocator(pm_alloc_fn alloc, pm_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr)) {
        set_error("pm_set_allocator: set both callbacks or neither");
        return PM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return PM_OK;
}

pm_status pm_load_graph(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                        const uint8_t *labels, int device, void *stream, pm_graph **out) {
    if (fault_injected("load")) {
        set_error("pm_load_graph: fault injected (PM_FAULT=load)");
        return PM_EINVAL;
    }
    return build_graph(n, m_raw, src, dst, labels, device, stream, out);
}

pm_status pm_prepare_csr(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                         int64_t *rowptr, int32_t *col, int32_t *new_id, int64_t *lowdeg) {
    return prepare_csr(n, m_raw, src, dst, rowptr, col, new_id, lowdeg);
}

pm_status pm_graph_get_info(const pm_graph *g, pm_graph_info *out) {
    if (!g || !out) return PM_EINVAL;
    out->n = g->n;
    out->m = g->m;
    out->self_loops = g->self_loops;
    out->duplicates = g->duplicates;
    out->max_degree = g->max_degree;
    out->device_bytes = int64_t(g->bytes);
    out->labeled = g->labeled;
    out->device = g->device;
    return PM_OK;
}

pm_status pm_graph_vertex_order(const pm_graph *g, int32_t *new_id) {
    if (!g || !new_id) return PM_EINVAL;
    std::memcpy(new_id, g->new_id.data(), sizeof(int32_t) * g->n);
    return PM_OK;
}

void pm_free_graph(pm_graph *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    const size_t b_rp = sizeof(int64_t) * (g->n + 1);
    dev_free(g->d_rowptr, b_rp, g->device);
    dev_free(g->d_col, sizeof(int32_t) * std::max<int64_t>(2 * g->m, 1), g->device);
    for (int sp = 0; sp < 3; sp++) dev_free(g->d_off[sp], b_rp, g->device);
    dev_free(g->d_labels, g->n, g->device);
    dev_free(g->d_hub, sizeof(int32_t) * g->n, g->device);
    dev_free(g->d_bits, sizeof(uint32_t) * size_t(g->n_hubs) * size_t(g->hub_words), g->device);
    dev_free(g->d_new_id, sizeof(int32_t) * size_t(g->n), g->device);
    delete g;
}

pm_status pm_plan(const pm_graph *g, const pm_pattern *queries, int32_t nq, pm_op op,
                  pm_morph_mode mode, pm_query_plan **out) {
    if (fault_injected("plan")) {
        set_error("pm_plan: fault injected (PM_FAULT=plan)");
        return PM_EUNSUPPORTED;
    }
    if (!queries || nq < 1 || !out) {
        set_error("pm_plan: null argument or empty query set");
        return PM_EINVAL;
    }
    if (op != PM_OP_COUNT && op != PM_OP_SUPPORT) {
        set_error("pm_plan: unknown op");
        return PM_EINVAL;
    }
    if (mode != PM_MORPH_NONE && mode != PM_MORPH_NAIVE && mode != PM_MORPH_COST) {
        set_error("pm_plan: unknown morph mode");
        return PM_EINVAL;
    }
    std::vector<Pat> pats(nq);
    for (int32_t i = 0; i < nq; i++) {
        pm_status st = to_pat(queries[i], g ? g->labeled : true, &pats[i]);
        if (st != PM_OK) return st;
        if (op == PM_OP_SUPPORT && pats[i].k > 6) {
            set_error("pm_plan: MNI support handles patterns of at most 6 vertices");
            return PM_EUNSUPPORTED;
        }
    }
    auto *p = new (std::nothrow) pm_query_plan();
    if (!p) return PM_ENOMEM;
    p->g = g;
    p->op = op;
    std::string why;
    std::function<double(const Pat &)> cost;
    if (mode == PM_MORPH_COST && g) {
        // sampling time of the whole selection: environment PM_COST_BUDGET_S
        // (default 30 s); patterns met after it get estimated costs
        double budget_s = 30.0;
        if (const char *env = std::getenv("PM_COST_BUDGET_S")) budget_s = std::atof(env);
        const auto deadline = std::chrono::steady_clock::now() +
                              std::chrono::microseconds(int64_t(std::max(0.0, budget_s) * 1e6));
        cost = [g, deadline](const Pat &q) { return pattern_cost(g, q, deadline); };
    }
    pm_status st = morph_select(pats, op, mode, p->morph, &why, g ? &cost : nullptr);
    if (st != PM_OK) {
        set_error("pm_plan: " + why);
        delete p;
        return st;
    }
    const size_t nm = p->morph.matched.size();
    p->dom_base.assign(nm, 0);
    int nb = 0;
    for (size_t j = 0; j < nm; j++) {
        p->dom_base[j] = nb;
        nb += p->morph.matched_columns[j];
    }
    p->n_bitsets = nb;
    p->rooted_begin.push_back(0);
    for (size_t j = 0; j < nm; j++) {
        auto v = compile_plans(p->morph.matched[j], int(j), p->dom_base[j],
                               p->morph.matched_orbit[j], op == PM_OP_COUNT);
        p->rooted.insert(p->rooted.end(), v.begin(), v.end());
        p->rooted_begin.push_back(int(p->rooted.size()));
        p->free_plans.push_back(compile_free_plan(p->morph.matched[j], int(j), p->dom_base[j],
                                                  p->morph.matched_orbit[j], op == PM_OP_COUNT));
    }
    p->choice.assign(nm, -1);
    p->split_code.assign(nm, 1);
    p->decomp_f.assign(nm, -1);
    if (op == PM_OP_COUNT)
        for (size_t j = 0; j < nm; j++) p->decomp_f[j] = decomp_formula(p->morph.matched[j]);
    if (op == PM_OP_SUPPORT) {
        // query columns -> bitset sources
        p->col_off.push_back(0);
        for (size_t i = 0; i < p->morph.mni_sources.size(); i++) {
            p->query_col_base.push_back(int(p->col_off.size()) - 1);
            for (auto &srcs : p->morph.mni_sources[i]) {
                for (auto &pr : srcs) p->col_src.push_back(p->dom_base[pr.first] + pr.second);
                p->col_off.push_back(int32_t(p->col_src.size()));
            }
        }
    }
    *out = p;
    return PM_OK;
}

pm_status pm_plan_get_info(const pm_query_plan *p, pm_plan_info *out) {
    if (!p || !out) return PM_EINVAL;
    out->n_queries = int32_t(p->morph.queries.size());
    out->n_matched = int32_t(p->morph.matched.size());
    out->n_kernels_plans = int32_t(p->rooted.size());
    out->op = p->op;
    return PM_OK;
}

pm_status pm_plan_matched(const pm_query_plan *p, pm_pattern *out) {
    if (!p || !out) return PM_EINVAL;
    for (size_t j = 0; j < p->morph.matched.size(); j++) {
        const Pat &q = p->morph.matched[j];
        pm_pattern r{};
        r.k = q.k;
        r.edge_mask = q.mask();
        for (int u = 0; u < PM_MAX_K; u++) r.label[u] = u < q.k ? q.lab[u] : -1;
        r.induced = q.vi ? PM_VERTEX_INDUCED : PM_EDGE_INDUCED;
        out[j] = r;
    }
    return PM_OK;
}

pm_status pm_plan_export(const pm_query_plan *p, int32_t family, void *out, int64_t cap) {
    static_assert(sizeof(DevPlan) == 112, "plan record layout is part of the ABI");
    static_assert(offsetof(DevPlan, lv) == 48, "plan record layout is part of the ABI");
    if (!p || !out || (family != PM_PLANS_ROOTED && family != PM_PLANS_FREE)) return PM_EINVAL;
    const std::vector<DevPlan> &v = family == PM_PLANS_FREE ? p->free_plans : p->rooted;
    const int64_t need = int64_t(sizeof(DevPlan) * v.size());
    if (cap < need) {
        set_error("pm_plan_export: buffer too small");
        return PM_EINVAL;
    }
    std::memcpy(out, v.data(), size_t(need));
    return PM_OK;
}

pm_status pm_plan_set_launch(pm_query_plan *p, int32_t mode) {
    if (!p || (mode != PM_LAUNCH_PER_PATTERN && mode != PM_LAUNCH_SINGLE)) return PM_EINVAL;
    if (p->graph_exec || p->graph_each) {
        set_error("pm_plan_set_launch: the plan was already captured");
        return PM_EINVAL;
    }
    p->launch_mode = mode;
    return PM_OK;
}

pm_status pm_plan_select(pm_query_plan *p, int32_t family) {
    if (!p || family < PM_PLANS_AUTO || family > PM_PLANS_DECOMP) return PM_EINVAL;
    p->forced = family;
    std::fill(p->choice.begin(), p->choice.end(), -1);
    return PM_OK;
}

pm_status pm_plan_autotune(pm_query_plan *p, void *stream, int32_t *families) {
    if (!p) return PM_EINVAL;
    if (!p->g) {
        set_error("pm_plan_autotune: plan was made without a graph");
        return PM_EINVAL;
    }
    DeviceGuard dg(p->g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    if (st != PM_OK) return st;
    st = autotune(p, (cudaStream_t)stream);
    if (st != PM_OK) return st;
    if (families)
        for (size_t j = 0; j < p->choice.size(); j++) families[j] = p->choice[j];
    return PM_OK;
}

pm_status pm_plan_last_kernel_ms(const pm_query_plan *p, float *ms) {
    if (!p || !ms) return PM_EINVAL;
    *ms = 0.f;
    if (!p->timed) return PM_OK;
    cudaError_t e = cudaEventElapsedTime(ms, p->ev0, p->ev1);
    if (e) return cuda_fail("pm_plan_last_kernel_ms", e);
    return PM_OK;
}

pm_status pm_plan_pattern_bytes(const pm_query_plan *p, uint64_t *bytes) {
    if (!p || !bytes) return PM_EINVAL;
    for (size_t j = 0; j < p->morph.matched.size(); j++)
        bytes[j] = j < p->pat_bytes.size() ? p->pat_bytes[j] : 0;
    return PM_OK;
}

pm_status pm_plan_last_launches(const pm_query_plan *p, int64_t *launches) {
    if (!p || !launches) return PM_EINVAL;
    *launches = p->launches;
    return PM_OK;
}

pm_status pm_plan_pattern_ms(const pm_query_plan *p, float *ms) {
    if (!p || !ms) return PM_EINVAL;
    for (size_t j = 0; j < p->morph.matched.size(); j++) {
        ms[j] = 0.f;
        if (j < p->pat_recorded.size() && p->pat_recorded[j]) {
            cudaError_t e = cudaEventElapsedTime(&ms[j], p->pat_ev[2 * j], p->pat_ev[2 * j + 1]);
            if (e) return cuda_fail("pm_plan_pattern_ms", e);
        }
    }
    return PM_OK;
}

void pm_free_plan(pm_query_plan *p) {
    if (!p) return;
    if (p->g && p->device_ready) {
        DeviceGuard dg(p->g->device);
        free_plan_device(p);
    }
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph_each) cudaGraphExecDestroy(p->graph_each);
    if (p->h_pinned) cudaFreeHost(p->h_pinned);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (cudaEvent_t ev : p->pat_ev)
        if (ev) cudaEventDestroy(ev);
    delete p;
}

pm_status pm_morph(const pm_query_plan *p, const uint64_t *matched, uint64_t *requested) {
    if (!p || !matched || !requested) return PM_EINVAL;
    for (size_t i = 0; i < p->morph.terms.size(); i++) {
        unsigned __int128 acc = 0;
        for (const Term &t : p->morph.terms[i]) {
            unsigned __int128 v;
            u128_from_words(matched + 2 * t.matched, &v);
            acc += (unsigned __int128)(__int128)t.coef * v;   // arithmetic modulo 2^128
        }
        requested[2 * i] = uint64_t(acc);
        requested[2 * i + 1] = uint64_t(acc >> 64);
    }
    return PM_OK;
}

pm_status pm_count(pm_query_plan *p, void *stream, double timeout_s, uint64_t *counts,
                   uint64_t *matched) {
    if (p && p->graph_exec) {
        if (!counts) return PM_EINVAL;
        DeviceGuard dg(p->g->device);
        cudaStream_t s = (cudaStream_t)stream;
        cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail("pm_count (graph replay)", e);
        const size_t nm = p->morph.matched.size();
        Control ctl;
        std::memcpy(&ctl, p->h_pinned + 2 * nm, sizeof(Control));
        if (ctl.status == 1) {
            rezero_wedge(p, s);
            cudaStreamSynchronize(s);
            set_error("pm_count: deadline expired");
            return PM_ETIMEOUT;
        }
        if (ctl.fault) return list_fault("pm_count (graph replay)", ctl.fault);
        p->timed = true;
        if (matched) std::memcpy(matched, p->h_pinned, sizeof(uint64_t) * 2 * nm);
        (void)timeout_s;
        return pm_morph(p, p->h_pinned, counts);
    }
    return run_count(p, stream, timeout_s, nullptr, 0, false, counts, matched);
}

// pm_count (each = false) or pm_count_each (each = true) recorded as one
// CUDA graph; every allocation and the autotuning happen before capture.
static pm_status capture_impl(pm_query_plan *p, void *stream, double timeout_s, double per_pattern_s,
                              bool each) {
    const char *who = each ? "pm_plan_capture_each" : "pm_plan_capture";
    if (!p || !p->g) {
        set_error(std::string(who) + ": plan without a graph");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_COUNT) {
        set_error(std::string(who) + ": counting plans only");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    cudaStream_t user = (cudaStream_t)stream;
    pm_status st = ensure_device(p);
    if (st == PM_OK) st = prepare_active(p, user);
    if (st != PM_OK) return st;
    bool needs_wedge = false, needs_clique = false;
    for (const DevPlan &dp : p->active.plans) {
        needs_wedge |= dp.kind == PLAN_WEDGE_PAIRS;
        needs_clique |= dp.kind == PLAN_CLIQUE;
    }
    if (needs_wedge) {
        st = ensure_wedge(p, user);
        if (st != PM_OK) return st;
    }
    if (needs_clique) {
        st = ensure_clique(p);
        if (st != PM_OK) return st;
    }
    if (!p->decomp_targets.empty()) {
        st = ensure_decomp(p, user);
        if (st != PM_OK) return st;
    }
    const size_t nm = p->morph.matched.size();
    if (each && !p->d_timed_out) {
        p->d_timed_out = (uint8_t *)dev_alloc(std::max<size_t>(nm, 1), g->device);
        if (!p->d_timed_out) return PM_ENOMEM;
    }
    if (each && p->launch_mode == PM_LAUNCH_SINGLE && !p->active.plans.empty() &&
        (!p->d_plan_done || p->plan_done_cap < p->active.plans.size())) {
        dev_free(p->d_plan_done, sizeof(unsigned int) * 3 * p->plan_done_cap, g->device);
        p->plan_done_cap = p->active.plans.size();
        p->d_plan_done = (unsigned int *)dev_alloc(sizeof(unsigned int) * 3 * p->plan_done_cap, g->device);
        if (!p->d_plan_done) {
            p->plan_done_cap = 0;
            return PM_ENOMEM;
        }
    }
    if (!p->h_pinned) {
        // counters, the control block, then the per-pattern expiry flags
        cudaError_t e = cudaMallocHost(&p->h_pinned, sizeof(uint64_t) * 2 * nm + sizeof(Control) + nm + 8);
        if (e) return cuda_fail(who, e);
    }
    cudaError_t e = cudaStreamSynchronize(user);
    if (e) return cuda_fail(who, e);
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) return cuda_fail(who, e);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (!e) {
        const DevTasks tasks = all_tasks(g);
        cudaMemsetAsync(p->d_counters, 0, p->bytes_counters, cs);
        if (each) cudaMemsetAsync(p->d_timed_out, 0, std::max<size_t>(nm, 1), cs);
        const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
        const uint64_t per = each && per_pattern_s > 0 ? uint64_t(per_pattern_s * 1e9) : 0;
        p->launches = 1;
        launch_arm(p->d_ctl, budget, cs);
        cudaEventRecord(p->ev0, cs);
        st = launch_table(p, p->active, tasks, 1, false, nullptr, cs, per,
                          each ? p->d_timed_out : nullptr, true, true);
        cudaEventRecord(p->ev1, cs);
        cudaMemcpyAsync(p->h_pinned, p->d_counters, sizeof(uint64_t) * 2 * nm,
                        cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(p->h_pinned + 2 * nm, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, cs);
        if (each)
            cudaMemcpyAsync(reinterpret_cast<uint8_t *>(p->h_pinned + 2 * nm) + sizeof(Control),
                            p->d_timed_out, nm, cudaMemcpyDeviceToHost, cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    cudaStreamDestroy(cs);
    if (st != PM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e) return cuda_fail(who, e);
    cudaGraphExec_t &slot = each ? p->graph_each : p->graph_exec;
    if (slot) cudaGraphExecDestroy(slot);
    e = cudaGraphInstantiate(&slot, graph, 0);
    cudaGraphDestroy(graph);
    if (e) {
        slot = nullptr;
        return cuda_fail(who, e);
    }
    return PM_OK;
}

pm_status pm_plan_capture(pm_query_plan *p, void *stream, double timeout_s) {
    return capture_impl(p, stream, timeout_s, 0.0, false);
}

pm_status pm_plan_capture_each(pm_query_plan *p, void *stream, double timeout_per_pattern_s,
                               double timeout_total_s) {
    return capture_impl(p, stream, timeout_total_s, timeout_per_pattern_s, true);
}

pm_status pm_count_roots(pm_query_plan *p, void *stream, double timeout_s, const int32_t *roots,
                         int64_t nroots, uint64_t *counts, uint64_t *matched) {
    if ((!roots && nroots > 0) || nroots < 0) {
        set_error("pm_count_roots: bad root list");
        return PM_EINVAL;
    }
    static const int32_t none = 0;
    return run_count(p, stream, timeout_s, roots ? roots : &none, nroots, true, counts, matched);
}

pm_status pm_count_instrumented(pm_query_plan *p, void *stream, uint64_t *counts,
                                uint64_t *alg_bytes) {
    if (!alg_bytes) {
        set_error("pm_count_instrumented: null alg_bytes");
        return PM_EINVAL;
    }
    return run_count(p, stream, 0.0, nullptr, 0, false, counts, nullptr, alg_bytes);
}

// The graph's caller-to-internal vertex map on the device (uploaded once).
static pm_status ensure_new_id(const pm_graph *g) {
    std::lock_guard<std::mutex> lk(g->new_id_mu);
    if (g->d_new_id) return PM_OK;
    g->d_new_id = (int32_t *)dev_alloc(sizeof(int32_t) * size_t(g->n), g->device);
    if (!g->d_new_id) {
        set_error("device allocation failed (vertex map)");
        return PM_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(g->d_new_id, g->new_id.data(), sizeof(int32_t) * size_t(g->n),
                               cudaMemcpyHostToDevice);
    if (e) return cuda_fail("vertex map upload", e);
    return PM_OK;
}

pm_status pm_support_roots(pm_query_plan *p, void *stream, double timeout_s, const int32_t *roots,
                           int64_t nroots, uint32_t *domains_dev) {
    if (!p || !domains_dev || (!roots && nroots > 0) || nroots < 0) {
        set_error("pm_support_roots: null argument or bad root list");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_SUPPORT || !p->g) {
        set_error("pm_support_roots: needs a PM_OP_SUPPORT plan made on a graph");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    if (st == PM_OK) st = ensure_new_id(g);
    if (st != PM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    static const int32_t none = 0;
    RootTasks rt;
    DevTasks tasks;
    st = root_tasks(g, roots ? roots : &none, nroots, s, rt, &tasks);
    if (st != PM_OK) return st;
    if (p->rooted_table.dirty) p->rooted_table.plans = p->rooted;
    st = upload_table(p->rooted_table, g->device);
    if (st != PM_OK) return st;
    const size_t ncols = p->col_off.size() - 1;
    cudaError_t e = cudaMemsetAsync(p->d_bitsets, 0, p->bytes_bitsets, s);
    if (e) return cuda_fail("pm_support_roots: memset", e);
    const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
    if (launch_arm(p->d_ctl, budget, s)) return PM_ECUDA;
    st = launch_table(p, p->rooted_table, tasks, 1, true, nullptr, s);
    if (st != PM_OK) return st;
    if (launch_mni_domains(p->d_bitsets, p->words, p->d_col_off, p->d_col_src, int(ncols),
                           g->d_new_id, g->n, domains_dev, s))
        return PM_ECUDA;
    Control ctl;
    e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail("pm_support_roots: kernel or readback", e);
    if (ctl.status == 1) {
        set_error("pm_support_roots: deadline expired");
        return PM_ETIMEOUT;
    }
    return PM_OK;
}

pm_status pm_domains_or(const uint32_t *parts_dev, int32_t n_parts, int64_t words, uint32_t *out_dev,
                        void *stream) {
    if (!parts_dev || !out_dev || n_parts < 1 || words < 0) {
        set_error("pm_domains_or: null pointer or empty input");
        return PM_EINVAL;
    }
    if (words == 0) return PM_OK;
    if (launch_domains_or(parts_dev, n_parts, words, out_dev, stream)) {
        set_error("pm_domains_or: launch failed");
        return PM_ECUDA;
    }
    return PM_OK;
}

pm_status pm_support_from_domains(pm_query_plan *p, const uint32_t *domains_dev, void *stream,
                                  uint64_t threshold, uint64_t *support, uint8_t *frequent) {
    if (!p || !domains_dev || !support) {
        set_error("pm_support_from_domains: null argument");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_SUPPORT || !p->g) {
        set_error("pm_support_from_domains: needs a PM_OP_SUPPORT plan made on a graph");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    if (st != PM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ncols = p->col_off.size() - 1;
    const int64_t words = (g->n + 31) / 32;
    cudaError_t e = cudaMemsetAsync(p->d_popc, 0, sizeof(unsigned long long) * std::max<size_t>(ncols, 1), s);
    if (e) return cuda_fail("pm_support_from_domains: memset", e);
    if (launch_column_popc(domains_dev, words, int(ncols), p->d_popc, s)) return PM_ECUDA;
    std::vector<unsigned long long> popc(ncols);
    e = ncols ? cudaMemcpyAsync(popc.data(), p->d_popc, sizeof(unsigned long long) * ncols,
                                cudaMemcpyDeviceToHost, s) : cudaSuccess;
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail("pm_support_from_domains: readback", e);
    const size_t nq = p->morph.queries.size();
    for (size_t i = 0; i < nq; i++) {
        const int c0 = p->query_col_base[i];
        const int c1 = (i + 1 < nq) ? p->query_col_base[i + 1] : int(ncols);
        uint64_t best = UINT64_MAX;
        for (int c = c0; c < c1; c++) best = std::min<uint64_t>(best, popc[c]);
        support[i] = best == UINT64_MAX ? 0 : best;
        if (frequent) frequent[i] = support[i] >= threshold ? 1 : 0;
    }
    return PM_OK;
}

// Listing through Theorem 3.1 (Section 3.2.1): the edge-induced matches of
// p are the vertex-induced matches of p and of its superpatterns q, each
// composed with the maps phi(p^E, q^E); one map per distinct image edge set
// (c(p, q) of them) lists every distinct occurrence of p exactly once, the
// union over q being disjoint (Corollary 3.1).  A vertex-induced query is
// listed directly.  Listing plans are the free plans with every level
// enumerated (one match per occurrence, symmetry broken).
pm_status pm_enumerate(pm_query_plan *p, void *stream, double timeout_s, int32_t *tuples,
                       int32_t *query_of, int64_t cap, int64_t *n_out) {
    if (!p || !n_out || (cap > 0 && !tuples) || cap < 0) {
        set_error("pm_enumerate: null argument");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_COUNT || !p->g) {
        set_error("pm_enumerate: needs a counting plan made on a graph");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    const size_t nq = p->morph.queries.size(), nm = p->morph.matched.size();
    // maps per matched pattern: (query, f) with f[u] = vertex of the matched
    // pattern that vertex u of the query goes to
    std::vector<std::vector<std::pair<int, Perm>>> maps(nm);
    for (size_t i = 0; i < nq; i++)
        for (const Term &t : p->morph.terms[i])
            if (t.coef <= 0) {
                set_error("pm_enumerate: a vertex-induced query morphed to edge-induced patterns "
                          "(Corollary 3.1 subtracts) cannot be listed; plan it with PM_MORPH_NONE");
                return PM_EUNSUPPORTED;
            }
    for (size_t i = 0; i < nq; i++) {
        Pat q = p->morph.queries[i];
        if (q.is_clique()) q.vi = false;
        for (const Term &t : p->morph.terms[i]) {
            const Pat &mq = p->morph.matched[t.matched];
            std::vector<Perm> fs;
            if (q.vi) {
                // a vertex-induced query is matched as itself (canonical numbering)
                fs = embeddings(q, mq);
                if (!fs.empty()) fs.resize(1);
            } else {
                Pat pe = q, me = mq;
                pe.vi = me.vi = false;
                std::vector<Perm> all = embeddings(pe, me);
                std::vector<uint64_t> seen;
                for (const Perm &f : all) {
                    uint64_t img = 0;   // image edge set of the query's edges
                    for (int a = 0; a < q.k; a++)
                        for (int b = a + 1; b < q.k; b++)
                            if (q.adjacent(a, b)) {
                                const int x = std::min(f[a], f[b]), y = std::max(f[a], f[b]);
                                img |= uint64_t(1) << (x * PM_MAX_K + y);
                            }
                    if (std::find(seen.begin(), seen.end(), img) == seen.end()) {
                        seen.push_back(img);
                        fs.push_back(f);
                    }
                }
            }
            if (int64_t(fs.size()) != t.coef) {
                set_error("pm_enumerate: internal error (maps do not match the morph coefficient)");
                return PM_EUNSUPPORTED;
            }
            for (const Perm &f : fs) maps[t.matched].push_back({int(i), f});
        }
    }
    // exact sizes from a count
    std::vector<uint64_t> req(2 * nq), mat(2 * nm);
    pm_status st = run_count(p, stream, timeout_s, nullptr, 0, false, req.data(), mat.data());
    if (st != PM_OK) return st;
    int64_t listed = 0, needed = 0;
    for (size_t j = 0; j < nm; j++) {
        if (mat[2 * j + 1]) {
            set_error("pm_enumerate: more matches than can be listed");
            return PM_EOVERFLOW;
        }
        listed += int64_t(mat[2 * j]);
        needed += int64_t(mat[2 * j]) * int64_t(maps[j].size());
    }
    *n_out = needed;
    if (needed > cap) {
        set_error("pm_enumerate: cap too small (*n_out holds the number of occurrences)");
        return PM_EOVERFLOW;
    }
    if (needed == 0) return PM_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // listing plans
    PlanTable table;
    for (size_t j = 0; j < nm; j++) {
        DevPlan dp = compile_free_plan(p->morph.matched[j], int(j), 0, p->morph.matched_orbit[j], false);
        if (dp.k >= 3) {
            dp.tail = 1;
            dp.n_enum = dp.k - 1;
        }
        dp.closed = 0;
        dp.pair = 0;
        table.plans.push_back(dp);
    }
    st = upload_table(table, g->device);
    if (st != PM_OK) return st;
    std::vector<int32_t> old_of(g->n), map_off(nm + 1, 0), map_query, query_k(nq);
    std::vector<uint8_t> map_f;
    for (int64_t v = 0; v < g->n; v++) old_of[g->new_id[v]] = int32_t(v);
    for (size_t j = 0; j < nm; j++) {
        for (auto &qf : maps[j]) {
            map_query.push_back(qf.first);
            for (int u = 0; u < PM_MAX_K; u++) map_f.push_back(qf.second[u]);
        }
        map_off[j + 1] = int32_t(map_query.size());
    }
    for (size_t i = 0; i < nq; i++) query_k[i] = p->morph.queries[i].k;
    // device buffers: listed matches (tuple + tag), output (tuple + query),
    // cursors, maps, the vertex map
    const size_t b_q = sizeof(int32_t) * size_t(listed) * (PM_MAX_K + 1);
    const size_t b_o = sizeof(int32_t) * size_t(needed) * (PM_MAX_K + 1);
    const size_t b_aux = sizeof(int32_t) * (size_t(g->n) + map_off.size() + map_query.size() + nq) +
                         map_f.size() + 64;
    char *dq = (char *)dev_alloc(b_q, g->device);
    char *dout = (char *)dev_alloc(b_o, g->device);
    char *daux = (char *)dev_alloc(b_aux, g->device);
    auto release = [&]() {
        dev_free(dq, b_q, g->device);
        dev_free(dout, b_o, g->device);
        dev_free(daux, b_aux, g->device);
        free_table(table, g->device);
    };
    if (!dq || !dout || !daux) {
        release();
        set_error("pm_enumerate: device allocation failed");
        return PM_ENOMEM;
    }
    int32_t *q_t = (int32_t *)dq, *q_tag = q_t + size_t(listed) * PM_MAX_K;
    int32_t *o_t = (int32_t *)dout, *o_q = o_t + size_t(needed) * PM_MAX_K;
    unsigned long long *cur = (unsigned long long *)daux;               // two cursors
    int32_t *d_old = (int32_t *)(daux + 16);
    int32_t *d_moff = d_old + g->n;
    int32_t *d_mq = d_moff + map_off.size();
    int32_t *d_qk = d_mq + map_query.size();
    uint8_t *d_mf = (uint8_t *)(d_qk + nq);
    cudaError_t e = cudaMemsetAsync(cur, 0, 16, s);
    if (!e) e = cudaMemcpyAsync(d_old, old_of.data(), sizeof(int32_t) * g->n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_moff, map_off.data(), sizeof(int32_t) * map_off.size(), cudaMemcpyHostToDevice, s);
    if (!e && !map_query.empty())
        e = cudaMemcpyAsync(d_mq, map_query.data(), sizeof(int32_t) * map_query.size(), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_qk, query_k.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s);
    if (!e && !map_f.empty()) e = cudaMemcpyAsync(d_mf, map_f.data(), map_f.size(), cudaMemcpyHostToDevice, s);
    if (e) {
        release();
        return cuda_fail("pm_enumerate: upload", e);
    }
    const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
    MatchLaunch L{};
    const DevTasks tasks = all_tasks(g);
    L.g = g->dev();
    L.plans = table.d;
    L.nplans = int(table.plans.size());
    L.max_enum = table.max_enum;
    L.tasks = tasks;
    L.n_echunks = echunks_for(table.plans, tasks);
    L.sample_stride = 1;
    L.counters = p->d_counters;
    L.ctl = p->d_ctl;
    L.defer = p->d_defer;
    L.defer_cap = p->defer_cap;
    L.piece_off = p->d_piece_off;
    L.list_out = q_t;
    L.list_tag = q_tag;
    L.list_cursor = cur;
    L.list_cap = listed;
    L.old_of = d_old;
    int rc = launch_arm(p->d_ctl, budget, s);
    if (!rc && L.n_echunks > 0) rc = launch_list(L, s);
    if (!rc) rc = launch_compose(q_t, q_tag, listed, d_moff, d_mq, d_mf, d_qk, o_t, o_q, cur + 1, needed, s);
    if (rc) {
        release();
        return PM_ECUDA;
    }
    unsigned long long cursors[2] = {0, 0};
    Control ctl;
    e = cudaMemcpyAsync(cursors, cur, 16, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(tuples, o_t, sizeof(int32_t) * size_t(needed) * PM_MAX_K,
                                cudaMemcpyDeviceToHost, s);
    if (!e && query_of) e = cudaMemcpyAsync(query_of, o_q, sizeof(int32_t) * size_t(needed),
                                            cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    release();
    if (e) return cuda_fail("pm_enumerate: kernel or readback", e);
    if (ctl.status == 1) {
        set_error("pm_enumerate: deadline expired");
        return PM_ETIMEOUT;
    }
    if (int64_t(cursors[0]) != listed || int64_t(cursors[1]) != needed) {
        set_error("pm_enumerate: listed matches disagree with the count");
        return PM_ECUDA;
    }
    return PM_OK;
}

pm_status pm_plan_query_columns(const pm_query_plan *p, int32_t *columns) {
    if (!p || !columns) return PM_EINVAL;
    if (p->op != PM_OP_SUPPORT) {
        set_error("pm_plan_query_columns: plan was made for PM_OP_COUNT");
        return PM_EINVAL;
    }
    for (size_t i = 0; i < p->morph.query_columns.size(); i++)
        for (int u = 0; u < PM_MAX_K; u++)
            columns[i * PM_MAX_K + u] =
                u < int(p->morph.query_columns[i].size()) ? p->morph.query_columns[i][u] : -1;
    return PM_OK;
}

pm_status pm_support(pm_query_plan *p, void *stream, double timeout_s, uint64_t threshold,
                     uint64_t *support, uint8_t *frequent, uint32_t *domains_dev) {
    if (!p || !support) {
        set_error("pm_support: null argument");
        return PM_EINVAL;
    }
    if (p->op != PM_OP_SUPPORT) {
        set_error("pm_support: plan was made for PM_OP_COUNT");
        return PM_EINVAL;
    }
    const pm_graph *g = p->g;
    if (!g) {
        set_error("pm_support: plan was made without a graph");
        return PM_EINVAL;
    }
    DeviceGuard dg(g->device);
    if (!dg.ok) return PM_ECUDA;
    pm_status st = ensure_device(p);
    if (st != PM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_active(p, s);
    if (st != PM_OK) return st;
    const DevTasks tasks = all_tasks(g);
    const size_t ncols = p->col_off.size() - 1;
    cudaError_t e = cudaMemsetAsync(p->d_bitsets, 0, p->bytes_bitsets, s);
    if (!e) e = cudaMemsetAsync(p->d_popc, 0, sizeof(unsigned long long) * std::max<size_t>(ncols, 1), s);
    if (e) return cuda_fail("pm_support: memset", e);
    const uint64_t budget = timeout_s > 0 ? uint64_t(timeout_s * 1e9) : 0;
    if (launch_arm(p->d_ctl, budget, s)) return PM_ECUDA;
    cudaEventRecord(p->ev0, s);
    st = launch_table(p, p->active, tasks, 1, true, nullptr, s);
    if (st != PM_OK) return st;
    cudaEventRecord(p->ev1, s);
    p->timed = true;
    if (launch_mni_reduce(p->d_bitsets, p->words, p->d_col_off, p->d_col_src, int(ncols),
                          p->d_popc, s))
        return PM_ECUDA;
    if (domains_dev) {
        st = ensure_new_id(g);
        if (st != PM_OK) return st;
        if (launch_mni_domains(p->d_bitsets, p->words, p->d_col_off, p->d_col_src, int(ncols),
                               g->d_new_id, g->n, domains_dev, s))
            return PM_ECUDA;
    }
    std::vector<unsigned long long> popc(ncols);
    Control ctl;
    e = ncols ? cudaMemcpyAsync(popc.data(), p->d_popc, sizeof(unsigned long long) * ncols,
                                cudaMemcpyDeviceToHost, s) : cudaSuccess;
    if (!e) e = cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail("pm_support: kernel or readback", e);
    if (ctl.status == 1) {
        set_error("pm_support: deadline expired");
        return PM_ETIMEOUT;
    }
    const size_t nq = p->morph.queries.size();
    for (size_t i = 0; i < nq; i++) {
        const int c0 = p->query_col_base[i];
        const int c1 = (i + 1 < nq) ? p->query_col_base[i + 1] : int(ncols);
        uint64_t best = UINT64_MAX;
        for (int c = c0; c < c1; c++) best = std::min<uint64_t>(best, popc[c]);
        support[i] = best == UINT64_MAX ? 0 : best;
        if (frequent) frequent[i] = support[i] >= threshold ? 1 : 0;
    }
    return PM_OK;
}

const char *pm_strerror(pm_status s) {
    switch (s) {
        case PM_OK: return "ok";
        case PM_EINVAL: return "invalid argument";
        case PM_ENOMEM: return "out of memory";
        case PM_ECUDA: return "CUDA error";
        case PM_ETIMEOUT: return "deadline expired";
        case PM_EOVERFLOW: return "result does not fit the output width";
        case PM_EUNSUPPORTED: return "unsupported request";
        case PM_ECANCELLED: return "cancelled";
    }
    return "unknown status";
}

const char *pm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
