// Library-internal host structures behind the opaque handles of pm.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/pm.h"
#include "pattern.hpp"
#include "plan.hpp"

struct pm_graph {
    int device = 0;
    int64_t n = 0, m = 0, self_loops = 0, duplicates = 0, max_degree = 0;
    int64_t max_updeg = 0;           // most neighbours ranked above one vertex
    bool labeled = false;
    std::vector<int32_t> new_id;     // caller id -> internal id
    std::vector<int32_t> lowdeg;     // internal id -> neighbours with smaller internal id
    std::vector<uint8_t> labels;     // internal id -> label (labeled graphs)
    int64_t *d_rowptr = nullptr;
    int32_t *d_col = nullptr;
    uint8_t *d_labels = nullptr;
    int64_t *d_off[3] = {nullptr, nullptr, nullptr};  // task offsets per TaskSpace, all roots
    int32_t *d_hub = nullptr;        // hub bitmap index per vertex (-1: none)
    uint32_t *d_bits = nullptr;      // hub adjacency bitmaps
    int64_t n_hubs = 0, hub_words = 0;
    int64_t ntasks[3] = {0, 0, 0};
    size_t bytes = 0;
    // caller id -> internal id on the device, uploaded when MNI domains are
    // first returned in caller ids (pm_support with domains_dev)
    mutable std::mutex new_id_mu;
    mutable int32_t *d_new_id = nullptr;
    // Autotuner cache: canonical pattern key -> chosen plan family
    // (0 rooted, 1 free); shared by every plan made on this graph.
    mutable std::mutex tune_mu;
    mutable std::map<pm::Key, int> tuned;
    mutable std::map<pm::Key, double> tuned_ms;   // sampled time of the chosen family
    mutable std::map<pm::Key, int> tuned_split;   // chosen task granularity (split code)
    mutable std::map<int, double> decomp_ms;      // decomposition time per pass set
    pm::DevGraph dev() const {
        return pm::DevGraph{n, 2 * m, d_rowptr, d_col, d_labels,
                            n_hubs ? d_hub : nullptr, d_bits, hub_words};
    }
};

namespace pm {

// One query's result as a signed combination of matched-pattern results
// (counting), or for MNI as, per query column, the matched bitsets to OR.
struct Term {
    int matched;
    int64_t coef;
};

struct MorphPlan {
    std::vector<Pat> queries;
    std::vector<Pat> matched;
    std::vector<std::vector<Term>> terms;            // counting: per query
    // MNI (support plans)
    std::vector<int> matched_columns;                // per matched pattern: number of orbits
    std::vector<std::vector<int>> matched_orbit;     // per matched pattern: column of each vertex
    std::vector<std::vector<std::vector<std::pair<int, int>>>> mni_sources;
    // mni_sources[query][query column] = list of (matched, matched column)
    std::vector<std::vector<int>> query_columns;     // per query: column of each pattern vertex
};

// Morph selection (Section 4.1, step a).  Returns PM_OK or an error status
// with *why set.
// cost (PM_MORPH_COST only): device cost of matching one pattern as given.
pm_status morph_select(const std::vector<Pat> &queries, pm_op op, pm_morph_mode mode,
                       MorphPlan &out, std::string *why,
                       const std::function<double(const Pat &)> *cost = nullptr);

// Size of the alternative set of a query set (morph selection only).
pm_status matched_set_size(const pm_graph *g, const pm_pattern *queries, int32_t nq,
                           pm_morph_mode mode, int32_t *n_matched);

// Rooted matching plans of one pattern (one per automorphism orbit).
// counting: the plans serve pm_count (a 4-cycle may then use the wedge kernel).
std::vector<DevPlan> compile_plans(const Pat &p, int counter, int dom_base,
                                   const std::vector<int> &column_of_vertex, bool counting);
// The free matching plan of one pattern (whole automorphism group broken).
DevPlan compile_free_plan(const Pat &p, int counter, int dom_base,
                          const std::vector<int> &column_of_vertex, bool counting);

// Device memory through the configured allocator.
void *dev_alloc(size_t bytes, int device);
void dev_free(void *ptr, size_t bytes, int device);

void set_error(const std::string &msg);

// Graph preparation on the device (graph_dev.cu): zeroes d_bits and fills
// the nh adjacency bitmaps (words 32-bit words each) of internal vertices
// n-1, ..., n-nh from the device CSR, and d_hub[r] = n-1-r for those ranks,
// -1 for the others; asynchronous on the stream.  Returns a cudaError_t
// value (0 on success).
int launch_hub_bitmaps(const int64_t *d_rowptr, const int32_t *d_col, int64_t n, int64_t nh,
                       int64_t words, int32_t *d_hub, uint32_t *d_bits, void *stream);

// Kernel launchers (match.cu).
// Resets the control block and arms the deadline (budget_ns = 0: none).
int launch_arm(Control *d_ctl, uint64_t budget_ns, void *stream);
// Resets the work counters, keeping the status and deadline.
int launch_rearm(Control *d_ctl, void *stream);
// Per-pattern deadlines: flag pattern prev_counter (>= 0) if its deadline
// expired, then reset the status and counters and arm budget_ns.
int launch_pattern_gate(Control *d_ctl, uint8_t *d_timed_out, int prev_counter,
                        uint64_t budget_ns, void *stream);
// One matching launch (both passes).  max_enum: largest n_enum over the
// plans (sizes the per-warp level buffers); stats (nullable): instrumented
// run adding the algorithmic bytes read.
struct MatchLaunch {
    DevGraph g;
    const DevPlan *plans;
    int nplans;
    int max_enum;
    DevTasks tasks;
    int64_t n_echunks;         // 32-task chunks per plan (largest task space in the launch)
    int32_t sample_stride;     // 1 = every chunk; s > 1 = every s-th chunk (autotuning)
    uint64_t *counters;        // counting
    uint32_t *bitsets;         // MNI domains
    int64_t words;
    Control *ctl;
    Deferred *defer;
    uint32_t defer_cap;
    uint32_t *piece_off;
    unsigned long long *stats;
    // listing (launch_list): output tuples, their tags, the shared cursor,
    // capacity in tuples, internal -> caller id map
    int32_t *list_out;
    int32_t *list_tag;
    unsigned long long *list_cursor;
    int64_t list_cap;
    const int32_t *old_of;
    unsigned int *plan_done;   // per-plan progress (3 x nplans, zeroed), or nullptr
};
int launch_plan_flags(Control *ctl, const DevPlan *plans, int nplans, const unsigned int *plan_done,
                      unsigned long long n_chunks, uint8_t *timed_out, void *stream);
int launch_count(const MatchLaunch &L, void *stream);
int launch_list(const MatchLaunch &L, void *stream);
int launch_compose(const int32_t *qt, const int32_t *qtag, int64_t n_listed, const int32_t *map_off,
                   const int32_t *map_query, const uint8_t *map_f, const int32_t *query_k, int32_t *out,
                   int32_t *out_query, unsigned long long *cursor, int64_t cap, void *stream);
int launch_domains(const MatchLaunch &L, void *stream);
// Wedge-pair kernels for one PLAN_WEDGE_PAIRS plan over the lower task space
// of `tasks`: roots a >= heavy_from by the shared-memory heavy-root kernel
// (lists: blocks * 2 * list_cap (cursor, end) pairs, list_cap >= the largest
// degree), the others with dense counters in scratch (blocks * n uint32,
// zero on entry and exit; unused when heavy_from == 0).
int wedge_blocks(int device);
int launch_wedge_pairs(const DevGraph &g, const DevTasks &tasks, int64_t heavy_from, int counter,
                       uint64_t *counters, uint32_t *scratch, uint2 *lists, int64_t list_cap,
                       int blocks, int sample_stride, Control *ctl, void *stream);
// Clique kernel (clique.cu) for one PLAN_CLIQUE plan (k = 4 or 5) over the
// lower task space of `tasks`.  spill: clique_warps(device) * 2 * spill_len
// int32 entries, where spill_len = clique_spill_len(max degree); nullptr is
// allowed only when that length is 0.  stats (nullable): add the algorithmic
// bytes read.
int64_t clique_warps(int device);
int64_t clique_spill_len(int64_t max_degree);
int launch_clique(const DevGraph &g, const DevTasks &tasks, int k, int counter,
                  uint64_t *counters, int32_t *spill, int64_t spill_len, int sample_stride,
                  Control *ctl, unsigned long long *stats, void *stream,
                  uint64_t *deg_out = nullptr);

// Edge-induced counts from local statistics (decomp.cu).  Sums (128-bit,
// 2 words each, DB_COUNT entries) accumulated by the passes:
enum DecompSum : int {
    DB_TRI, DB_K4, DB_K5, DB_K4DEG3, DB_K5P3, DB_DE, DB_C4,
    DB_STAR3, DB_STAR4, DB_P4E, DB_TX3, DB_PAW, DB_FORK, DB_P5A, DB_TVD, DB_CRICKET,
    DB_LOLLI_V, DB_BOWTIE_V, DB_BULL, DB_LOLLI_E, DB_KITE, DB_DART_E, DB_BOOK,
    DB_C5TRI, DB_DART_TRI, DB_GEM_TRI, DB_BANNER2, DB_HOUSE, DB_C5Q, DB_C5CORR, DB_C5TM,
    DB_K23I, DB_W4, DB_K23, DB_K23E, DB_K5E, DB_COUNT
};
// The patterns counted this way (unlabeled, edge-induced).
enum DecompFormula : int {
    DF_STAR3, DF_P4, DF_PAW, DF_DIAMOND,                       // 4 vertices
    DF_STAR4, DF_FORK, DF_P5, DF_CRICKET, DF_BULL, DF_LOLLIPOP, DF_BANNER, DF_C5, DF_KITE,
    DF_DART, DF_BOWTIE, DF_HOUSE, DF_BOOK, DF_GEM, DF_K4PENDANT,   // 5 vertices
    DF_K4, DF_K5, DF_K5P3,                                         // cliques, K5 minus a 2-path
    DF_W4, DF_K23, DF_K23E,                     // 4-wheel, K2,3, K2,3 plus an edge in its 3-side
    DF_K5E,                                     // K5 minus an edge
    DF_COUNT
};
// Passes beyond triangle pass 1, the mirror and the vertex/edge pass:
// triangle pass 2, 2-path pass (with the 5-cycle scan), out-neighbourhood
// bitmaps (4-cliques; 5-cliques; 4-cliques per edge), neighbourhood graphs
// (common-neighbour lists with the 4-wheel pass; with the K2,3 root pass).
enum DecompPass : int {
    DP_TRI2 = 1, DP_PATHS = 2, DP_C5 = 4, DP_LOCAL = 8, DP_K5 = 16, DP_K4E = 32,
    DP_W4 = 64, DP_K23E = 128, DP_K5E = 256,
    DP_WHEEL = DP_W4 | DP_K23E | DP_K5E        // passes that need the common-neighbour lists
};
// Neighbourhood-graph pass (wheel.cu).
struct WheelArgs {
    DevGraph g;
    const int32_t *t;         // triangles per CSR slot (both endpoints' rows)
    int64_t *toff;            // nnz + 1 list offsets (exclusive scan of t)
    int32_t *T;               // common-neighbour lists, positions in the slot's own row
    int64_t T_len;            // entries allocated for T (bounds checks of the PM_DEBUG build)
    int64_t *bsum;            // scan scratch: one word per 8192 slots
    int32_t *hub_rank;        // popcount rank index of the hub bitmaps, or nullptr
    int64_t n_hubs;
    int32_t *mpos;            // DP_K23E: per slot (v, u), v's position in u's row
    uint32_t *gcnt;           // DP_W4: per block 32-bit counters above 65536 positions, or nullptr
    int64_t gcnt_words;
    int w4_blocks;
    uint32_t *kW;             // DP_K23E: per block n 2-path counters (zero on entry and exit)
    unsigned long long *kE;   // per block n diamond counters (zero on entry and exit)
    int32_t *ktouched;        // per block n touched vertices
    int k23_blocks;
    int k23_narrow;           // largest degree < 65536: 16-bit 2-path and 32-bit diamond counters
    uint32_t *k5g;            // DP_K5E: per warp 32-bit counters above 2048 positions, or nullptr
    int64_t k5g_words;
    int k5e_blocks;
    uint64_t *basis;
    Control *ctl;
    unsigned long long *stats;   // nullable: algorithmic bytes
};
size_t w4_smem_bytes();
int w4_blocks(int device);
int k23_blocks(int device);
int k5e_blocks(int device);
int64_t k5e_global_words(int64_t max_updeg, int64_t max_degree);
int64_t w4_global_words(int64_t max_degree);
int64_t tscan_blocks(int64_t nnz);
int launch_wheel(const WheelArgs &A, int passes, void *stream);
int launch_list_offsets(const WheelArgs &A, void *stream);
int wheel_launches(const WheelArgs &A, int passes);
// Out-neighbourhood bitmap pass (local.cu).
struct LocalArgs {
    DevGraph g;
    const int64_t *low_off;   // lower-neighbour task offsets over the implicit roots n-1..0
    uint32_t *k4e;            // 4-cliques per edge at its slot in the lower endpoint's row, or nullptr
    uint64_t *basis;
    Control *ctl;
    uint32_t *grows;          // per block: rows of neighbourhoods above the shared-memory size
    int32_t *gmem;            // per block: their members (max_s entries)
    uint32_t *gts;            // per block: their per-member triangle sums (max_s entries)
    int64_t grow_words;
    int64_t max_s;
    int want_k5;
    unsigned long long *stats;   // nullable: algorithmic bytes
};
size_t local_smem_bytes();
int local_blocks(int device);
int64_t local_grow_words(int64_t max_s);
int launch_local(const LocalArgs &A, int blocks, void *stream);
// formula of an unlabeled edge-induced pattern, or -1 (morph.cpp)
int decomp_formula(const Pat &p);
int decomp_passes(int formula);
struct DecompLaunch {
    DevGraph g;
    DevTasks tasks;           // lower-neighbour tasks over every root
    int passes;
    int32_t *t;               // one int32 per CSR slot
    uint32_t *k4e;            // one uint32 per CSR slot (DP_K4E), or nullptr
    LocalArgs local;          // DP_LOCAL: scratch of the bitmap pass
    int local_blocks;
    WheelArgs wheel;          // DP_W4 | DP_K23E: lists and counters of the neighbourhood-graph pass
    uint32_t *W;              // path_blocks x n (zero on entry and exit)
    int32_t *touched;         // path_blocks x n
    int path_blocks;
    uint64_t *basis;          // 2 x DB_COUNT words
    Control *ctl;
    unsigned long long *stats;   // nullable: algorithmic bytes of every pass
};
int decomp_path_blocks(int device);
int launch_decomp(const DecompLaunch &L, void *stream);
// triangle pass 1 and the mirror only: t for every slot (list sizes)
int launch_decomp_triangles(const DecompLaunch &L, void *stream);
int launch_flag_targets(Control *ctl, uint8_t *timed_out, const int32_t *targets, int n_targets,
                        void *stream);
int launch_decomp_combine(const uint64_t *basis, const int32_t *targets, int n_targets,
                          uint64_t *counters, void *stream);
int launch_mni_reduce(const uint32_t *d_bitsets, int64_t words_per_bitset, const int32_t *d_src_off,
                      const int32_t *d_src, int n_columns, unsigned long long *d_popc,
                      void *stream);
int launch_domains_or(const uint32_t *parts, int n_parts, int64_t words, uint32_t *out, void *stream);
int launch_column_popc(const uint32_t *cols, int64_t words, int n_columns, unsigned long long *popc,
                       void *stream);
// Query columns as n-bit bitsets in caller vertex ids: bit v of column c of
// out (words_per_bitset words each) = bit new_id[v] of the OR of c's sources.
int launch_mni_domains(const uint32_t *d_bitsets, int64_t words_per_bitset,
                       const int32_t *d_src_off, const int32_t *d_src, int n_columns,
                       const int32_t *d_new_id, int64_t n, uint32_t *out, void *stream);
int device_sm_count(int device);

}  // namespace pm
