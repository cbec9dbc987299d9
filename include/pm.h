/*
 * pm.h — C ABI of the B300 pattern-morphing library (exact subgraph-pattern
 * counting and MNI support on a CSR data graph, with pattern morphing).
 *
 * Problem statement followed (Jamshidi & Vora, "Pattern Morphing for
 * Efficient Graph Mining", Section 2): a data graph G, a set of query
 * patterns (simple connected graphs, optionally vertex-labeled) each either
 * edge-induced (p^E: no anti-edges) or vertex-induced (p^V: an anti-edge on
 * every non-adjacent pair), and an operation: counting (Motif Counting, sum
 * aggregation) or minimum-node-image support (Frequent Subgraph Mining).
 * The library morphs the query set into an alternative pattern set
 * (Section 3), matches that set on the GPU, and transforms the aggregated
 * results back (Theorems 3.1 / 3.2, Corollary 3.1).
 *
 * Conventions for every entry point:
 *  - Status codes are returned; the library never aborts the process.
 *  - Fault injection on the host, for testing error paths: the environment
 *    variable PM_FAULT, read at each call, makes every device allocation
 *    fail ("alloc": PM_ENOMEM from the call that needed it), every
 *    pm_load_graph fail ("load": PM_EINVAL) or every pm_plan fail ("plan":
 *    PM_EUNSUPPORTED), each with a pm_last_error() text saying so.
 *  - The plan handle type is pm_query_plan (the C name pm_plan is the
 *    function that makes one).
 *  - Host input arrays are read during the call only and never retained;
 *    the caller keeps ownership.  Handles (pm_graph, pm_query_plan) are owned by
 *    the library and released with pm_free_graph / pm_free_plan.
 *  - A graph is read-only after loading; several plans (on several streams)
 *    may share it.  A plan is used by one stream at a time.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Vertex ids in inputs and outputs are the caller's; internally vertices
 *    are renumbered by (degree, caller id) ascending.
 *  - Counts are exact 128-bit unsigned integers stored as two uint64 words
 *    (low word first); the morph transform runs modulo 2^128, which is exact
 *    whenever every true result fits in 128 bits.
 */
#ifndef PM_H
#define PM_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_graph pm_graph;
typedef struct pm_query_plan pm_query_plan;   /* made by pm_plan() */

typedef enum {
    PM_OK = 0,
    PM_EINVAL = -1,        /* bad argument: null pointer, id out of range, pattern not connected, ... */
    PM_ENOMEM = -2,        /* host or device allocation failed */
    PM_ECUDA = -3,         /* a CUDA runtime call failed (pm_last_error() has the text) */
    PM_ETIMEOUT = -4,      /* the device deadline expired; partial results are not returned */
    PM_EOVERFLOW = -5,     /* a result does not fit the requested output width */
    PM_EUNSUPPORTED = -6,  /* valid request the library does not handle (e.g. MNI vertex-from-edge morph) */
    PM_ECANCELLED = -7     /* cancelled by the caller */
} pm_status;

/* Section 2: edge-induced patterns have no anti-edges; vertex-induced ones
 * have anti-edges on all non-adjacent pairs.  Cliques are both. */
typedef enum { PM_EDGE_INDUCED = 0, PM_VERTEX_INDUCED = 1 } pm_induced;

/* Section 2 applications: counting (Motif Counting) or MNI support (FSM). */
typedef enum { PM_OP_COUNT = 0, PM_OP_SUPPORT = 1 } pm_op;

/* Section 4.2 variants: no morphing (query patterns matched as given),
 * naive morphing (edge-induced queries -> vertex-induced superpatterns,
 * vertex-induced queries -> edge-induced superpatterns), and cost-based
 * selection among the alternative sets (Section 4.1): every count is
 * obtained the cheapest way — a vertex-induced count by matching it or as
 * its edge-induced count minus its superpatterns' vertex-induced counts
 * (Corollary 3.1, recursively), an edge-induced count by matching it or as
 * a sum over vertex-induced superpatterns (Theorem 3.1) — where the cost of
 * a pattern is the autotuner's sampled GPU time on the plan's graph (counting
 * kernels, also for MNI) and patterns already selected for other queries
 * cost nothing.  PM_MORPH_COST needs a graph in pm_plan.  Its sampling is
 * bounded (environment PM_COST_BUDGET_S, default 30 s per pm_plan): patterns
 * met after that get an estimate instead (decomposed patterns cheap, else
 * growing tenfold per vertex, and twentyfold for vertex-induced ones). */
typedef enum { PM_MORPH_NONE = 0, PM_MORPH_NAIVE = 1, PM_MORPH_COST = 2 } pm_morph_mode;

#define PM_MAX_K 8

/* A query pattern on vertices 0..k-1 (2 <= k <= PM_MAX_K, at most 6 for
 * PM_OP_SUPPORT).  edge_mask bit i is the i-th pair (a, b), a < b, in
 * lexicographic order (0,1), (0,2), ..., (0,k-1), (1,2), ...  label[u] is the
 * vertex label required at u, or -1 for any label.  The pattern must be
 * connected (Section 2), otherwise PM_EINVAL. */
typedef struct {
    int32_t k;
    uint32_t edge_mask;
    int8_t label[PM_MAX_K];
    int32_t induced;        /* pm_induced */
} pm_pattern;

typedef struct {
    int64_t n;               /* vertices */
    int64_t m;               /* undirected edges after cleaning */
    int64_t self_loops;      /* input edges dropped as self-loops */
    int64_t duplicates;      /* input edges dropped as duplicates (either direction) */
    int64_t max_degree;
    int64_t device_bytes;    /* device memory held by the graph */
    int32_t labeled;
    int32_t device;
} pm_graph_info;

typedef struct {
    int32_t n_queries;       /* requested patterns */
    int32_t n_matched;       /* distinct patterns the GPU matches (alternative set) */
    int32_t n_kernels_plans; /* matching plans (one per automorphism orbit of each matched pattern) */
    int32_t op;
} pm_plan_info;

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * callbacks must be set together; NULL restores cudaMalloc/cudaFree.  They
 * are called with the target device current and must return device memory
 * aligned to at least 256 bytes, or NULL on failure. */
typedef void *(*pm_alloc_fn)(size_t bytes, int device, void *ctx);
typedef void (*pm_free_fn)(void *ptr, size_t bytes, int device, void *ctx);
pm_status pm_set_allocator(pm_alloc_fn alloc, pm_free_fn release, void *ctx);

/* Load an undirected data graph (Section 2: G with vertices V, edges E and
 * optional labels L).  n vertices with ids 0..n-1; m_raw edges (src[i], dst[i])
 * in either direction; self-loops and duplicates are dropped and reported.
 * labels: n bytes or NULL (unlabeled).  The graph is renumbered by
 * (degree, id) ascending, stored as CSR with sorted rows (int64 row offsets,
 * int32 column ids, uint8 labels) on `device`, uploaded on `stream`, and the
 * call returns after the upload completes.  Vertices of degree >= the
 * environment variable PM_HUB_MIN_DEGREE (default 1024) also get an n-bit
 * adjacency bitmap (highest degrees first, at most 256 MiB in total) that
 * turns membership tests in their lists into single bit reads.
 * Errors: PM_EINVAL (null pointer,
 * n < 1 or n > 2^31-1, an id outside [0, n)), PM_ENOMEM, PM_ECUDA,
 * PM_EUNSUPPORTED (2^32 or more adjacency entries). */
pm_status pm_load_graph(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                        const uint8_t *labels, int device, void *stream, pm_graph **out);
pm_status pm_graph_get_info(const pm_graph *g, pm_graph_info *out);
/* new_id[v] = internal (degree-ordered) id of caller vertex v; n entries. */
pm_status pm_graph_vertex_order(const pm_graph *g, int32_t *new_id);
/* The host half of pm_load_graph alone (Section 2's data graph as the
 * matching kernels read it), touching no device: self-loops and duplicate
 * edges dropped, both directions stored, vertices renumbered by (degree,
 * caller id) ascending, rows in internal ids sorted ascending.  All buffers
 * are host memory owned by the caller.  rowptr: n + 1 int64 row offsets;
 * col: room for 2 * m_raw int32 entries (an upper bound), of which rowptr[n]
 * (twice the simple edge count) are written; new_id (NULL to skip): n int32,
 * the internal id of each caller vertex; lowdeg (NULL to skip): n int64, per
 * internal id the neighbours with smaller internal ids (where its row
 * crosses its own id).  Labels are not taken: a caller permutes its own
 * with new_id.
 * Errors: PM_EINVAL (null rowptr or col, n < 1 or n > 2^31-1, null edge
 * arrays with m_raw > 0, an id outside [0, n)), PM_ENOMEM, PM_EUNSUPPORTED
 * (2^32 or more adjacency entries). */
pm_status pm_prepare_csr(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                         int64_t *rowptr, int32_t *col, int32_t *new_id, int64_t *lowdeg);
void pm_free_graph(pm_graph *g);

/* Plan a query set (Section 4.1 "external module", step a): canonicalise and
 * deduplicate the nq query patterns, choose each one's alternative pattern
 * set by `mode` (Theorem 3.1 for edge-induced queries, Corollary 3.1 applied
 * recursively for vertex-induced ones; MNI support morphs only edge-induced
 * queries, Section 3.2.3), deduplicate the matched patterns across queries,
 * and compile one matching plan per automorphism orbit of each matched
 * pattern.  Host-only (device tables are made on the first pm_count or
 * pm_support); the plan keeps a reference to g (free plans first).  g may
 * be NULL: the plan then serves pm_morph, pm_plan_matched and
 * pm_plan_export only, and running it returns PM_EINVAL.
 * Errors: PM_EINVAL (bad pattern, labels on an unlabeled graph),
 * PM_EUNSUPPORTED, PM_ENOMEM. */
pm_status pm_plan(const pm_graph *g, const pm_pattern *queries, int32_t nq, pm_op op,
                  pm_morph_mode mode, pm_query_plan **out);
pm_status pm_plan_get_info(const pm_query_plan *p, pm_plan_info *out);
/* The matched (alternative) patterns, n_matched entries. */
pm_status pm_plan_matched(const pm_query_plan *p, pm_pattern *out);
void pm_free_plan(pm_query_plan *p);
/* Plan families.  Rooted plans (one per automorphism orbit of a matched
 * pattern) pin the orbit to each occurrence's highest-ranked vertex, which
 * makes per-root counts exact (pm_count_roots always uses them).  The free
 * plan of a pattern counts every occurrence once from its cheapest vertex,
 * breaking the whole automorphism group.  pm_count and pm_support use, per
 * matched pattern, the family the autotuner found faster on the plan's graph
 * (PM_PLANS_AUTO), unless pm_plan_select forces one.  The rooted plan of an
 * unlabeled 4- or 5-clique runs in the clique kernel, which the autotuner
 * does not yet choose (its hub-to-hub tasks are not load-balanced); it runs
 * when the rooted family is selected and in pm_count_roots (environment
 * variable PM_CLIQUE_BALANCED=1, read at each launch, spreads a root's
 * tasks over chunks and weighs intersection sides by search depth; exact
 * either way).  The rooted plan
 * of the edge-induced 4-cycle runs in the wedge kernels: roots among the
 * H highest-ranked vertices (environment variable PM_WEDGE_HEAVY, read when
 * a plan first runs the 4-cycle; default 16384) keep their pair counters in
 * shared memory, the others in per-block global counters. */
#define PM_PLANS_AUTO (-1)
#define PM_PLANS_ROOTED 0
#define PM_PLANS_FREE 1
/* No timing: free plans, except the rooted 4-cycle plan that runs the
 * wedge kernel (for latency-bound callers such as the serving loop), and the
 * decomposition kernels where they apply. */
#define PM_PLANS_QUICK 2
/* Decomposition kernels for the unlabeled edge-induced patterns they cover
 * (4 vertices: star K1,3, path P4, tailed triangle, diamond; 5 vertices:
 * star, fork, path, cricket, bull, lollipop, banner, 5-cycle, kite, dart,
 * bowtie, house, book K1,1,3, gem, 4-clique with a pendant), autotuned
 * families for the other patterns.  Their counts come from exact identities
 * over per-vertex and per-edge quantities (degrees, triangles per edge,
 * 2-paths from each vertex to the vertices below it, 4-cliques with their
 * degree sums) instead of enumerating occurrences.  Counting plans use them
 * by default (PM_PLANS_AUTO and PM_PLANS_QUICK); PM_PLANS_ROOTED or
 * PM_PLANS_FREE forces set-operation plans for every pattern.  Scratch:
 * 4 bytes per CSR entry, and for the 4-cycle based patterns (path P5,
 * banner, house, 5-cycle) 8 bytes per vertex per resident block of the
 * 2-path kernel (at most 2 per SM). */
#define PM_PLANS_DECOMP 3
pm_status pm_plan_select(pm_query_plan *p, int32_t family);
/* How a plan's set-operation plans are launched.  PM_LAUNCH_PER_PATTERN
 * (default): one launch sequence (both matching passes and the piece scan)
 * per matched pattern, one after another on the stream.  PM_LAUNCH_SINGLE:
 * all plans in one persistent launch over one shared queue of (plan, edge
 * chunk) tasks.  On R-MAT scale 20 the 4-motif set ran in 0.96 s per
 * pattern against 1.67 s in a single launch (the plans contend for L2), so
 * the single launch suits batches of many small patterns.  Must be set
 * before pm_plan_capture. */
#define PM_LAUNCH_PER_PATTERN 0
#define PM_LAUNCH_SINGLE 1
pm_status pm_plan_set_launch(pm_query_plan *p, int32_t mode);
/* Run the autotuner now (it otherwise runs inside the first pm_count or
 * pm_support): for each matched pattern not yet decided on this graph, time
 * its rooted and free plans on the same sample of about 4096 task chunks
 * (0.5 s deadline; an 8x, then 64x sparser sample when both run past it) and
 * keep the faster, then time that family's task granularity -- the
 * second-level candidates a task chunk keeps before the rest is deferred to
 * other warps, which sets how many warps share a hub root -- at a quarter
 * and at four times the compiled value, keeping one only if it is more than
 * 10% faster; decisions are cached on the graph.  Patterns are timed
 * smallest first, at most 30 s of sampling per call (environment
 * PM_AUTOTUNE_BUDGET_S); the rest take the quick rule (decomposition where
 * it applies, the rooted family for the wedge kernels, else free) without
 * being cached.  families (nullable): n_matched entries receiving
 * PM_PLANS_ROOTED, PM_PLANS_FREE or (counting plans, unless a set-operation
 * family is forced) PM_PLANS_DECOMP. */
pm_status pm_plan_autotune(pm_query_plan *p, void *stream, int32_t *families);
/* Copy the compiled plans of one family (PM_PLANS_ROOTED: n_kernels_plans
 * records; PM_PLANS_FREE: n_matched records) into out (cap bytes).  A record
 * is 112 bytes: int32 k, n_enum, tail, closed, counter, dom_base, n_columns,
 * split, task_space, kind (0 set operations, 1 wedge pairs, 2 clique), pair (1: the
 * last two levels are an independent pair counted as |A||B| - |A n B|, with
 * the merged constraints of A n B in level k), int32 pad;
 * then 8 levels of uint8 isect, diff, lt,
 * gt, neq, int8 label, uint8 column, vertex (the pattern vertex the level
 * binds).  For inspection and tests;
 * PM_EINVAL if cap is too small. */
pm_status pm_plan_export(const pm_query_plan *p, int32_t family, void *out, int64_t cap);

/* Section 4.1 step b for counting: requested[2*i..] = sum_j T[i][j] *
 * matched[2*j..] modulo 2^128, where T holds the morph coefficients
 * (c(p, q) = number of distinct copies of p spanning q, signed for
 * vertex-from-edge).  matched: 2*n_matched words, requested: 2*n_queries.
 * Pure host arithmetic, usable on its own. */
pm_status pm_morph(const pm_query_plan *p, const uint64_t *matched, uint64_t *requested);

/* Count every query pattern (Section 2, Motif Counting: sum aggregation of
 * distinct occurrences = matches / |Aut(p)|; morphed plans combine the
 * matched patterns' counts by Theorem 3.1 / Corollary 3.1).
 * Runs the matching kernels on `stream`, waits for them, applies pm_morph.
 * counts: 2*n_queries words (128-bit, low word first).  matched (nullable):
 * 2*n_matched words receiving the alternative set's raw counts.
 * timeout_s <= 0 means no deadline; otherwise the kernels stop at the
 * deadline and the call returns PM_ETIMEOUT. */
pm_status pm_count(pm_query_plan *p, void *stream, double timeout_s, uint64_t *counts,
                   uint64_t *matched);

/* pm_count with a deadline per matched pattern: with per-pattern launches
 * the matched patterns run one after another, each with
 * timeout_per_pattern_s; in PM_LAUNCH_SINGLE mode they share one launch and
 * each has timeout_per_pattern_s from its start; either way capped by
 * timeout_total_s from the start of the call (<= 0: no limit);
 * a query whose alternative set uses a pattern whose deadline expired gets
 * status PM_ETIMEOUT and count 0, the others PM_OK and their exact counts.
 * status: n_queries entries.  Returns PM_OK unless the call itself fails. */
pm_status pm_count_each(pm_query_plan *p, void *stream, double timeout_per_pattern_s,
                        double timeout_total_s, uint64_t *counts, int32_t *status);

/* As pm_count, restricted to occurrences whose highest-ranked vertex —
 * rank ordering vertices by (degree, caller id) — is one of the nroots
 * caller vertex ids in roots[].  Summing over a partition of V gives
 * pm_count's result, so sampled roots give exactly checkable partial counts. */
pm_status pm_count_roots(pm_query_plan *p, void *stream, double timeout_s, const int32_t *roots,
                         int64_t nroots, uint64_t *counts, uint64_t *matched);

/* Record the whole of pm_count for this plan (counter reset, arming, both
 * matching passes and the piece scan, the wedge or clique kernels, the copy of the raw
 * counts into pinned host memory) as one CUDA graph; later pm_count calls on
 * the plan replay it with one cudaGraphLaunch on their stream.  Autotuning
 * and all buffer set-up happen here, before capture.  timeout_s (<= 0: none)
 * is fixed into the graph; pm_count's own timeout_s is then ignored. */
pm_status pm_plan_capture(pm_query_plan *p, void *stream, double timeout_s);

/* pm_count_each recorded as one CUDA graph (the per-pattern and total
 * deadlines are fixed into it); later pm_count_each calls on the plan replay
 * it and ignore their own deadlines.  In PM_LAUNCH_SINGLE mode the plans
 * of each pattern size share one persistent launch (sizes in increasing
 * order) and every pattern's deadline runs from its launch's start: the
 * patterns whose work the deadline cuts (counted from per-plan progress
 * counters) report PM_ETIMEOUT, the others their exact counts. */
pm_status pm_plan_capture_each(pm_query_plan *p, void *stream, double timeout_per_pattern_s,
                               double timeout_total_s);

/* pm_count with an instrumented kernel that also returns the algorithmic
 * bytes of the matching: 4 B per element of every set-operation operand,
 * each operand cut to the plan's (lower, upper) id window (merge accounting
 * |A'| + |B'| per intersection or difference), 16 B per row-offset pair,
 * 28 B per task and 24 B plus 8 B per excluded vertex for each closed-form
 * count, plus the bytes of the clique and decomposition kernels (below).
 * Slower than pm_count; meant for roofline measurement. */
pm_status pm_count_instrumented(pm_query_plan *p, void *stream, uint64_t *counts,
                                uint64_t *alg_bytes);
/* Algorithmic bytes of each matched pattern in the plan's last
 * pm_count_instrumented (n_matched entries): its own launches in per-pattern
 * mode, all set-operation plans on the first one in PM_LAUNCH_SINGLE mode,
 * the decomposition passes (4 B per list element read, 16 B per row-offset
 * pair, 4 B per counter read or written, 8 B per atomic update) on the first
 * decomposed pattern, nothing for the wedge kernels. */
pm_status pm_plan_pattern_bytes(const pm_query_plan *p, uint64_t *bytes);

/* Device time (CUDA events on the launch stream) of the matching kernel of
 * the plan's last completed pm_count / pm_count_roots / pm_support call;
 * 0 if that call launched none. */
pm_status pm_plan_last_kernel_ms(const pm_query_plan *p, float *ms);

/* Device time (CUDA events on the launch stream) of each matched pattern's
 * launch sequence in the plan's last completed pm_count (or its captured
 * replay), in per-pattern launch mode: ms[j] for matched pattern j
 * (n_matched entries), 0 for patterns that did not run on their own
 * (single-launch mode, pm_count_roots, pm_count_instrumented).  Also
 * filled by pm_count_each. */
pm_status pm_plan_pattern_ms(const pm_query_plan *p, float *ms);
/* Number of the library's kernels launched by the plan's last pm_count
 * (or pm_count_each, or captured into its CUDA graph), counting the arming
 * and gate kernels. */
pm_status pm_plan_last_launches(const pm_query_plan *p, int64_t *launches);

/* MNI support (Section 2, FSM; Theorem 3.2 with MNI tables for morphed
 * plans) of every query of a PM_OP_SUPPORT plan: one column per orbit of the
 * query's label-preserving automorphism group, holding the images of the
 * orbit's vertices over all matches; support = the smallest column.
 * support: n_queries words; frequent (nullable): n_queries bytes, 1 when
 * support >= threshold.  domains_dev (nullable, device memory on the
 * graph's device, caller-owned): the columns themselves, one bitset of
 * ceil(n / 32) uint32 words per column, queries in order and each query's
 * columns in column order (pm_plan_query_columns); bit v % 32 of word v / 32
 * is set when caller vertex v is in the column.  Written asynchronously on
 * `stream` and complete when the call returns.  The first call with
 * domains_dev on a graph uploads the caller-to-internal vertex map (4n bytes,
 * kept with the graph).  Errors: PM_EINVAL, PM_ENOMEM, PM_ECUDA,
 * PM_ETIMEOUT (nothing returned). */
pm_status pm_support(pm_query_plan *p, void *stream, double timeout_s, uint64_t threshold,
                     uint64_t *support, uint8_t *frequent, uint32_t *domains_dev);
/* Column of every vertex of every query of a PM_OP_SUPPORT plan:
 * columns[i * PM_MAX_K + u] for vertex u of query i (-1 for u >= k).
 * Columns are the automorphism orbits numbered by their smallest vertex;
 * query i has 1 + max_u columns[i * PM_MAX_K + u] of them. */
pm_status pm_plan_query_columns(const pm_query_plan *p, int32_t *columns);

/* List every occurrence of every query of a counting plan (Section 3.2.1:
 * materialising M(q^V) o phi(p^E, q^E), Theorem 3.1).  An edge-induced query
 * planned with morphing is listed from the matches of its vertex-induced
 * superpatterns, each composed with one map per distinct copy of the query
 * it contains, so every distinct occurrence (edge subgraph) appears exactly
 * once; queries matched as given (PM_MORPH_NONE, cliques) are listed
 * directly.  A vertex-induced query morphed to edge-induced patterns cannot
 * be listed (Corollary 3.1 subtracts): PM_EUNSUPPORTED.
 * tuples: cap x PM_MAX_K int32 (host), occurrence r is tuples[r * PM_MAX_K
 * + u] = the caller vertex that query vertex u maps to (-1 for u >= k);
 * query_of (nullable): cap int32, the query of each occurrence.  Order is
 * unspecified.  *n_out = number of occurrences; PM_EOVERFLOW (nothing
 * written) when it exceeds cap.  Runs a count first to size the output;
 * device memory of (PM_MAX_K + 1) x 4 bytes per listed match is taken
 * through the allocator for the call.  Errors: PM_EINVAL, PM_EUNSUPPORTED,
 * PM_EOVERFLOW, PM_ENOMEM, PM_ECUDA, PM_ETIMEOUT. */
pm_status pm_enumerate(pm_query_plan *p, void *stream, double timeout_s, int32_t *tuples,
                       int32_t *query_of, int64_t cap, int64_t *n_out);

/* Sharded MNI support.  Every match has one highest-ranked vertex (rank =
 * (degree, caller id)), so the MNI columns of a query over all matches are
 * the union (OR) of its columns over the matches whose highest-ranked vertex
 * lies in each part of a partition of the vertices; a process per part fills
 * its columns with pm_support_roots, the columns are gathered, ORed with
 * pm_domains_or, and pm_support_from_domains takes each query's smallest
 * column.
 * pm_support_roots: the query columns (layout of pm_support's domains_dev,
 * device memory on the graph's device) over the matches whose highest-ranked
 * vertex is one of the nroots caller ids in roots (rooted plans).
 * pm_domains_or: out[w] = OR over p < n_parts of parts[p * words + w]
 * (device memory, asynchronous on stream).
 * pm_support_from_domains: support (n_queries words) and frequent (nullable)
 * from a complete set of query columns.  Errors: PM_EINVAL, PM_ENOMEM,
 * PM_ECUDA, PM_ETIMEOUT. */
pm_status pm_support_roots(pm_query_plan *p, void *stream, double timeout_s, const int32_t *roots,
                           int64_t nroots, uint32_t *domains_dev);
pm_status pm_domains_or(const uint32_t *parts_dev, int32_t n_parts, int64_t words, uint32_t *out_dev,
                        void *stream);
pm_status pm_support_from_domains(pm_query_plan *p, const uint32_t *domains_dev, void *stream,
                                  uint64_t threshold, uint64_t *support, uint8_t *frequent);

/* Frequent subgraph mining with MNI support (Section 2, FSM), level-wise
 * up to max_edges (1..5) edges on a labeled graph.  Level 1: every labeled
 * edge whose two labels occur in the graph.  Level j+1: connected labeled
 * patterns made by adding one edge (between existing vertices, or to a new
 * vertex with a label that occurs) to a frequent level-j pattern, kept only
 * if every connected one-edge-smaller subpattern is frequent; MNI support is
 * anti-monotone, so no frequent pattern is lost.  Each level runs pm_plan
 * (PM_OP_SUPPORT, mode) + pm_support(threshold); frequent means support >=
 * threshold.  Outputs every candidate of every level, in level order:
 * out[i] (edge-induced labeled pattern), support[i], frequent[i] (nullable).
 * cap: entries the caller provides; *n_out: entries produced (PM_EOVERFLOW
 * with *n_out = the size needed when cap is too small). */
pm_status pm_fsm(const pm_graph *g, int32_t max_edges, uint64_t threshold, pm_morph_mode mode,
                 void *stream, double timeout_s, pm_pattern *out, uint64_t *support,
                 uint8_t *frequent, int32_t cap, int32_t *n_out);

/* Edge-induced 4-cycle count of a graph given as a device CSR, for callers
 * that cannot allocate device memory during the call (a fully reserved
 * memory pool, a real-time loop that must not enter an allocator, an
 * embedder that owns every device byte).  The paper has no counterpart: this
 * is a library convenience.  rowptr: n+1 int64 row offsets, col: int32
 * neighbour ids, both device memory owned by the caller, describing an
 * undirected simple graph (each edge in both rows, no self-loops) with
 * every row sorted ascending; count: 2 device uint64 words (low, high)
 * receiving the exact 128-bit count.  Asynchronous on `stream`.  The call
 * allocates nothing: its scratch is a 16 MiB array built into the library
 * (held on every GPU that loads it until exit), so n may be at most
 * 4194304 (PM_EINVAL beyond).  Each block keeps n counters in that array,
 * so the call runs min(SMs, 4194304 / n) blocks: all SMs up to about 28K
 * vertices, 64 blocks at 65536, 4 blocks at 2^20 and one above 2^21, so
 * large graphs count much more slowly here than with pm_count.  The first call on a device looks up that
 * array's device address, so make it before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. */
pm_status pm_count_c4_noalloc(const int64_t *rowptr, const int32_t *col, int64_t n,
                              uint64_t *count, void *stream);

/* Serving (continuous batching of count requests against device-resident
 * graphs).  Each graph gets workers_per_graph worker threads with their own
 * CUDA streams.  A free worker takes the requests queued for its graph (up
 * to max_batch_patterns patterns) as one batch: one pm_plan over all their
 * queries (morph selection with `mode` deduplicates the matched patterns the
 * requests share) and one pm_count_each with batch_timeout_s as the deadline
 * of each matched pattern and batch_total_s for the batch; each request then
 * receives its own slice of the
 * counts, and fails with PM_ETIMEOUT only if one of its queries needed a
 * pattern whose deadline expired.  Requests arriving while batches run
 * join the next batch as soon as a worker is free and the batch's device
 * memory estimate fits hbm_budget_bytes beside the batches in flight;
 * batches on different workers overlap on the device.  Latency is measured
 * from pm_server_submit to the end of the request's batch.  With
 * request_timeout_s > 0 a request still queued that long after submission
 * completes with PM_ETIMEOUT without device work (load shedding: the queue
 * cannot grow without bound when requests arrive faster than batches
 * finish), and a batch's total deadline is cut to the time left to its
 * oldest request. */
typedef struct pm_server pm_server;
typedef struct {
    int32_t workers_per_graph;
    int32_t max_batch_patterns;
    int64_t hbm_budget_bytes;
    double batch_timeout_s;     /* deadline of each matched pattern of a batch (<= 0: none) */
    double batch_total_s;       /* deadline of the whole batch (<= 0: none) */
    int32_t mode;               /* pm_morph_mode */
    int32_t family;             /* plan family for every batch (pm_plan_select) */
    double request_timeout_s;   /* deadline of a request from its submission (<= 0: none) */
} pm_server_config;
typedef struct {
    int64_t requests_submitted, requests_done, batches, patterns_done;
    int64_t matched_alone;      /* sum over requests of matched patterns if planned alone */
    int64_t matched_batched;    /* sum over batches of matched patterns (after deduplication) */
    int64_t timeouts, failures; /* requests whose batch hit the deadline / failed otherwise */
    int64_t shed;               /* of the timeouts: dropped unrun after request_timeout_s */
} pm_server_stats;
/* graphs stay owned by the caller and must outlive the server. */
pm_status pm_server_create(const pm_graph *const *graphs, int32_t n_graphs,
                           const pm_server_config *cfg, pm_server **out);
/* Queue a request of nq patterns (copied) for graphs[graph]; malformed
 * patterns are rejected here.  *id identifies it for pm_server_wait. */
pm_status pm_server_submit(pm_server *s, int32_t graph, const pm_pattern *queries, int32_t nq,
                           uint64_t *id);
/* Wait up to timeout_s (< 0: forever, 0: poll) for request id.  *done = 1
 * when it finished: counts (2*nq words, nullable), *latency_s,
 * *request_status (PM_OK only if every query of the request succeeded) and
 * query_status (nq entries, nullable: each query's own status; a query
 * whose patterns all finished has PM_OK and its count even when another
 * query of the request timed out) are then filled and the request is
 * forgotten. */
pm_status pm_server_wait(pm_server *s, uint64_t id, double timeout_s, int32_t *done,
                         uint64_t *counts, double *latency_s, pm_status *request_status,
                         int32_t *query_status);
pm_status pm_server_get_stats(pm_server *s, pm_server_stats *out);
/* Stops the workers after their current batches; queued requests are dropped. */
void pm_server_destroy(pm_server *s);

const char *pm_strerror(pm_status s);
/* Text of the last error raised on the calling thread ("" if none). */
const char *pm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */
