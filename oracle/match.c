/*
 * Oracle matcher: plain backtracking over injective maps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product never does.
 *
 * A match of a pattern p in a data graph G (Section 2, "Pattern Semantics")
 * is an injective map m: V(p) -> V(G) with (m(u), m(v)) an edge of G for
 * every edge (u, v) of p and a non-edge for every anti-edge, and (when p
 * carries labels) label(m(u)) equal to label(u).  This file enumerates those
 * maps with no symmetry breaking at all: every automorphic copy is visited,
 * and the caller divides by |Aut(p)|.
 *
 * The maps are partitioned by the data vertex of highest rank in their image
 * (rank = the caller's total order on V(G)): a root r and a pattern vertex j
 * with m(j) = r, every other image ranked below r.  Summing over all roots
 * and all j visits every map exactly once; summing over a subset of roots
 * counts exactly the maps whose highest-ranked vertex lies in that subset.
 *
 * Edge and anti-edge tests are binary searches in the sorted adjacency list.
 * At the last pattern vertex the valid candidates are counted (or, for MNI
 * domains, each one is recorded) instead of recursing further.
 */
#include <stdint.h>
#include <string.h>
#include <omp.h>

typedef unsigned __int128 u128;

#define KMAX 8

typedef struct {
    const int64_t *rowptr;
    const int32_t *col;
    const int32_t *labels;   /* may be NULL */
    const int64_t *rank;
    int k;
    int order[KMAX];         /* pattern vertices in visiting order */
    int parent[KMAX];        /* an earlier pattern neighbour of order[i] */
    int8_t rel[KMAX][KMAX];  /* +1 edge, -1 anti-edge, 0 free */
    int32_t plab[KMAX];      /* -1 = any label */
    int64_t root_rank;
    int32_t map[KMAX];       /* map[u] = image of pattern vertex u */
    uint8_t *dom;            /* k * n flags, or NULL when counting */
    int64_t n;
} ctx_t;

static int has_edge(const ctx_t *c, int32_t a, int32_t b)
{
    int64_t lo = c->rowptr[a], hi = c->rowptr[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t x = c->col[mid];
        if (x == b) return 1;
        if (x < b) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/* Can pattern vertex order[level] map to data vertex x, given order[0..level-1]? */
static int admissible(const ctx_t *c, int level, int32_t x)
{
    int u = c->order[level];
    if (c->plab[u] >= 0 && (c->labels == NULL || c->labels[x] != c->plab[u])) return 0;
    if (c->rank[x] >= c->root_rank) return 0;
    for (int i = 0; i < level; i++) {
        int w = c->order[i];
        int32_t y = c->map[w];
        if (y == x) return 0;
        if (c->rel[u][w] == 1 && !has_edge(c, x, y)) return 0;
        if (c->rel[u][w] == -1 && has_edge(c, x, y)) return 0;
    }
    return 1;
}

/* Optional wall-clock budget (orc_set_budget): once it has passed, every
 * walk returns at once and orc_count reports -2.  Checked every 4096 calls
 * per thread; it changes no count that completes within the budget. */
static double g_deadline = 0.0;
static volatile int g_expired = 0;

static int expired(void)
{
    static __thread unsigned tick = 0;
    if (g_deadline <= 0.0) return 0;
    if (g_expired) return 1;
    if ((++tick & 4095u) == 0 && omp_get_wtime() > g_deadline) g_expired = 1;
    return g_expired;
}

static u128 extend(ctx_t *c, int level)
{
    if (expired()) return 0;
    int u = c->order[level];
    int32_t pv = c->map[c->parent[level]];
    u128 total = 0;
    for (int64_t e = c->rowptr[pv]; e < c->rowptr[pv + 1]; e++) {
        int32_t x = c->col[e];
        if (!admissible(c, level, x)) continue;
        c->map[u] = x;
        if (level == c->k - 1) {
            total += 1;
            if (c->dom) {
                for (int w = 0; w < c->k; w++)
                    __atomic_store_n(&c->dom[(int64_t)w * c->n + c->map[w]], 1, __ATOMIC_RELAXED);
            }
        } else {
            total += extend(c, level + 1);
        }
    }
    return total;
}

/* Visiting order: breadth-first from pattern vertex j (p is connected). */
static int bfs_order(ctx_t *c, int j)
{
    int seen[KMAX] = {0};
    int head = 0, tail = 0;
    c->order[tail] = j; c->parent[tail] = -1; tail++; seen[j] = 1;
    while (head < tail) {
        int v = c->order[head++];
        for (int w = 0; w < c->k; w++) {
            if (!seen[w] && c->rel[v][w] == 1) {
                seen[w] = 1;
                c->order[tail] = w; c->parent[tail] = v; tail++;
            }
        }
    }
    return tail == c->k;
}

/*
 * Number of matches of the pattern (k vertices, relation matrix rel[k*k],
 * labels plab[k]) whose highest-ranked image vertex is one of roots[0..nroots)
 * (roots == NULL: every vertex).  Result as 128 bits in out[0] (low), out[1].
 * If dom != NULL, also sets dom[u*n + x] = 1 for every match m with m(u) = x.
 * Returns 0, -1 on bad arguments (k out of range, pattern disconnected), or
 * -2 when the budget set by orc_set_budget ran out (the result is then
 * incomplete).
 */
int orc_count(int64_t n, const int64_t *rowptr, const int32_t *col,
              const int32_t *labels, const int64_t *rank,
              int k, const int8_t *rel, const int32_t *plab,
              int64_t nroots, const int32_t *roots, int nthreads,
              uint64_t *out, uint8_t *dom)
{
    if (k < 1 || k > KMAX) return -1;
    ctx_t proto;
    memset(&proto, 0, sizeof proto);
    proto.rowptr = rowptr; proto.col = col; proto.labels = labels; proto.rank = rank;
    proto.k = k; proto.dom = dom; proto.n = n;
    for (int a = 0; a < k; a++) {
        proto.plab[a] = plab[a];
        for (int b = 0; b < k; b++) proto.rel[a][b] = rel[a * k + b];
    }
    if (!bfs_order(&proto, 0)) return -1;
    int64_t count = roots ? nroots : n;
    u128 total = 0;
    if (nthreads > 0) omp_set_num_threads(nthreads);
    #pragma omp parallel
    {
        u128 local = 0;
        ctx_t c = proto;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < count; i++) {
            int32_t r = roots ? roots[i] : (int32_t)i;
            for (int j = 0; j < k; j++) {
                if (c.plab[j] >= 0 && (labels == NULL || labels[r] != c.plab[j])) continue;
                bfs_order(&c, j);
                c.root_rank = rank[r];
                c.map[j] = r;
                if (k == 1) {
                    local += 1;
                    if (dom) __atomic_store_n(&dom[r], 1, __ATOMIC_RELAXED);
                } else {
                    local += extend(&c, 1);
                }
            }
        }
        #pragma omp critical
        total += local;
    }
    out[0] = (uint64_t)total;
    out[1] = (uint64_t)(total >> 64);
    return g_expired ? -2 : 0;
}

/* Wall-clock budget for the following orc_count calls, from now; 0 = none. */
void orc_set_budget(double seconds)
{
    g_expired = 0;
    g_deadline = seconds > 0.0 ? omp_get_wtime() + seconds : 0.0;
}

int orc_max_threads(void) { return omp_get_max_threads(); }
