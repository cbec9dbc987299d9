// Matching plans and device-side data layouts shared by host and kernels.
//
// A rooted plan matches one pattern p with one automorphism orbit O of p
// pinned to the task's root: the root is the highest-ranked (largest internal id)
// vertex of the occurrence and is the image of O's representative.  Every
// occurrence of p has exactly one highest-ranked vertex, whose preimage lies
// in exactly one orbit, so the plans of p partition p's occurrences; within a
// plan the remaining symmetry (the stabiliser of the representative) is
// broken by ordering constraints chosen as in Grochow & Kellis (RECOMB 2007):
// at each vertex v, in matching order, v's image is the smallest over v's
// orbit under the current stabiliser, which then shrinks to fix v.  Rooted
// plans make per-root counts exact (pm_count_roots).  A free plan counts all
// of p's occurrences with a single plan: it breaks the whole automorphism
// group the same way and bounds nothing by the root, so it can start at the
// cheapest vertex (e.g. a diamond's chord, whose two other vertices then form
// one binomial tail per chord edge).
//
// Level i of a plan binds pattern vertex order[i].  Its candidates are the
// data vertices x with
//   x in N(m_j)      for every j in isect  (edges of p: set intersection)
//   x not in N(m_j)  for every j in diff   (anti-edges of p^V: set difference)
//   x < m_j (j in lt), x > m_j (j in gt)   (root bound, symmetry breaking)
//   x != m_j (j in neq)                    (injectivity not implied above)
//   label(x) == label                      (labeled patterns)
// Pair finals: when the last two vertices u, v are independent leaves (each
// a single closed adjacency range, no edge, anti-edge or ordering between
// them, v only required to differ from u), the prefix contributes
// |A| * |B| - |A n B| (choices of u and v minus collisions u = v), where
// lv[n_enum] and lv[n_enum + 1] give A and B and lv[k] holds the merged
// constraints of A n B (counted by a scan); n_enum = k - 2, tail = 2.
// Levels 0 (root) and 1 (a lower-ranked neighbour of the root) come from the
// task, an oriented edge.  Levels 2..n_enum-1 are enumerated.  The last `tail`
// levels share one candidate set C and are totally ordered among themselves,
// so they contribute C(|C|, tail) without enumeration; when that set is a
// single adjacency range minus a few known vertices (`closed`), |C| comes
// from binary searches alone.
#pragma once

#include <cstdint>

namespace pm {

constexpr int PLAN_KMAX = 8;

struct DevLevel {
    uint8_t isect;
    uint8_t diff;
    uint8_t lt;
    uint8_t gt;
    uint8_t neq;
    int8_t label;
    uint8_t column;   // MNI column (orbit index) of the pattern vertex bound here
    uint8_t vertex;   // the pattern vertex bound here (listing output)
};

// Which oriented edges (root, v) a plan's tasks range over.
enum TaskSpace : int32_t {
    TASKS_LOWER = 0,   // v < root: rooted plans (root = highest-ranked vertex)
    TASKS_UPPER = 1,   // v > root: free plans whose symmetry orders root and v
    TASKS_BOTH = 2     // every directed edge: free plans without that order
};

// How a plan is executed.  Set-operation plans run in the matching kernel.
// The rooted plan of the edge-induced 4-cycle runs in a wedge kernel: for the
// root a and each opposite vertex c < a, the occurrences with a as highest-
// ranked vertex are C(w, 2) with w = |N(a) n N(c) n [0, a)|; counting the
// 2-paths a-b-c into per-c counters and adding each counter's old value
// gives that sum, since C(w, 2) = 0 + 1 + ... + (w - 1).  The rooted plan of
// the unlabeled 4- or 5-clique runs in a clique kernel: for the root a and
// each lower neighbour b, the occurrences with a highest-ranked and b second
// are the (k-2)-cliques inside S = N(a) n N(b) n [0, b), counted on S once
// it is materialised.  In both cases the plan's levels still describe the
// same occurrences.
enum PlanKind : int32_t { PLAN_SETOPS = 0, PLAN_WEDGE_PAIRS = 1, PLAN_CLIQUE = 2 };

struct DevPlan {
    int32_t k;
    int32_t n_enum;
    int32_t tail;
    int32_t closed;
    int32_t counter;      // output slot: index of the matched pattern
    int32_t dom_base;     // first MNI bitset of the matched pattern (support plans)
    int32_t n_columns;    // MNI columns of the matched pattern
    int32_t split;        // second-level candidates a task chunk keeps before deferring the rest
    int32_t task_space;   // TaskSpace
    int32_t kind;         // PlanKind
    int32_t pair;         // 1: the last two levels are an independent pair (see below)
    int32_t pad;
    DevLevel lv[PLAN_KMAX];
};

// Device view of a loaded graph: CSR over internal ids 0..n-1 (ascending
// (degree, caller id)), rows sorted ascending.
struct DevGraph {
    int64_t n;
    int64_t nnz;               // 2 * undirected edges
    const int64_t *rowptr;     // n + 1
    const int32_t *col;        // nnz
    const uint8_t *labels;     // n, or nullptr
    // Adjacency bitmaps of the highest-degree vertices: hub[v] >= 0 is the
    // index of v's bitmap (n bits, `words` 32-bit words each) in `bits`, so a
    // membership test in N(v) is one bit read instead of a binary search.
    const int32_t *hub;        // n, or nullptr (no bitmaps)
    const uint32_t *bits;
    int64_t words;
};

// Task spaces: oriented edges (root, v) grouped by root, for each TaskSpace.
// roots == nullptr means the implicit root list n-1, n-2, ..., 0 (highest
// ranked first); an explicit list serves TASKS_LOWER only.  off[s][i] =
// number of tasks of roots 0..i-1 of the list in space s (nroots + 1
// entries); ntasks[s] = off[s][nroots].
struct DevTasks {
    const int32_t *roots;
    const int64_t *off[3];
    int64_t nroots;
    int64_t ntasks[3];
};

// Per-launch control block in device memory: the shared chunk counter, a
// status word (1 = deadline expired), and the deadline on the GPU's global
// timer (0 = none), written on the device by the arming kernel so host and
// device clocks never need to agree.
struct Control {
    unsigned long long work;      // first-pass chunk counter
    int status;
    int fault;                    // non-zero: a pass found its inputs inconsistent
    unsigned long long deadline;
    unsigned long long work2;     // second-pass piece counter
    unsigned int n_deferred;      // chunks appended to the deferred list
    unsigned int n_pieces;        // pieces of the deferred chunks (after the scan)
    unsigned long long work3;     // root counter of the wedge kernel
    unsigned long long call_deadline;  // pm_count_each: caps every pattern's deadline (0 = none)
};

// A chunk whose second-level candidate range [split, total) awaits the
// second pass.
struct Deferred {
    uint32_t chunk;
    uint32_t total;
};

}  // namespace pm
