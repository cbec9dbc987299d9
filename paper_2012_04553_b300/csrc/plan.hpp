// Matching plans and device-side data layouts shared by host and kernels.
//
// A plan matches one pattern p with one automorphism orbit O of p pinned to
// the task's root: the root is the highest-ranked (largest internal id)
// vertex of the occurrence and is the image of O's representative.  Every
// occurrence of p has exactly one highest-ranked vertex, whose preimage lies
// in exactly one orbit, so the plans of p partition p's occurrences; within a
// plan the remaining symmetry (the stabiliser of the representative) is
// broken by ordering constraints chosen as in Grochow & Kellis (RECOMB 2007):
// at each vertex v, in matching order, v's image is the smallest over v's
// orbit under the current stabiliser, which then shrinks to fix v.
//
// Level i of a plan binds pattern vertex order[i].  Its candidates are the
// data vertices x with
//   x in N(m_j)      for every j in isect  (edges of p: set intersection)
//   x not in N(m_j)  for every j in diff   (anti-edges of p^V: set difference)
//   x < m_j (j in lt), x > m_j (j in gt)   (root bound, symmetry breaking)
//   x != m_j (j in neq)                    (injectivity not implied above)
//   label(x) == label                      (labeled patterns)
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
    uint8_t pad;
};

struct DevPlan {
    int32_t k;
    int32_t n_enum;
    int32_t tail;
    int32_t closed;
    int32_t counter;      // output slot: index of the matched pattern
    int32_t dom_base;     // first MNI bitset of the matched pattern (support plans)
    int32_t n_columns;    // MNI columns of the matched pattern
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
};

// Task space: oriented edges (root, v) with v < root, grouped by root.
// roots == nullptr means the implicit root list n-1, n-2, ..., 0 (highest
// ranked first).  off[i] = number of oriented edges of roots 0..i-1 of the
// list (nroots + 1 entries).
struct DevTasks {
    const int32_t *roots;
    const int64_t *off;
    int64_t nroots;
    int64_t ntasks;
};

// Per-launch control block in device memory: the shared chunk counter, a
// status word (1 = deadline expired), and the deadline on the GPU's global
// timer (0 = none), written on the device by the arming kernel so host and
// device clocks never need to agree.
struct Control {
    unsigned long long work;
    int status;
    int pad;
    unsigned long long deadline;
};

}  // namespace pm
