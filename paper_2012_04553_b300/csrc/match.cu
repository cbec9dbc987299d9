// Matching kernels (sm_103a): counting and MNI-domain collection over a
// shared queue of (plan, oriented-edge chunk) tasks, plus the MNI morph
// reduction.
//
// Work decomposition.  A task chunk is one plan and 32 consecutive oriented
// edges (root, v) with v < root, roots taken highest-ranked first so hub work
// starts early.  Warps pull chunks from one global counter (persistent grid,
// one launch for every plan of every matched pattern).  A chunk whose
// flattened second-level candidate range exceeds the plan's split size keeps
// only the first `split` candidates and appends the rest to a deferred list;
// a scan kernel turns the list into split-sized pieces that a second pass
// of the same kernel spreads over all warps (hub roots otherwise leave a
// few warps running long after the rest have finished).
//
// Set operations.  A level's candidate set is never materialised: it is the
// bounded slice of the smallest intersected adjacency list, cut by two binary
// searches to the (gt, lt) id window, and filtered one element per lane
// (membership in the other intersected lists and absence from the
// differenced lists by binary search; injectivity and label tests).  Each
// warp buffers up to 64 prefixes per level in shared memory and flattens the
// slices of all buffered prefixes into one index space, so a step always
// gives every lane a (prefix, candidate) pair whatever the set sizes;
// survivors are compacted with __ballot_sync into the next level's buffer,
// which is expanded as soon as it holds 32 prefixes (depth-first over
// batches).  The last `tail` levels are counted as C(|C|, tail); when C is
// one adjacency range minus known vertices, |C| comes from binary searches
// alone, one prefix per lane.
//
// Aggregation.  Counts accumulate per lane in 128 bits, are summed across the
// warp, and are added to the pattern's 128-bit counter with a carry into the
// high word, so totals are exact modulo 2^128.  MNI domains are n-bit bitsets
// per (matched pattern, column) set with atomicOr, skipping words whose bit is
// already set.
#include <climits>
#include <cstdio>

#include "devgraph.cuh"
#include "internal.hpp"

namespace pm {

constexpr int CAP = 64;       // prefixes per level buffer
constexpr int WARPS = 4;      // warps per block

// Bound vertices of levels 0..L in registers; every access uses a
// compile-time index (unrolled loops) so the array never leaves registers.
struct Bound {
    int32_t v[PLAN_KMAX];
    __device__ __forceinline__ int32_t get(int j) const {
        int32_t r = 0;
#pragma unroll
        for (int i = 0; i < PLAN_KMAX; i++)
            if (i == j) r = v[i];
        return r;
    }
    __device__ __forceinline__ void set(int j, int32_t x) {
#pragma unroll
        for (int i = 0; i < PLAN_KMAX; i++)
            if (i == j) v[i] = x;
    }
};

struct Slice {
    uint32_t base;     // index into col
    int32_t len;
    int32_t src;
    int32_t lo, hi;    // open id window (lo, hi)
};

// Candidate slice of level `lv` given the bound prefix.
__device__ __forceinline__ Slice make_slice(const DevGraph &g, const DevLevel &lv, const Bound &m) {
    Slice s;
    int32_t hi = INT_MAX, lo = -1;
    int best = -1;
    int32_t bestd = INT_MAX;
    int64_t bestb = 0;
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if ((lv.lt >> j) & 1) hi = min(hi, m.v[j]);
        if ((lv.gt >> j) & 1) lo = max(lo, m.v[j]);
        if ((lv.isect >> j) & 1) {
            const int64_t b = __ldg(g.rowptr + m.v[j]);
            const int32_t d = int32_t(__ldg(g.rowptr + m.v[j] + 1) - b);
            if (d < bestd) { bestd = d; best = j; bestb = b; }
        }
    }
    s.lo = lo;
    s.hi = hi;
    if (best < 0) {   // no intersected list: cannot happen for levels >= 1
        s.base = 0; s.len = 0; s.src = 0;
        return s;
    }
    const int32_t *a = g.col + bestb;
    const int32_t a0 = lo < 0 ? 0 : lower_bound_dev(a, bestd, lo + 1);
    const int32_t a1 = hi == INT_MAX ? bestd : lower_bound_dev(a, bestd, hi);
    s.base = uint32_t(bestb + a0);
    s.len = a1 > a0 ? a1 - a0 : 0;
    s.src = best;
    return s;
}

__device__ __forceinline__ bool admissible(const DevGraph &g, const DevLevel &lv, int src,
                                           const Bound &m, int32_t x) {
    if (lv.label >= 0 && __ldg(g.labels + x) != uint8_t(lv.label)) return false;
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if (((lv.neq >> j) & 1) && x == m.v[j]) return false;
    }
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if (((lv.isect >> j) & 1) && j != src && !contains(g, m.v[j], x)) return false;
        if (((lv.diff >> j) & 1) && contains(g, m.v[j], x)) return false;
    }
    return true;
}

// |C| for a closed final stage: slice length minus the excluded bound
// vertices that fall inside the slice.
__device__ __forceinline__ int64_t closed_count(const DevGraph &g, const DevLevel &lv,
                                                const Bound &m) {
    const Slice s = make_slice(g, lv, m);
    int64_t c = s.len;
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if ((lv.neq >> j) & 1) {
            const int32_t v = m.v[j];
            if (v > s.lo && v < s.hi && contains(g, m.get(s.src), v)) c--;
        }
    }
    return c;
}

__device__ __forceinline__ void set_bit(uint32_t *bits, int32_t x) {
    uint32_t *w = bits + (x >> 5);
    const uint32_t b = 1u << (x & 31);
    if (!(*(volatile uint32_t *)w & b)) atomicOr(w, b);
}

// Exact C(c, r) for r <= 6: 64-bit arithmetic for r <= 2, otherwise the
// 128-bit falling product divided by r! with 32-bit-digit long division.
__device__ __forceinline__ u128 binom_fast(int64_t c, int r) {
    if (r <= 0) return r == 0 ? 1 : 0;
    if (c < r) return 0;
    const uint64_t uc = uint64_t(c);
    if (r == 1) return uc;
    if (r == 2) return (uc & 1) ? u128(uc) * ((uc - 1) >> 1) : u128(uc >> 1) * (uc - 1);
    u128 num = 1;
    uint32_t den = 1;
    for (int i = 0; i < r; i++) {
        num *= u128(uc - uint64_t(i));
        den *= uint32_t(i + 1);
    }
    uint64_t rem = 0;
    u128 q = 0;
#pragma unroll
    for (int d = 3; d >= 0; d--) {
        const uint64_t cur = (rem << 32) | uint64_t(uint32_t(num >> (32 * d)));
        q |= u128(cur / den) << (32 * d);
        rem = cur % den;
    }
    return q;
}

// ---------------------------------------------------------------------------
// Warp-batched depth-first enumeration (see the file comment).

struct LevelBuf {
    int32_t v[CAP];
    uint32_t base[CAP];    // slice start (index into col) for the next level
    int32_t scan[CAP];     // inclusive prefix sum of slice lengths
    uint8_t parent[CAP];
    uint8_t src[CAP];      // intersected level used as the slice source
    int32_t cnt, t, total, pad;
};

struct WarpTail {
    int32_t fcount[CAP];   // per-prefix final-stage counts / flags
};

__device__ __forceinline__ Bound tuple_of(const LevelBuf *B, int L, int p) {
    Bound m;
    int q = p;
#pragma unroll
    for (int l = PLAN_KMAX - 1; l >= 0; l--) {
        m.v[l] = 0;
        if (l <= L) {
            m.v[l] = B[l].v[q];
            q = B[l].parent[q];
        }
    }
    return m;
}

// Warp-wide inclusive scan over the (up to 64) slice lengths of a buffer.
__device__ __forceinline__ void store_scan(LevelBuf &b, int lane, int32_t len0, int32_t len1) {
    int32_t a = len0, c = len1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t ya = __shfl_up_sync(FULL, a, off);
        const int32_t yc = __shfl_up_sync(FULL, c, off);
        if (lane >= off) { a += ya; c += yc; }
    }
    const int32_t first = __shfl_sync(FULL, a, 31);
    b.scan[lane] = a;
    b.scan[lane + 32] = c + first;
}

template <bool STATS>
__device__ __forceinline__ uint64_t operand_bytes(const DevGraph &g, const DevLevel &lv,
                                                  const Slice &s, const Bound &m) {
    if (!STATS) return 0;
    uint64_t bytes = 4ull * uint64_t(s.len) + 16;
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if ((((lv.isect >> j) & 1) && j != s.src) || ((lv.diff >> j) & 1)) {
            const int64_t b = __ldg(g.rowptr + m.v[j]);
            const int32_t d = int32_t(__ldg(g.rowptr + m.v[j] + 1) - b);
            const int32_t a0 = s.lo < 0 ? 0 : lower_bound_dev(g.col + b, d, s.lo + 1);
            const int32_t a1 = lower_bound_dev(g.col + b, d, s.hi);
            bytes += 16 + 4ull * uint64_t(a1 > a0 ? a1 - a0 : 0);
        }
    }
    return bytes;
}

// Slices of buffer L's prefixes for the level with constraints `nl` (the
// next level, or a pair's merged level), and their scan.
template <bool STATS>
__device__ __forceinline__ void setup_level_with(const DevGraph &g, const DevLevel &nl, LevelBuf *B,
                                                 int L, int lane, uint64_t &stat) {
    LevelBuf &b = B[L];
    const int cnt = b.cnt;
    int32_t lens[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int p = lane + 32 * h;
        if (p < cnt) {
            const Bound m = tuple_of(B, L, p);
            const Slice s = make_slice(g, nl, m);
            b.base[p] = s.base;
            b.src[p] = uint8_t(s.src);
            lens[h] = s.len;
            stat += operand_bytes<STATS>(g, nl, s, m);
        }
    }
    store_scan(b, lane, lens[0], lens[1]);
    __syncwarp();
    if (lane == 0) {
        b.t = 0;
        b.total = cnt > 0 ? b.scan[cnt - 1] : 0;
    }
    __syncwarp();
}

template <bool STATS>
__device__ __forceinline__ void setup_level(const DevGraph &g, const DevPlan &P, LevelBuf *B, int L,
                                            int lane, uint64_t &stat) {
    setup_level_with<STATS>(g, P.lv[L + 1], B, L, lane, stat);
}

// Prefix that owns flattened candidate index e of a buffer.
__device__ __forceinline__ int prefix_of(const LevelBuf &b, int32_t e) {
    int lo = 0, hi = b.cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (b.scan[mid] <= e) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool deadline_hit(uint64_t deadline, int *status, int lane, uint32_t &tick) {
    if (!deadline || ((++tick & 63u) != 0)) return false;
    int hit = 0;
    if (lane == 0) {
        hit = *(volatile int *)status;
        if (!hit && global_ns() > deadline) {
            atomicExch(status, 1);
            hit = 1;
        }
    }
    return __shfl_sync(FULL, hit, 0) != 0;
}

// Listing output (pm_enumerate): every match a listing plan reaches is
// written as PLAN_KMAX caller vertex ids indexed by pattern vertex, with the
// matched pattern's index as its tag, at a slot taken from a shared cursor
// (matches past `cap` are counted but not written).
struct ListOut {
    int32_t *out;
    int32_t *tag;
    unsigned long long *cursor;
    int64_t cap;
    const int32_t *old_of;    // internal id -> caller id
};

__device__ __forceinline__ void emit_match(const ListOut &lo, const DevPlan &P, const Bound &m, int L,
                                           int32_t x, bool with_x) {
    const unsigned long long pos = atomicAdd(lo.cursor, 1ull);
    if (pos >= (unsigned long long)lo.cap) return;
    int32_t *t = lo.out + int64_t(pos) * PLAN_KMAX;
#pragma unroll
    for (int l = 0; l < PLAN_KMAX; l++)
        if (l <= L) t[P.lv[l].vertex] = __ldg(lo.old_of + m.v[l]);
    if (with_x) t[P.lv[L + 1].vertex] = __ldg(lo.old_of + x);
    lo.tag[pos] = P.counter;
}

// Final stage over the prefixes of buffer L: levels n_enum .. k-1 counted.
// For the flattened (scanned) stage only candidates [t_begin, t_end) are
// visited; a range narrower than the whole buffer is used only when
// tail == 1 in counting mode, where partial counts add up.
template <bool DOMAINS, bool STATS, bool LIST>
__device__ bool final_stage(const DevGraph &g, const DevPlan &P, LevelBuf *B, WarpTail &T, int L,
                            int32_t t_begin, int32_t t_end, int lane, u128 &acc, uint64_t &stat,
                            uint32_t *bitsets, int64_t words, uint64_t deadline, int *status,
                            uint32_t &tick, const ListOut &lo) {
    LevelBuf &b = B[L];
    const int cnt = b.cnt;
    if (P.tail == 0) {   // k == 2: each prefix is a match
        if (LIST) {
            for (int p = lane; p < cnt; p += 32) emit_match(lo, P, tuple_of(B, L, p), L, 0, false);
        } else if (DOMAINS) {
            for (int p = lane; p < cnt; p += 32) {
                const Bound m = tuple_of(B, L, p);
#pragma unroll
                for (int l = 0; l < 2; l++)
                    set_bit(bitsets + int64_t(P.dom_base + P.lv[l].column) * words, m.v[l]);
            }
        } else if (lane == 0) {
            acc += uint64_t(cnt);
        }
        return true;
    }
    const DevLevel &lv = P.lv[P.n_enum];
    if (!DOMAINS && P.pair) {
        // |A| * |B| per prefix (once per chunk), minus collisions A n B (scanned)
        if (t_begin == 0) {
            const DevLevel &lb = P.lv[P.n_enum + 1];
            for (int p = lane; p < cnt; p += 32) {
                const Bound m = tuple_of(B, L, p);
                acc += u128(uint64_t(closed_count(g, lv, m))) * u128(uint64_t(closed_count(g, lb, m)));
                if (STATS) stat += 48 + 8ull * (__popc(lv.neq) + __popc(lb.neq));
            }
        }
        const DevLevel &lm = P.lv[P.k];
        setup_level_with<STATS>(g, lm, B, L, lane, stat);
        const int32_t total = min(b.total, t_end);
        for (int32_t t0 = t_begin; t0 < total; t0 += 32) {
            if (deadline_hit(deadline, status, lane, tick)) return false;
            const int32_t e = t0 + lane;
            if (e < total) {
                const int p = prefix_of(b, e);
                const int32_t off = e - (p ? b.scan[p - 1] : 0);
                const int32_t x = __ldg(g.col + b.base[p] + off);
                const Bound m = tuple_of(B, L, p);
                if (admissible(g, lm, b.src[p], m, x)) acc -= 1;
            }
        }
        __syncwarp();
        return true;
    }
    if (!DOMAINS && P.closed) {
        for (int p = lane; p < cnt; p += 32) {
            const Bound m = tuple_of(B, L, p);
            acc += binom_fast(closed_count(g, lv, m), P.tail);
            if (STATS) stat += 24 + 8ull * __popc(lv.neq);
        }
        return true;
    }
    setup_level<STATS>(g, P, B, L, lane, stat);
    const int32_t total = min(b.total, t_end);
    const int passes = (DOMAINS && P.tail > 1) ? 2 : 1;
    for (int pass = 0; pass < passes; pass++) {
        const bool counting = DOMAINS ? (pass == 0 && P.tail > 1) : true;
        if (pass == 0)
            for (int p = lane; p < CAP; p += 32) T.fcount[p] = 0;
        __syncwarp();
        uint32_t *tail_bits = DOMAINS ? bitsets + int64_t(P.dom_base + lv.column) * words : nullptr;
        for (int32_t t0 = t_begin; t0 < total; t0 += 32) {
            if (deadline_hit(deadline, status, lane, tick)) return false;
            const int32_t e = t0 + lane;
            bool ok = false;
            int p = 0;
            int32_t x = 0;
            if (e < total) {
                p = prefix_of(b, e);
                const int32_t off = e - (p ? b.scan[p - 1] : 0);
                x = __ldg(g.col + b.base[p] + off);
                const Bound m = tuple_of(B, L, p);
                ok = admissible(g, lv, b.src[p], m, x);
            }
            if (LIST) {
                if (ok) emit_match(lo, P, tuple_of(B, L, p), L, x, true);
            } else if (!DOMAINS && P.tail == 1) {
                if (ok) acc += 1;
            } else if (counting) {
                if (ok) atomicAdd(&T.fcount[p], 1);
            } else {
                // record domains: tail == 1 flags the prefix; tail > 1 needs >= tail survivors
                if (ok && (P.tail == 1 || T.fcount[p] >= P.tail)) {
                    set_bit(tail_bits, x);
                    if (P.tail == 1) T.fcount[p] = 1;
                }
            }
        }
        __syncwarp();
    }
    if (!DOMAINS && P.tail > 1) {
        for (int p = lane; p < cnt; p += 32) acc += binom_fast(T.fcount[p], P.tail);
    }
    if (DOMAINS) {
        for (int p = lane; p < cnt; p += 32) {
            if (T.fcount[p] >= (P.tail > 1 ? P.tail : 1)) {
                const Bound m = tuple_of(B, L, p);
#pragma unroll
                for (int l = 0; l < PLAN_KMAX; l++)
                    if (l < P.n_enum)
                        set_bit(bitsets + int64_t(P.dom_base + P.lv[l].column) * words, m.v[l]);
            }
        }
    }
    __syncwarp();
    return true;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int mask) {
    const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(v), mask);
    const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(v >> 64), mask);
    return (u128(hi) << 64) | lo;
}

struct KernelArgs {
    DevGraph g;
    const DevPlan *plans;
    int nplans;
    int n_buf;
    DevTasks tasks;
    int64_t n_echunks;          // 32-task chunks per plan in the first pass
    int32_t sample_stride;      // first pass visits chunks (c / nplans) % stride == 0 only
    uint64_t *counters;
    uint32_t *bitsets;
    int64_t words;
    Control *ctl;
    Deferred *defer;            // deferred chunks (first pass appends, second pass reads)
    uint32_t defer_cap;
    const uint32_t *piece_off;  // exclusive scan of pieces per deferred chunk
    unsigned long long *stats;
    ListOut list;               // listing instance only
    // per plan: first-pass chunks finished, second-pass pieces finished and
    // pieces made (3 x nplans), or nullptr: a plan whose counts fall short
    // was cut by the deadline (per-pattern deadlines in one launch)
    unsigned int *plan_done;
};

// One chunk (plan c % nplans, oriented edges (c / nplans) * 32 + 0..31),
// restricted to flattened second-level candidates [t_begin, t_end).  In the
// first pass (may_defer) a range larger than the plan's split is cut to the
// split and the remainder deferred.  Returns false once the deadline expired.
template <bool DOMAINS, bool STATS, bool LIST>
__device__ bool process_chunk(const KernelArgs &A, LevelBuf *B, WarpTail &T, unsigned long long c,
                              int32_t t_begin, int32_t t_end, bool may_defer, int lane,
                              uint64_t deadline, uint32_t &tick, uint64_t &stat) {
    const DevGraph &g = A.g;
    int *status = &A.ctl->status;
    const DevPlan &P = A.plans[c % A.nplans];
    const int64_t e = int64_t(c / A.nplans) * 32 + lane;
    const int sp = P.task_space;
    const int64_t *off = A.tasks.off[sp];
    int32_t root = -1, v1 = -1;
    if (e < A.tasks.ntasks[sp]) {
        int64_t lo = 0, hi = A.tasks.nroots;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(off + mid) <= e) lo = mid;
            else hi = mid;
        }
        root = A.tasks.roots ? __ldg(A.tasks.roots + lo) : int32_t(g.n - 1 - lo);
        const int64_t idx = e - __ldg(off + lo);
        // lower and all-neighbour tasks index the row from its start, higher
        // neighbour tasks from the first neighbour above the root
        const int64_t row = sp == TASKS_UPPER
            ? __ldg(g.rowptr + root + 1) - (__ldg(off + lo + 1) - __ldg(off + lo))
            : __ldg(g.rowptr + root);
        v1 = __ldg(g.col + row + idx);
        if (P.lv[0].label >= 0 && __ldg(g.labels + root) != uint8_t(P.lv[0].label)) root = -1;
        if (P.lv[1].label >= 0 && __ldg(g.labels + v1) != uint8_t(P.lv[1].label)) root = -1;
        if (STATS && may_defer) stat += 28;   // a second-pass piece re-reads its chunk's tasks
    }
    // tasks -> buffers 0 (roots) and 1 (second vertices)
    const uint32_t vm = __ballot_sync(FULL, root >= 0);
    if (root >= 0) {
        const int pos = __popc(vm & ((1u << lane) - 1));
        B[0].v[pos] = root;
        B[0].parent[pos] = 0;
        B[1].v[pos] = v1;
        B[1].parent[pos] = uint8_t(pos);
    }
    if (lane == 0) {
        B[0].cnt = B[1].cnt = __popc(vm);
        for (int l = 2; l < A.n_buf; l++) B[l].cnt = 0;
    }
    __syncwarp();
    if (!vm) return true;
    u128 acc = 0;
    bool alive = true;
    // second-level ranges may be split when the final stage adds up partial
    // counts (n_enum > 2) or counts a single scanned level one by one
    const bool splittable =
        P.n_enum > 2 || (!DOMAINS && ((!P.closed && P.tail == 1) || P.pair));
    if (!splittable) {
        alive = final_stage<DOMAINS, STATS, LIST>(g, P, B, T, 1, 0, INT_MAX, lane, acc, stat, A.bitsets,
                                                 A.words, deadline, status, tick, A.list);
    } else {
        uint64_t resetup = 0;
        // the split range is over the second level's candidates, or, for a
        // pair final right after the task, over the collisions it scans
        const DevLevel &first = (P.n_enum == 2 && P.pair && !DOMAINS) ? P.lv[P.k] : P.lv[2];
        setup_level_with<STATS>(g, first, B, 1, lane, may_defer ? stat : resetup);
        const int32_t T1 = B[1].total;
        int32_t t_end_eff = min(t_end, T1);
        if (may_defer && T1 > P.split) {
            if (lane == 0) {
                const uint32_t slot = atomicAdd(&A.ctl->n_deferred, 1u);
                if (slot < A.defer_cap) {
                    A.defer[slot].chunk = uint32_t(c);
                    A.defer[slot].total = uint32_t(T1);
                    t_end_eff = P.split;
                }
            }
            t_end_eff = __shfl_sync(FULL, t_end_eff, 0);
        }
        if (P.n_enum == 2) {
            alive = final_stage<DOMAINS, STATS, LIST>(g, P, B, T, 1, t_begin, t_end_eff, lane, acc, stat,
                                                     A.bitsets, A.words, deadline, status, tick, A.list);
        } else {
            if (lane == 0) {
                B[1].t = t_begin;
                B[1].total = t_end_eff;
            }
            __syncwarp();
            int L = 1;
            while (alive) {
                if (L + 1 == P.n_enum) {
                    alive = final_stage<DOMAINS, STATS, LIST>(g, P, B, T, L, 0, INT_MAX, lane, acc,
                                                             stat, A.bitsets, A.words, deadline,
                                                             status, tick, A.list);
                    if (lane == 0) B[L].cnt = 0;
                    __syncwarp();
                    L--;
                    continue;
                }
                LevelBuf &b = B[L];
                LevelBuf &nb = B[L + 1];
                const int32_t t = b.t, tot = b.total, ncnt = nb.cnt;
                if (t < tot && ncnt < 32) {
                    if (deadline_hit(deadline, status, lane, tick)) { alive = false; break; }
                    const int32_t ei = t + lane;
                    bool ok = false;
                    int p = 0;
                    int32_t x = 0;
                    if (ei < tot) {
                        p = prefix_of(b, ei);
                        const int32_t off = ei - (p ? b.scan[p - 1] : 0);
                        x = __ldg(g.col + b.base[p] + off);
                        const Bound m = tuple_of(B, L, p);
                        ok = admissible(g, P.lv[L + 1], b.src[p], m, x);
                    }
                    const uint32_t sm = __ballot_sync(FULL, ok);
                    if (ok) {
                        const int pos = ncnt + __popc(sm & ((1u << lane) - 1));
                        nb.v[pos] = x;
                        nb.parent[pos] = uint8_t(p);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        nb.cnt = ncnt + __popc(sm);
                        b.t = t + 32;
                    }
                    __syncwarp();
                    continue;
                }
                if (ncnt > 0 && (ncnt >= 32 || t >= tot)) {
                    L++;
                    if (L + 1 < P.n_enum) setup_level<STATS>(g, P, B, L, lane, stat);
                    continue;
                }
                if (lane == 0) b.cnt = 0;
                __syncwarp();
                L--;
                if (L < 1) break;
            }
        }
    }
    if (!DOMAINS && !LIST) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += shfl_xor_u128(acc, off);
        if (lane == 0 && acc != 0) add_u128(A.counters + 2 * int64_t(P.counter), acc);
    }
    return alive;
}

// pass 0: chunks from the shared counter (deferring oversized ranges);
// pass 1: split-sized pieces of the deferred chunks.
template <bool DOMAINS, bool STATS, bool LIST>
__global__ void __launch_bounds__(WARPS * 32)
match_kernel(KernelArgs A, int pass) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t per_warp = sizeof(LevelBuf) * A.n_buf + sizeof(WarpTail);
    LevelBuf *B = reinterpret_cast<LevelBuf *>(smem + per_warp * warp);
    WarpTail &T = *reinterpret_cast<WarpTail *>(smem + per_warp * warp + sizeof(LevelBuf) * A.n_buf);
    Control *ctl = A.ctl;
    int *status = &ctl->status;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const unsigned long long stride = (unsigned long long)(A.sample_stride > 1 ? A.sample_stride : 1);
    const unsigned long long n_sampled = ((unsigned long long)A.n_echunks + stride - 1) / stride;
    const unsigned long long total = pass == 0
        ? n_sampled * (unsigned long long)A.nplans
        : (unsigned long long)(*(volatile uint32_t *)&ctl->n_pieces);
    const uint32_t n_def = pass == 0 ? 0u
        : min(*(volatile uint32_t *)&ctl->n_deferred, A.defer_cap);
    uint32_t tick = 0;
    uint64_t stat = 0;
    while (true) {
        unsigned long long w = 0;
        int stop = 0;
        if (lane == 0) {
            w = atomicAdd(pass == 0 ? &ctl->work : &ctl->work2, 1ull);
            stop = *(volatile int *)status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(status, 1);
                stop = 1;
            }
        }
        w = __shfl_sync(FULL, w, 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (w >= total || stop) break;
        bool alive;
        if (pass == 0) {
            const unsigned long long c = (w / A.nplans) * stride * A.nplans + w % A.nplans;
            alive = process_chunk<DOMAINS, STATS, LIST>(A, B, T, c, 0, INT_MAX, true, lane, deadline,
                                                       tick, stat);
        } else {
            // piece w: deferred chunk i with piece_off[i] <= w < piece_off[i+1]
            uint32_t lo = 0, hi = n_def;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(A.piece_off + mid) <= w) lo = mid;
                else hi = mid;
            }
            const unsigned long long chunk = A.defer[lo].chunk;
            const uint32_t tot = A.defer[lo].total;
            const DevPlan &P = A.plans[chunk % A.nplans];
            const int32_t j = int32_t(w - __ldg(A.piece_off + lo)) + 1;   // piece 0 ran in pass 0
            const int32_t tb = j * P.split;
            const int32_t te = min(int32_t(tot), tb + P.split);
            alive = process_chunk<DOMAINS, STATS, LIST>(A, B, T, chunk, tb, te, false, lane, deadline,
                                                       tick, stat);
        }
        if (!alive) break;
        if (A.plan_done && lane == 0) {
            const unsigned long long chunk = pass == 0 ? w % A.nplans : 0;
            if (pass == 0) {
                atomicAdd(A.plan_done + chunk, 1u);
            } else {
                uint32_t lo = 0, hi = n_def;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (__ldg(A.piece_off + mid) <= w) lo = mid;
                    else hi = mid;
                }
                atomicAdd(A.plan_done + A.nplans + A.defer[lo].chunk % A.nplans, 1u);
            }
        }
    }
    if (STATS) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) stat += __shfl_xor_sync(FULL, stat, off);
        if (lane == 0) atomicAdd(A.stats, (unsigned long long)stat);
    }
}

// Pieces per deferred chunk (all but the first) -> exclusive scan (one block).
__global__ void piece_scan_kernel(const Deferred *defer, uint32_t cap, const DevPlan *plans,
                                  int nplans, uint32_t *piece_off, Control *ctl,
                                  unsigned int *plan_done) {
    __shared__ uint32_t partial[1024];
    const uint32_t n = min(*(volatile uint32_t *)&ctl->n_deferred, cap);
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(n, b + per);
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; i++) {
        const uint32_t split = uint32_t(plans[defer[i].chunk % nplans].split);
        sum += (defer[i].total + split - 1) / split - 1;
    }
    partial[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (unsigned t = 0; t < blockDim.x; t++) {
            const uint32_t v = partial[t];
            partial[t] = run;
            run += v;
        }
        ctl->n_pieces = run;
    }
    __syncthreads();
    uint32_t run = partial[threadIdx.x];
    for (uint32_t i = b; i < e; i++) {
        piece_off[i] = run;
        const uint32_t split = uint32_t(plans[defer[i].chunk % nplans].split);
        const uint32_t pieces = (defer[i].total + split - 1) / split - 1;
        run += pieces;
        if (plan_done && pieces) atomicAdd(plan_done + 2 * nplans + defer[i].chunk % nplans, pieces);
    }
}

// Per-pattern deadlines in one launch: after the launch, every plan with a
// first-pass chunk or a second-pass piece left unfinished flags its
// pattern; then the control block is reset for what follows (as between
// two patterns, with the call's deadline).
__global__ void plan_flags_kernel(Control *ctl, const DevPlan *plans, int nplans,
                                  const unsigned int *plan_done, unsigned long long n_chunks,
                                  uint8_t *timed_out) {
    if (ctl->status == 1) {
        for (int p = 0; p < nplans; p++)
            if (plan_done[p] < n_chunks || plan_done[nplans + p] < plan_done[2 * nplans + p])
                timed_out[plans[p].counter] = 1;
    }
    ctl->status = 0;
    ctl->work = 0;
    ctl->work2 = 0;
    ctl->work3 = 0;
    ctl->n_deferred = 0;
    ctl->n_pieces = 0;
    ctl->deadline = ctl->call_deadline;
}

int launch_plan_flags(Control *ctl, const DevPlan *plans, int nplans, const unsigned int *plan_done,
                      unsigned long long n_chunks, uint8_t *timed_out, void *stream) {
    plan_flags_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, plans, nplans, plan_done, n_chunks,
                                                         timed_out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// MNI morph (Theorem 3.2 with MNI tables): column c of a query is the OR of
// the matched bitsets src[src_off[c] .. src_off[c+1]); popc[c] receives the
// column size.
__global__ void mni_reduce_kernel(const uint32_t *__restrict__ bitsets, int64_t words,
                                  const int32_t *__restrict__ src_off,
                                  const int32_t *__restrict__ src, int n_columns,
                                  unsigned long long *popc) {
    const int col = blockIdx.y;
    if (col >= n_columns) return;
    const int s0 = src_off[col], s1 = src_off[col + 1];
    unsigned long long local = 0;
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += int64_t(gridDim.x) * blockDim.x) {
        uint32_t v = 0;
        for (int s = s0; s < s1; s++) v |= __ldg(bitsets + int64_t(src[s]) * words + w);
        local += __popc(v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULL, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(popc + col, local);
}

// MNI domains returned to the caller (Theorem 3.2 with MNI tables): word w
// of column c covers caller vertices 32w .. 32w + 31; each one's bit is the
// bit of its internal id in the OR of the column's matched bitsets.
__global__ void mni_domains_kernel(const uint32_t *__restrict__ bitsets, int64_t words,
                                   const int32_t *__restrict__ src_off,
                                   const int32_t *__restrict__ src, int n_columns,
                                   const int32_t *__restrict__ new_id, int64_t n,
                                   uint32_t *__restrict__ out) {
    const int col = blockIdx.y;
    if (col >= n_columns) return;
    const int s0 = src_off[col], s1 = src_off[col + 1];
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += int64_t(gridDim.x) * blockDim.x) {
        uint32_t word = 0;
        const int64_t v0 = w * 32;
        const int nv = int(n - v0 < 32 ? n - v0 : 32);
        for (int j = 0; j < nv; j++) {
            const int32_t iv = __ldg(new_id + v0 + j);
            uint32_t bit = 0;
            for (int s = s0; s < s1 && !bit; s++)
                bit = (__ldg(bitsets + int64_t(src[s]) * words + (iv >> 5)) >> (iv & 31)) & 1u;
            word |= bit << j;
        }
        out[int64_t(col) * words + w] = word;
    }
}

int device_sm_count(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return sms;
}

// Wedge-pair counting for the edge-induced 4-cycle (see PlanKind).  For the
// root a and every 2-path a-b-c with b, c < a, an atomicAdd on a per-c
// counter returns the old value, whose running sum is sum_c C(w_c, 2).
// Roots split by rank: the 2-paths concentrate on the highest-ranked roots
// (on R-MAT scale 20 the top 16,384 of 2^20 roots carry 99 % of them).
//
// Heavy roots (a >= heavy_from): one block per root keeps the counters in
// shared memory for a window [w0, w0 + W) of c at a time.  Every lower
// neighbour b with neighbours below a is an entry (cursor, end) into b's
// row; a window consumes, warp by warp, each entry's run of c inside the
// window (a prefix of what is left, rows being sorted), keeps unfinished
// entries for the next window and starts that window at their smallest c,
// so empty stretches of ids cost nothing and no counter touches DRAM.
//
// Light roots (a < heavy_from): one block per root with dense per-c
// counters in global memory (blocks x n); warps take lower neighbours b,
// lanes the neighbours c < a of b, and a second walk over the same 2-paths
// resets the touched counters to zero.
constexpr int WEDGE_THREADS = 512;
constexpr int WH_THREADS = 1024;
constexpr int WH_W = 53248;          // counters per window (208 KiB of shared memory)

__global__ void __launch_bounds__(WEDGE_THREADS)
wedge_pairs_kernel(DevGraph g, DevTasks tasks, int64_t heavy_from, int counter, uint64_t *counters,
                   uint32_t *scratch, int sample_stride, Control *ctl) {
    __shared__ unsigned long long s_root;
    __shared__ int s_stop;
    __shared__ unsigned long long s_acc[WEDGE_THREADS / 32];
    uint32_t *cnt = scratch + size_t(blockIdx.x) * size_t(g.n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const int64_t stride = sample_stride > 1 ? sample_stride : 1;
    const int64_t nr = (tasks.nroots + stride - 1) / stride;
    unsigned long long acc = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_root = atomicAdd(&ctl->work3, 1ull);
            int stop = *(volatile int *)&ctl->status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(&ctl->status, 1);
                stop = 1;
            }
            s_stop = stop;
        }
        __syncthreads();
        const int64_t r = int64_t(s_root) * stride;
        const bool done = s_root >= (unsigned long long)nr || s_stop;
        __syncthreads();
        if (done) break;
        const int32_t a = tasks.roots ? __ldg(tasks.roots + r) : int32_t(g.n - 1 - r);
        if (a >= heavy_from) continue;                 // counted by the heavy-root kernel
        const int32_t lo = int32_t(__ldg(tasks.off[0] + r + 1) - __ldg(tasks.off[0] + r));
        const int64_t abase = __ldg(g.rowptr + a);
        for (int pass = 0; pass < 2; pass++) {
            for (int i = warp; i < lo; i += nwarps) {
                const int32_t b = __ldg(g.col + abase + i);
                const int64_t bb = __ldg(g.rowptr + b);
                const int32_t bd = int32_t(__ldg(g.rowptr + b + 1) - bb);
                const int32_t bl = lower_bound_dev(g.col + bb, bd, a);   // neighbours of b below a
                for (int32_t j = lane; j < bl; j += 32) {
                    const int32_t c = __ldg(g.col + bb + j);
                    if (pass == 0) acc += atomicAdd(cnt + c, 1u);
                    else cnt[c] = 0;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 total = 0;
        for (int w = 0; w < nwarps; w++) total += s_acc[w];
        if (total) add_u128(counters + 2 * int64_t(counter), total);
    }
}

// lists: per block two entry lists of list_cap (cursor, end) pairs, list_cap
// >= the largest degree.
__global__ void __launch_bounds__(WH_THREADS, 1)
wedge_heavy_kernel(DevGraph g, DevTasks tasks, int64_t heavy_from, int counter,
                   uint64_t *counters, uint2 *lists, int64_t list_cap, int sample_stride,
                   Control *ctl) {
    extern __shared__ uint32_t wh_cnt[];
    __shared__ unsigned long long s_root;
    __shared__ int s_stop;
    __shared__ int s_n[2];
    __shared__ int s_minc[2];
    __shared__ unsigned long long s_acc[WH_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    uint2 *const L0 = lists + size_t(blockIdx.x) * 2 * size_t(list_cap);
    uint2 *const L1 = L0 + list_cap;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const int64_t stride = sample_stride > 1 ? sample_stride : 1;
    const int64_t nr = (tasks.nroots + stride - 1) / stride;
    unsigned long long acc = 0;
    for (;;) {
        if (tid == 0) {
            s_root = atomicAdd(&ctl->work2, 1ull);
            int stop = *(volatile int *)&ctl->status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(&ctl->status, 1);
                stop = 1;
            }
            s_stop = stop;
            s_n[0] = 0;
            s_minc[0] = INT_MAX;
        }
        __syncthreads();
        const int64_t r = int64_t(s_root) * stride;
        const bool done = s_root >= (unsigned long long)nr || s_stop;
        if (done) break;
        // with the implicit root list the heavy roots are the first ones
        if (!tasks.roots && g.n - 1 - r < heavy_from) break;
        const int32_t a = tasks.roots ? __ldg(tasks.roots + r) : int32_t(g.n - 1 - r);
        if (a < heavy_from) {
            __syncthreads();
            continue;
        }
        const int32_t lo = int32_t(__ldg(tasks.off[0] + r + 1) - __ldg(tasks.off[0] + r));
        const int64_t abase = __ldg(g.rowptr + a);
        for (int i = tid; i < lo; i += blockDim.x) {
            const int32_t b = __ldg(g.col + abase + i);
            const int64_t bb = __ldg(g.rowptr + b);
            const int32_t bl = lower_bound_dev(g.col + bb, int32_t(__ldg(g.rowptr + b + 1) - bb), a);
            if (bl > 0) {
                const int slot = atomicAdd(&s_n[0], 1);
                L0[slot] = make_uint2(uint32_t(bb), uint32_t(bb + bl));
                atomicMin(&s_minc[0], __ldg(g.col + bb));
            }
        }
        __syncthreads();
        int cur = 0;
        int nact = s_n[0];
        int64_t w0 = s_minc[0];
        while (nact > 0) {
            for (int j = tid; j < WH_W; j += blockDim.x) wh_cnt[j] = 0;
            if (tid == 0) {
                s_n[cur ^ 1] = 0;
                s_minc[cur ^ 1] = INT_MAX;
                int stop = *(volatile int *)&ctl->status;
                if (!stop && deadline && global_ns() > deadline) {
                    atomicExch(&ctl->status, 1);
                    stop = 1;
                }
                s_stop = stop;
            }
            __syncthreads();
            if (s_stop) break;
            const int64_t w1 = w0 + WH_W;
            for (int e = warp; e < nact; e += nwarps) {
                const uint2 en = (cur ? L1 : L0)[e];
                uint32_t p = en.x;
                for (;;) {
                    const uint32_t idx = p + uint32_t(lane);
                    const int32_t c = idx < en.y ? __ldg(g.col + idx) : INT_MAX;
                    const bool in = c < w1;              // the run inside the window is a prefix
                    if (in) acc += atomicAdd(&wh_cnt[c - w0], 1u);
                    const int k = __popc(__ballot_sync(FULL, in));
                    p += uint32_t(k);
                    if (k < 32 || p >= en.y) break;
                }
                if (lane == 0 && p < en.y) {
                    const int slot = atomicAdd(&s_n[cur ^ 1], 1);
                    (cur ? L0 : L1)[slot] = make_uint2(p, en.y);
                    atomicMin(&s_minc[cur ^ 1], __ldg(g.col + p));
                }
            }
            __syncthreads();
            nact = s_n[cur ^ 1];
            w0 = s_minc[cur ^ 1];
            cur ^= 1;
            __syncthreads();
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        u128 total = 0;
        for (int w = 0; w < nwarps; w++) total += s_acc[w];
        if (total) add_u128(counters + 2 * int64_t(counter), total);
    }
}

int wedge_blocks(int device) { return device_sm_count(device); }

int launch_wedge_pairs(const DevGraph &g, const DevTasks &tasks, int64_t heavy_from, int counter,
                       uint64_t *counters, uint32_t *scratch, uint2 *lists, int64_t list_cap,
                       int blocks, int sample_stride, Control *ctl, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(uint32_t) * WH_W;
    cudaFuncSetAttribute(wedge_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaMemsetAsync(&ctl->work2, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(&ctl->work3, 0, sizeof(unsigned long long), s);
    if (heavy_from < g.n)
        wedge_heavy_kernel<<<blocks, WH_THREADS, smem, s>>>(g, tasks, heavy_from, counter, counters,
                                                            lists, list_cap, sample_stride, ctl);
    if (heavy_from > 0)
        wedge_pairs_kernel<<<blocks, WEDGE_THREADS, 0, s>>>(g, tasks, heavy_from, counter, counters,
                                                           scratch, sample_stride, ctl);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("wedge kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

// Between the launches of two matched patterns when each pattern has its own
// deadline: records whether the previous pattern's deadline expired, then
// clears the status, resets the work counters and arms the next deadline.
__global__ void pattern_gate_kernel(Control *ctl, uint8_t *timed_out, int prev_counter,
                                    uint64_t budget_ns) {
    if (prev_counter >= 0 && ctl->status == 1) timed_out[prev_counter] = 1;
    ctl->status = 0;
    ctl->work = 0;
    ctl->work2 = 0;
    ctl->work3 = 0;
    ctl->n_deferred = 0;
    ctl->n_pieces = 0;
    const unsigned long long own = budget_ns ? global_ns() + budget_ns : 0;
    const unsigned long long cap = ctl->call_deadline;
    ctl->deadline = (own && cap) ? min(own, cap) : (own ? own : cap);
}

int launch_pattern_gate(Control *d_ctl, uint8_t *d_timed_out, int prev_counter,
                        uint64_t budget_ns, void *stream) {
    pattern_gate_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_ctl, d_timed_out, prev_counter,
                                                           budget_ns);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Resets the work counters between launches that share one armed deadline.
__global__ void rearm_kernel(Control *ctl) {
    ctl->work = 0;
    ctl->work2 = 0;
    ctl->work3 = 0;
    ctl->n_deferred = 0;
    ctl->n_pieces = 0;
}

int launch_rearm(Control *d_ctl, void *stream) {
    rearm_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void arm_kernel(Control *ctl, uint64_t budget_ns) {
    ctl->work = 0;
    ctl->work3 = 0;
    ctl->work2 = 0;
    ctl->status = 0;
    ctl->fault = 0;
    ctl->n_deferred = 0;
    ctl->n_pieces = 0;
    ctl->deadline = budget_ns ? global_ns() + budget_ns : 0;
    ctl->call_deadline = ctl->deadline;
}

int launch_arm(Control *d_ctl, uint64_t budget_ns, void *stream) {
    arm_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_ctl, budget_ns);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("arm kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

template <bool DOMAINS, bool STATS, bool LIST = false>
static int launch_match(const MatchLaunch &L, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    const int sms = device_sm_count(device);
    const int n_buf = L.max_enum < 2 ? 2 : L.max_enum;
    const size_t smem = (sizeof(LevelBuf) * n_buf + sizeof(WarpTail)) * WARPS;
    auto kern = match_kernel<DOMAINS, STATS, LIST>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t stride = L.sample_stride > 1 ? L.sample_stride : 1;
    const int64_t chunks = ((L.n_echunks + stride - 1) / stride) * int64_t(L.nplans);
    const int64_t blocks = int64_t(sms) * per_sm;
    const int64_t need = (chunks + WARPS - 1) / WARPS;
    const int64_t blocks0 = need < blocks ? (need > 0 ? need : 1) : blocks;
    KernelArgs A;
    A.g = L.g;
    A.plans = L.plans;
    A.nplans = L.nplans;
    A.n_buf = n_buf;
    A.tasks = L.tasks;
    A.n_echunks = L.n_echunks;
    A.sample_stride = L.sample_stride;
    A.counters = L.counters;
    A.bitsets = L.bitsets;
    A.words = L.words;
    A.ctl = L.ctl;
    A.defer = L.defer;
    A.defer_cap = L.defer_cap;
    A.piece_off = L.piece_off;
    A.stats = L.stats;
    A.list = ListOut{L.list_out, L.list_tag, L.list_cursor, L.list_cap, L.old_of};
    A.plan_done = L.plan_done;
    cudaStream_t s = (cudaStream_t)stream;
    kern<<<unsigned(blocks0), WARPS * 32, smem, s>>>(A, 0);
    piece_scan_kernel<<<1, 1024, 0, s>>>(L.defer, L.defer_cap, L.plans, L.nplans, L.piece_off,
                                         L.ctl, L.plan_done);
    kern<<<unsigned(blocks), WARPS * 32, smem, s>>>(A, 1);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("match kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

int launch_count(const MatchLaunch &L, void *stream) {
    if (L.stats) return launch_match<false, true>(L, stream);
    return launch_match<false, false>(L, stream);
}

int launch_domains(const MatchLaunch &L, void *stream) {
    return launch_match<true, false>(L, stream);
}

int launch_list(const MatchLaunch &L, void *stream) {
    return launch_match<false, false, true>(L, stream);
}

// Theorem 3.1 on listed matches: every listed match t of a matched pattern
// j, composed with each map f of j's list (query i, f: vertex of i -> vertex
// of j), gives the match u -> t[f[u]] of query i.
__global__ void compose_kernel(const int32_t *__restrict__ qt, const int32_t *__restrict__ qtag,
                               int64_t n_listed, const int32_t *__restrict__ map_off,
                               const int32_t *__restrict__ map_query, const uint8_t *__restrict__ map_f,
                               const int32_t *__restrict__ query_k, int32_t *out, int32_t *out_query,
                               unsigned long long *cursor, int64_t cap) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_listed;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int j = qtag[i];
        const int32_t *t = qt + i * PLAN_KMAX;
        for (int m = map_off[j]; m < map_off[j + 1]; m++) {
            const unsigned long long pos = atomicAdd(cursor, 1ull);
            if (pos >= (unsigned long long)cap) continue;
            const int q = map_query[m];
            const int k = query_k[q];
            int32_t *o = out + int64_t(pos) * PLAN_KMAX;
#pragma unroll
            for (int u = 0; u < PLAN_KMAX; u++) o[u] = u < k ? t[map_f[m * PLAN_KMAX + u]] : -1;
            out_query[pos] = q;
        }
    }
}

int launch_compose(const int32_t *qt, const int32_t *qtag, int64_t n_listed, const int32_t *map_off,
                   const int32_t *map_query, const uint8_t *map_f, const int32_t *query_k, int32_t *out,
                   int32_t *out_query, unsigned long long *cursor, int64_t cap, void *stream) {
    if (n_listed == 0) return 0;
    int device = 0;
    cudaGetDevice(&device);
    int64_t blocks = (n_listed + 255) / 256;
    if (blocks > 8 * int64_t(device_sm_count(device))) blocks = 8 * int64_t(device_sm_count(device));
    compose_kernel<<<unsigned(blocks), 256, 0, (cudaStream_t)stream>>>(
        qt, qtag, n_listed, map_off, map_query, map_f, query_k, out, out_query, cursor, cap);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mni_domains(const uint32_t *d_bitsets, int64_t words, const int32_t *d_src_off,
                       const int32_t *d_src, int n_columns, const int32_t *d_new_id, int64_t n,
                       uint32_t *out, void *stream) {
    if (n_columns == 0) return 0;
    int device = 0;
    cudaGetDevice(&device);
    const int sms = device_sm_count(device);
    int64_t bx = (words + 255) / 256;
    if (bx > 4 * sms) bx = 4 * sms;
    if (bx < 1) bx = 1;
    dim3 grid{unsigned(bx), unsigned(n_columns), 1u};
    mni_domains_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_bitsets, words, d_src_off, d_src,
                                                               n_columns, d_new_id, n, out);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("mni domains launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

// OR of n_parts bitsets of `words` words each (the per-shard MNI columns of
// a sharded support), and the popcount of each column of a set of columns.
__global__ void domains_or_kernel(const uint32_t *__restrict__ parts, int n_parts, int64_t words,
                                  uint32_t *__restrict__ out) {
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += int64_t(gridDim.x) * blockDim.x) {
        uint32_t v = 0;
        for (int p = 0; p < n_parts; p++) v |= __ldg(parts + int64_t(p) * words + w);
        out[w] = v;
    }
}

__global__ void column_popc_kernel(const uint32_t *__restrict__ cols, int64_t words, int n_columns,
                                   unsigned long long *popc) {
    const int c = blockIdx.y;
    if (c >= n_columns) return;
    unsigned long long local = 0;
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < words;
         w += int64_t(gridDim.x) * blockDim.x)
        local += __popc(__ldg(cols + int64_t(c) * words + w));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULL, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(popc + c, local);
}

int launch_domains_or(const uint32_t *parts, int n_parts, int64_t words, uint32_t *out, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    int64_t blocks = (words + 255) / 256;
    const int64_t cap = 8 * int64_t(device_sm_count(device));
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    domains_or_kernel<<<unsigned(blocks), 256, 0, (cudaStream_t)stream>>>(parts, n_parts, words, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_column_popc(const uint32_t *cols, int64_t words, int n_columns, unsigned long long *popc,
                       void *stream) {
    if (n_columns == 0) return 0;
    int device = 0;
    cudaGetDevice(&device);
    int64_t bx = (words + 255) / 256;
    if (bx > 4 * device_sm_count(device)) bx = 4 * device_sm_count(device);
    if (bx < 1) bx = 1;
    dim3 grid{unsigned(bx), unsigned(n_columns), 1u};
    column_popc_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(cols, words, n_columns, popc);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mni_reduce(const uint32_t *d_bitsets, int64_t words, const int32_t *d_src_off,
                      const int32_t *d_src, int n_columns, unsigned long long *d_popc,
                      void *stream) {
    if (n_columns == 0) return 0;
    int device = 0;
    cudaGetDevice(&device);
    const int sms = device_sm_count(device);
    int64_t bx = (words + 255) / 256;
    if (bx > 4 * sms) bx = 4 * sms;
    if (bx < 1) bx = 1;
    dim3 grid{unsigned(bx), unsigned(n_columns), 1u};
    mni_reduce_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_bitsets, words, d_src_off, d_src,
                                                              n_columns, d_popc);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("mni reduce launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

}  // namespace pm
