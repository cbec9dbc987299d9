// Edge-induced counts of small unlabeled patterns from local statistics
// (sm_103a): a pattern-specific way of counting the members of a morphed
// pattern set that have no anti-edges (Theorem 3.1 turns them into the
// requested vertex-induced counts).  Every count below is an exact integer
// identity over per-vertex and per-edge quantities of the data graph, so no
// occurrence is enumerated one by one; on R-MAT hubs that is the difference
// between seconds and hours.
//
// Quantities (d_v degree, t_e triangles on edge e, t_v triangles at v,
// T all triangles, S_v = sum of the neighbours' degrees):
//   triangle pass 1: t_e for every edge, by listing every triangle once from
//     its highest-ranked vertex a and second b (the third c lies in
//     N(a) n N(b) n [0, b)); written to the slot of the edge in the row of
//     its higher-ranked endpoint, then mirrored to the other endpoint's row;
//   vertex/edge pass: sums over vertices and edges of polynomials in d, t;
//   triangle pass 2: sums over triangles of products of their edges' t;
//   2-path pass (rooted at the highest-ranked vertex a of an occurrence):
//     W_a[c] = #{b in N(a): b < a, c in N(b), c < a}; 4-cycles are
//     sum_c C(W_a[c], 2), the 4-cycle sums of degrees and of edge triangle
//     counts follow from a second walk over the same 2-paths, and the
//     5-cycles with highest vertex a from sum over edges {c, x} of
//     W_a[c] W_a[x] minus the walks that repeat a vertex;
//   clique pass: 4-cliques and the sum of their vertices' degrees.
// The combination of these sums into each pattern's count is the table in
// combine_kernel.  Sums are kept modulo 2^128 (signed terms in two's
// complement), exact whenever every true count fits in 128 bits.
#include <climits>

#include "devgraph.cuh"
#include "internal.hpp"

namespace pm {

constexpr int DC_WARPS = 8;          // warps per block of the triangle and vertex passes
constexpr int P2_THREADS = 1024;     // threads per block of the 2-path pass
constexpr int32_t P2_LONG = 64;      // rows longer than this: walked by a whole warp

__device__ __forceinline__ int32_t deg_of(const DevGraph &g, int32_t v) {
    return int32_t(__ldg(g.rowptr + v + 1) - __ldg(g.rowptr + v));
}

__device__ __forceinline__ u128 c2(int64_t x) { return x >= 2 ? u128(uint64_t(x)) * uint64_t(x - 1) / 2 : 0; }
__device__ __forceinline__ u128 c3(int64_t x) {
    return x >= 3 ? u128(uint64_t(x)) * uint64_t(x - 1) * uint64_t(x - 2) / 6 : 0;
}
__device__ __forceinline__ u128 c4(int64_t x) {
    return x >= 4 ? u128(uint64_t(x)) * uint64_t(x - 1) * uint64_t(x - 2) * uint64_t(x - 3) / 24 : 0;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(v), o);
        const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(v >> 64), o);
        v += (u128(hi) << 64) | lo;
    }
    return v;
}

__device__ __forceinline__ void flush(uint64_t *basis, int idx, u128 v, int lane) {
    v = warp_sum_u128(v);
    if (lane == 0 && v != 0) add_u128(basis + 2 * idx, v);
}

// Algorithmic bytes (instrumented runs, stats != nullptr): 4 B per element of
// every list read (each operand of an intersection cut to its id window, the
// elements a binary search probes), 16 B per row-offset pair, 4 B per
// counter read or written (8 B for an atomic update).
__device__ __forceinline__ uint64_t probe_bytes(int64_t len) {
    return 4ull * uint64_t(len > 1 ? 65 - __clzll(uint64_t(len)) : 1);
}

__device__ __forceinline__ void flush_stat(unsigned long long *stats, uint64_t v, int lane) {
    if (!stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(stats, (unsigned long long)v);
}

__device__ __forceinline__ bool dc_stop(Control *ctl, uint64_t deadline, int lane) {
    int stop = 0;
    if (lane == 0) {
        stop = *(volatile int *)&ctl->status;
        if (!stop && deadline && global_ns() > deadline) {
            atomicExch(&ctl->status, 1);
            stop = 1;
        }
    }
    return __shfl_sync(FULL, stop, 0) != 0;
}

struct TriArgs {
    DevGraph g;
    DevTasks tasks;     // lower-neighbour tasks over every root
    int32_t *t;         // per CSR slot
    uint64_t *basis;
    Control *ctl;
    unsigned long long *stats;   // nullable: algorithmic bytes
    int with_c5;        // MODE 0: also the 5-cycle triangle term
};

// Triangle passes over the tasks (a, b), b < a, with the strided chunk
// mapping of the clique kernel (task c + j * n_chunks), so the tasks of one
// hub row go to different warps.  MODE 0 adds 1 to t of the three edges of
// every triangle (a, b, c), c < b, in the slots of their higher endpoints,
// and sums, for the 5-cycle correction, the neighbours of the triangle's
// vertices ranked above a.  MODE 1 reads the complete t and sums the dart
// and gem terms.
template <int MODE>
__global__ void __launch_bounds__(DC_WARPS * 32) tri_kernel(TriArgs A) {
    const int lane = threadIdx.x & 31;
    const DevGraph &g = A.g;
    Control *ctl = A.ctl;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const int64_t ntasks = A.tasks.ntasks[TASKS_LOWER];
    const int64_t *off = A.tasks.off[TASKS_LOWER];
    const unsigned long long n_chunks = (unsigned long long)((ntasks + 31) / 32);
    u128 acc0 = 0, acc1 = 0, tri = 0;
    uint64_t stat = 0;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(&ctl->work3, 1ull);
        w = __shfl_sync(FULL, w, 0);
        if (w >= n_chunks || dc_stop(ctl, deadline, lane)) break;
        const int64_t e = int64_t(w) + int64_t(lane) * int64_t(n_chunks);
        int32_t a = -1, b = -1, ia = 0, lowa = 0;
        if (e < ntasks) {
            int64_t lo = 0, hi = A.tasks.nroots;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(off + mid) <= e) lo = mid;
                else hi = mid;
            }
            a = int32_t(g.n - 1 - lo);
            ia = int32_t(e - __ldg(off + lo));
            lowa = int32_t(__ldg(off + lo + 1) - __ldg(off + lo));
            b = __ldg(g.col + __ldg(g.rowptr + a) + ia);
        }
        for (int q = 0; q < 32; q++) {
            const int32_t ra = __shfl_sync(FULL, a, q);
            const int32_t rb = __shfl_sync(FULL, b, q);
            const int32_t la = __shfl_sync(FULL, ia, q);      // = |N(a) n [0, b)|
            const int32_t lowra = __shfl_sync(FULL, lowa, q);
            if (ra < 0) break;
            const int64_t rowa = __ldg(g.rowptr + ra);
            const int64_t rowb = __ldg(g.rowptr + rb);
            const int32_t da = int32_t(__ldg(g.rowptr + ra + 1) - rowa);
            const int32_t db = int32_t(__ldg(g.rowptr + rb + 1) - rowb);
            int32_t lb = 0, pba = 0;
            if (lane == 0) {
                lb = lower_bound_dev(g.col + rowb, db, rb);
                if (MODE == 0) pba = lb + lower_bound_dev(g.col + rowb + lb, db - lb, ra);
            }
            lb = __shfl_sync(FULL, lb, 0);
            pba = __shfl_sync(FULL, pba, 0);
            if (A.stats && lane == 0) stat += 32 + 4ull * uint64_t(la <= lb ? la : lb) + (MODE == 1 ? 4 : 8);
            const int32_t n = la <= lb ? la : lb;
            if (n == 0) continue;
            const bool from_a = la <= lb;
            const int64_t src = from_a ? rowa : rowb;
            const int64_t oth = from_a ? rowb : rowa;
            const int32_t olen = from_a ? lb : la;
            // membership in the other row: one bit read when it has a hub
            // bitmap (the binary search then runs only for the triangles,
            // whose slot it finds), else the binary search itself
            const uint32_t *obits = nullptr;
            if (g.hub) {
                const int32_t h = __ldg(g.hub + (from_a ? rb : ra));
                if (h >= 0) obits = g.bits + int64_t(h) * g.words;
            }
            const int64_t up_ab = int64_t(da - lowra) + int64_t(db - pba - 1);
            int32_t t_ab = 0;
            if (MODE == 1) t_ab = __ldg(A.t + rowa + la);
            uint32_t cnt = 0;
            for (int32_t j0 = 0; j0 < n; j0 += 32) {
                const int32_t j = j0 + lane;
                if (j < n) {
                    const int32_t x = __ldg(g.col + src + j);
                    const bool maybe = !obits || ((__ldg(obits + (x >> 5)) >> (x & 31)) & 1u);
                    const int32_t p = maybe ? lower_bound_dev(g.col + oth, olen, x) : olen;
                    if (A.stats) stat += obits ? 4 : probe_bytes(olen);   // membership test
                    if (p < olen && __ldg(g.col + oth + p) == x) {
                        const int64_t s_ac = from_a ? src + j : oth + p;
                        const int64_t s_bc = from_a ? oth + p : src + j;
                        const int64_t rowx = __ldg(g.rowptr + x);
                        const int32_t dx = int32_t(__ldg(g.rowptr + x + 1) - rowx);
                        if (MODE == 0) {
                            atomicAdd(A.t + s_ac, 1);
                            atomicAdd(A.t + s_bc, 1);
                            cnt++;
                            if (A.with_c5) {
                                const int32_t pxa = lower_bound_dev(g.col + rowx, dx, ra);
                                acc0 += u128(uint64_t(up_ab + int64_t(dx - pxa - 1)));
                            }
                            if (A.stats)
                                stat += 16 + (obits ? probe_bytes(olen) : 0) + (A.with_c5 ? 16 + probe_bytes(dx) : 0);
                        } else {
                            if (A.stats) stat += 24 + (obits ? probe_bytes(olen) : 0);
                            const int64_t tac = __ldg(A.t + s_ac), tbc = __ldg(A.t + s_bc);
                            const int64_t tab = t_ab;
                            acc0 += u128(uint64_t((tab - 1) * dx + (tbc - 1) * da + (tac - 1) * db));
                            acc1 += u128(uint64_t((tab - 1) * (tac - 1))) +
                                    u128(uint64_t((tab - 1) * (tbc - 1))) +
                                    u128(uint64_t((tac - 1) * (tbc - 1)));
                        }
                    }
                }
            }
            if (MODE == 0) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
                if (lane == 0 && cnt) atomicAdd(A.t + rowa + la, int32_t(cnt));
                if (lane == 0) tri += cnt;
            }
        }
    }
    flush_stat(A.stats, stat, lane);
    if (MODE == 0) {
        flush(A.basis, DB_C5TRI, acc0, lane);
        flush(A.basis, DB_TRI, tri, lane);
    } else {
        flush(A.basis, DB_DART_TRI, acc0, lane);
        flush(A.basis, DB_GEM_TRI, acc1, lane);
    }
}

// t of every slot (u, v) with v > u from the canonical slot (v, u) in v's row.
__global__ void __launch_bounds__(DC_WARPS * 32) mirror_kernel(DevGraph g, int32_t *t,
                                                              unsigned long long *stats) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * DC_WARPS;
    uint64_t stat = 0;
    for (int64_t u = int64_t(blockIdx.x) * DC_WARPS + (threadIdx.x >> 5); u < g.n; u += warps) {
        const int64_t row = __ldg(g.rowptr + u);
        const int32_t d = int32_t(__ldg(g.rowptr + u + 1) - row);
        const int32_t lo = lower_bound_dev(g.col + row, d, int32_t(u));
        if (stats && lane == 0) stat += 16 + probe_bytes(d);
        for (int32_t j = lo + lane; j < d; j += 32) {
            const int32_t v = __ldg(g.col + row + j);
            const int64_t rv = __ldg(g.rowptr + v);
            const int32_t dv = int32_t(__ldg(g.rowptr + v + 1) - rv);
            const int32_t p = lower_bound_dev(g.col + rv, dv, int32_t(u));
            t[row + j] = t[rv + p];
            if (stats) stat += 4 + 16 + probe_bytes(dv) + 8;
        }
    }
    flush_stat(stats, stat, lane);
}

// Sums over vertices and edges (each undirected edge once, from its higher
// endpoint u towards x < u).
__global__ void __launch_bounds__(DC_WARPS * 32) ve_kernel(DevGraph g, const int32_t *__restrict__ t,
                                                          const uint32_t *__restrict__ k4e,
                                                          uint64_t *basis, Control *ctl,
                                                          unsigned long long *stats) {
    uint64_t stat = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * DC_WARPS;
    u128 p4e = 0, bull = 0, lolli_e = 0, de = 0, kite = 0, dart_e = 0, book = 0;
    u128 star3 = 0, star4 = 0, tx3 = 0, paw = 0, fork = 0, p5a = 0, tvd = 0, cricket = 0,
         lolli_v = 0, bowtie_v = 0, k5p3 = 0, k4deg3 = 0;
    for (int64_t u = int64_t(blockIdx.x) * DC_WARPS + (threadIdx.x >> 5); u < g.n; u += warps) {
        const int64_t row = __ldg(g.rowptr + u);
        const int64_t d = __ldg(g.rowptr + u + 1) - row;
        uint64_t st = 0, S = 0, S1 = 0, S2 = 0;
        if (stats) stat += lane == 0 ? 16 : 0;
        if (stats) stat += (d > lane ? uint64_t((d - 1 - lane) / 32 + 1) : 0) * (k4e ? 28 : 24);
        for (int64_t j = lane; j < d; j += 32) {
            const int32_t x = __ldg(g.col + row + j);
            const int64_t tx = __ldg(t + row + j);
            const int64_t dx = deg_of(g, x);
            st += uint64_t(tx);
            S += uint64_t(dx);
            S1 += uint64_t(dx - 1);
            S2 += uint64_t(dx - 1) * uint64_t(dx - 1);
            if (k4e && x > u) {
                // 4-cliques on the edge, kept at its slot in the lower endpoint's row
                const uint64_t q = __ldg(k4e + row + j);
                if (q) {
                    k5p3 += u128(q) * uint64_t(tx - 2);
                    k4deg3 += u128(q) * uint64_t(d + dx);
                }
            }
            if (x < u) {
                p4e += u128(uint64_t((d - 1) * (dx - 1)));
                if (tx > 0) {
                    bull += u128(uint64_t(tx)) * uint64_t((d - 2) * (dx - 2) - tx + 1);
                    lolli_e += u128(uint64_t(tx)) * uint64_t(d + dx + 2 * tx);
                    de += c2(tx);
                    kite += c2(tx) * uint64_t(d + dx - 6 > 0 ? d + dx - 6 : 0);
                    dart_e += u128(uint64_t(tx - 1)) * uint64_t(tx);
                    book += c3(tx);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st += __shfl_xor_sync(FULL, st, o);
            S += __shfl_xor_sync(FULL, S, o);
            S1 += __shfl_xor_sync(FULL, S1, o);
            S2 += __shfl_xor_sync(FULL, S2, o);
        }
        if (lane == 0) {
            const int64_t tu = int64_t(st / 2);
            star3 += c3(d);
            star4 += c4(d);
            tx3 += u128(uint64_t(tu));
            if (tu > 0) {
                paw += u128(uint64_t(tu)) * uint64_t(d - 2);
                tvd += u128(uint64_t(tu)) * uint64_t(d);
                cricket += u128(uint64_t(tu)) * c2(d - 2);
                lolli_v += u128(uint64_t(tu)) * uint64_t(int64_t(S) - d + 4);
                bowtie_v += c2(tu);
            }
            fork += c2(d - 1) * uint64_t(int64_t(S) - d) - u128(uint64_t(2 * tu)) * uint64_t(d >= 2 ? d - 2 : 0);
            p5a += (u128(S1) * S1 - S2) / 2;
        }
    }
    flush(basis, DB_P4E, p4e, lane);
    flush(basis, DB_BULL, bull, lane);
    flush(basis, DB_LOLLI_E, lolli_e, lane);
    flush(basis, DB_DE, de, lane);
    flush(basis, DB_KITE, kite, lane);
    flush(basis, DB_DART_E, dart_e, lane);
    flush(basis, DB_BOOK, book, lane);
    flush(basis, DB_STAR3, star3, lane);
    flush(basis, DB_STAR4, star4, lane);
    flush(basis, DB_TX3, tx3, lane);
    flush(basis, DB_PAW, paw, lane);
    flush(basis, DB_FORK, fork, lane);
    flush(basis, DB_P5A, p5a, lane);
    flush(basis, DB_TVD, tvd, lane);
    flush(basis, DB_CRICKET, cricket, lane);
    flush(basis, DB_LOLLI_V, lolli_v, lane);
    flush(basis, DB_BOWTIE_V, bowtie_v, lane);
    if (k4e) {
        flush(basis, DB_K5P3, k5p3, lane);
        flush(basis, DB_K4DEG3, k4deg3, lane);
    }
    flush_stat(stats, stat, lane);
    (void)ctl;
}

// Several lists per warp, one per lane (cnt_l entries each): prefix sums
// over the lanes, and for entry e of their concatenation the lane that
// holds it (last lane whose exclusive prefix is <= e).  Every lane calls
// both, so owner context can be fetched with shuffles.
__device__ __forceinline__ int32_t lanes_scan(int32_t cnt, int lane, int32_t &excl) {
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    excl = incl - cnt;
    return __shfl_sync(FULL, incl, 31);
}

__device__ __forceinline__ int lanes_owner(int32_t excl, int32_t e) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(FULL, excl, lo + step) <= e) lo += step;
    return lo;
}

// 2-path pass: one block per root a at a time (highest-ranked first, from a
// shared counter), with the block's counters W (n words, zero between roots)
// and its list of touched vertices in global memory.
//   walk 1: W[c] += 1 over the 2-paths a-b-c (b, c < a); the old values sum
//           to sum_c C(W[c], 2), the 4-cycles with highest vertex a;
//   walk 2: over the same 2-paths, (W[c] - 1) times the 4-cycle terms of the
//           banner (degrees) and the house (t of the edges a-b, b-c), and
//           per b the 5-cycle corrections |N(b) n [0, a)| W[b] and W[b];
//   touched vertices c: C(W[c], 3) and, for 5-cycles,
//           W[c] * sum_{x in N(c), x < c} W[x];
//   reset:  W[c] = 0 for the touched c.
__global__ void __launch_bounds__(P2_THREADS) paths2_kernel(DevGraph g, const int32_t *__restrict__ t,
                                                            uint32_t *Wall, int32_t *touched_all,
                                                            uint64_t *basis, Control *ctl,
                                                            int with_c5, unsigned long long *stats) {
    uint64_t stat = 0;
    __shared__ unsigned long long s_root;
    __shared__ int s_stop;
    __shared__ int s_nt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    uint32_t *W = Wall + size_t(blockIdx.x) * size_t(g.n);
    int32_t *touched = touched_all + size_t(blockIdx.x) * size_t(g.n);
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    u128 c4acc = 0, banner = 0, house = 0, qh = 0, k23 = 0, corr = 0, tm = 0;
    for (;;) {
        if (tid == 0) {
            s_root = atomicAdd(&ctl->work3, 1ull);
            int stop = *(volatile int *)&ctl->status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(&ctl->status, 1);
                stop = 1;
            }
            s_stop = stop;
            s_nt = 0;
        }
        __syncthreads();
        if (s_root >= (unsigned long long)g.n || s_stop) break;
        const int32_t a = int32_t(g.n - 1 - int64_t(s_root));
        const int64_t rowa = __ldg(g.rowptr + a);
        const int32_t da = int32_t(__ldg(g.rowptr + a + 1) - rowa);
        const int32_t la = lower_bound_dev(g.col + rowa, da, a);
        if (stats && tid == 0) stat += 16 + probe_bytes(da) + 4ull * uint64_t(la);
        // walk 1 (32 neighbours b per warp, one per lane, their rows below a
        // walked together)
        // neighbours per warp round: up to 32, fewer when the root has few
        const int per = min(32, max(1, (la + nwarps - 1) / nwarps));
        for (int i0 = warp * per; i0 < la; i0 += nwarps * per) {
            const int i = i0 + lane;
            int64_t rowb = 0;
            int32_t bl = 0;
            if (lane < per && i < la) {
                const int32_t b = __ldg(g.col + rowa + i);
                rowb = __ldg(g.rowptr + b);
                const int64_t db = __ldg(g.rowptr + b + 1) - rowb;
                bl = lower_bound_dev(g.col + rowb, int32_t(db), a);
                if (stats) stat += 2 * (16 + probe_bytes(db)) + uint64_t(bl) * (12 + 28);
            }
            auto bump = [&](int32_t c) {
                if (!PM_DCHECK(ctl, c >= 0 && c < g.n)) return;
                const uint32_t old = atomicAdd(W + c, 1u);
                c4acc += old;
                if (old == 0) {
                    const int q = atomicAdd(&s_nt, 1);
                    if (PM_DCHECK(ctl, q < g.n)) touched[q] = c;
                }
            };
            // long rows one at a time with all lanes, short ones together
            for (unsigned longs = __ballot_sync(FULL, bl > P2_LONG); longs; longs &= longs - 1) {
                const int l = __ffs(longs) - 1;
                const int64_t orow = __shfl_sync(FULL, rowb, l);
                const int32_t on = __shfl_sync(FULL, bl, l);
                for (int32_t j = lane; j < on; j += 32) bump(__ldg(g.col + orow + j));
            }
            int32_t excl;
            const int32_t total = lanes_scan(bl <= P2_LONG ? bl : 0, lane, excl);
            for (int32_t e0 = 0; e0 < total; e0 += 32) {
                const int32_t e = e0 + lane;
                const int o = lanes_owner(excl, e);
                const int64_t orow = __shfl_sync(FULL, rowb, o);
                const int32_t oex = __shfl_sync(FULL, excl, o);
                if (e < total) bump(__ldg(g.col + orow + (e - oex)));
            }
        }
        __syncthreads();
        // walk 2 (same grouping)
        for (int i0 = warp * per; i0 < la; i0 += nwarps * per) {
            const int i = i0 + lane;
            int64_t rowb = 0;
            int32_t bl = 0, db = 0, tab = 0;
            if (lane < per && i < la) {
                const int32_t b = __ldg(g.col + rowa + i);
                rowb = __ldg(g.rowptr + b);
                db = int32_t(__ldg(g.rowptr + b + 1) - rowb);
                bl = lower_bound_dev(g.col + rowb, db, a);
                tab = __ldg(t + rowa + i);
                const uint32_t wb = W[b];
                corr += u128(uint64_t(bl)) * wb;
                tm += wb;
            }
            auto visit = [&](int64_t slot, int32_t odb, int32_t otab) {
                const int32_t c = __ldg(g.col + slot);
                const uint32_t w = W[c];
                if (w > 1) {
                    const int64_t dc = deg_of(g, c);
                    banner += u128(w - 1) * uint64_t(2 * int64_t(odb) + da + dc - 8);
                    house += u128(w - 1) * uint64_t(int64_t(otab) + __ldg(t + slot));
                }
            };
            for (unsigned longs = __ballot_sync(FULL, bl > P2_LONG); longs; longs &= longs - 1) {
                const int l = __ffs(longs) - 1;
                const int64_t orow = __shfl_sync(FULL, rowb, l);
                const int32_t on = __shfl_sync(FULL, bl, l);
                const int32_t odb = __shfl_sync(FULL, db, l);
                const int32_t otab = __shfl_sync(FULL, tab, l);
                for (int32_t j = lane; j < on; j += 32) visit(orow + j, odb, otab);
            }
            int32_t excl;
            const int32_t total = lanes_scan(bl <= P2_LONG ? bl : 0, lane, excl);
            for (int32_t e0 = 0; e0 < total; e0 += 32) {
                const int32_t e = e0 + lane;
                const int o = lanes_owner(excl, e);
                const int64_t orow = __shfl_sync(FULL, rowb, o);
                const int32_t oex = __shfl_sync(FULL, excl, o);
                const int32_t odb = __shfl_sync(FULL, db, o);
                const int32_t otab = __shfl_sync(FULL, tab, o);
                if (e < total) visit(orow + (e - oex), odb, otab);
            }
        }
        // touched vertices (32 per warp; for 5-cycles their rows below them
        // walked together)
        const int nt = s_nt;
        const int per_t = min(32, max(1, (nt + nwarps - 1) / nwarps));
        for (int q0 = warp * per_t; q0 < nt; q0 += nwarps * per_t) {
            const int q = q0 + lane;
            int32_t c = 0, lc = 0;
            uint32_t w = 0;
            int64_t rowc = 0;
            if (lane < per_t && q < nt) {
                c = touched[q];
                w = W[c];
                k23 += c3(w);
                if (stats) stat += 8 + 4;       // touched entry, its counter, the reset
                if (with_c5) {
                    rowc = __ldg(g.rowptr + c);
                    const int64_t dcc = __ldg(g.rowptr + c + 1) - rowc;
                    lc = lower_bound_dev(g.col + rowc, int32_t(dcc), c);
                    if (stats) stat += 16 + probe_bytes(dcc) + 8ull * uint64_t(lc);
                }
            }
            if (!with_c5) continue;
            for (unsigned longs = __ballot_sync(FULL, lc > P2_LONG); longs; longs &= longs - 1) {
                const int l = __ffs(longs) - 1;
                const int64_t orow = __shfl_sync(FULL, rowc, l);
                const int32_t on = __shfl_sync(FULL, lc, l);
                const uint32_t ow = __shfl_sync(FULL, w, l);
                uint64_t sum = 0;
                for (int32_t j = lane; j < on; j += 32) sum += W[__ldg(g.col + orow + j)];
                qh += u128(ow) * sum;
            }
            int32_t excl;
            const int32_t total = lanes_scan(lc <= P2_LONG ? lc : 0, lane, excl);
            for (int32_t e0 = 0; e0 < total; e0 += 32) {
                const int32_t e = e0 + lane;
                const int o = lanes_owner(excl, e);
                const int64_t orow = __shfl_sync(FULL, rowc, o);
                const int32_t oex = __shfl_sync(FULL, excl, o);
                const uint32_t ow = __shfl_sync(FULL, w, o);
                if (e < total) qh += u128(ow) * W[__ldg(g.col + orow + (e - oex))];
            }
        }
        __syncthreads();
        for (int q = tid; q < nt; q += blockDim.x) W[touched[q]] = 0;
        __syncthreads();
    }
    flush(basis, DB_C4, c4acc, lane);
    flush(basis, DB_BANNER2, banner, lane);
    flush(basis, DB_HOUSE, house, lane);
    flush(basis, DB_C5Q, qh, lane);
    flush(basis, DB_C5CORR, corr, lane);
    flush(basis, DB_C5TM, tm, lane);
    flush(basis, DB_K23I, k23, lane);
    flush_stat(stats, stat, lane);
}

__device__ __forceinline__ u128 ld128(const uint64_t *basis, int i) {
    return u128(basis[2 * i]) | (u128(basis[2 * i + 1]) << 64);
}

// Each target's count from the sums: targets[2i] = formula, targets[2i+1] =
// output slot (128-bit counter index).
__global__ void combine_kernel(const uint64_t *basis, const int32_t *targets, int n_targets,
                               uint64_t *counters) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const u128 T = ld128(basis, DB_TRI);
    const u128 K4 = ld128(basis, DB_K4);
    const u128 DE = ld128(basis, DB_DE);
    const u128 C4 = ld128(basis, DB_C4);
    for (int i = 0; i < n_targets; i++) {
        u128 v = 0;
        switch (targets[2 * i]) {
            case DF_STAR3: v = ld128(basis, DB_STAR3); break;
            case DF_P4: v = ld128(basis, DB_P4E) - 3 * T; break;
            case DF_PAW: v = ld128(basis, DB_PAW); break;
            case DF_DIAMOND: v = DE; break;
            case DF_STAR4: v = ld128(basis, DB_STAR4); break;
            case DF_FORK: v = ld128(basis, DB_FORK); break;
            case DF_P5: v = ld128(basis, DB_P5A) - 4 * C4 - 2 * ld128(basis, DB_TVD) + 9 * T; break;
            case DF_CRICKET: v = ld128(basis, DB_CRICKET); break;
            case DF_BULL: v = ld128(basis, DB_BULL); break;
            case DF_LOLLIPOP: v = ld128(basis, DB_LOLLI_V) - ld128(basis, DB_LOLLI_E); break;
            case DF_BANNER: v = ld128(basis, DB_BANNER2) / 2 - 2 * DE; break;
            case DF_C5:
                v = ld128(basis, DB_C5Q) - ld128(basis, DB_C5CORR) + ld128(basis, DB_C5TM) / 2 -
                    ld128(basis, DB_C5TRI);
                break;
            case DF_KITE: v = ld128(basis, DB_KITE); break;
            case DF_DART: v = ld128(basis, DB_DART_TRI) - 2 * ld128(basis, DB_DART_E) - 12 * K4; break;
            case DF_BOWTIE: v = ld128(basis, DB_BOWTIE_V) - 2 * DE; break;
            case DF_HOUSE: v = ld128(basis, DB_HOUSE) - 4 * DE; break;
            case DF_BOOK: v = ld128(basis, DB_BOOK); break;
            case DF_GEM: v = ld128(basis, DB_GEM_TRI) - 12 * K4; break;
            case DF_K4PENDANT: v = ld128(basis, DB_K4DEG3) / 3 - 12 * K4; break;
            case DF_K4: v = K4; break;
            case DF_K5: v = ld128(basis, DB_K5); break;
            case DF_K5P3: v = ld128(basis, DB_K5P3); break;
            case DF_W4: v = ld128(basis, DB_W4); break;
            case DF_K23: v = ld128(basis, DB_K23); break;
            case DF_K23E: v = ld128(basis, DB_K23E); break;
            case DF_K5E: v = ld128(basis, DB_K5E); break;
            default: break;
        }
        const int slot = targets[2 * i + 1];
        counters[2 * slot] = uint64_t(v);
        counters[2 * slot + 1] = uint64_t(v >> 64);
    }
}

// Per-pattern deadlines: if the decomposition group's deadline expired,
// every one of its patterns is flagged; then the status and counters are
// reset as between two patterns.
__global__ void flag_targets_kernel(Control *ctl, uint8_t *timed_out, const int32_t *targets,
                                    int n_targets) {
    if (ctl->status == 1)
        for (int i = 0; i < n_targets; i++) timed_out[targets[2 * i + 1]] = 1;
    ctl->status = 0;
    ctl->work = 0;
    ctl->work2 = 0;
    ctl->work3 = 0;
    ctl->n_deferred = 0;
    ctl->n_pieces = 0;
    ctl->deadline = ctl->call_deadline;
}

int launch_flag_targets(Control *ctl, uint8_t *timed_out, const int32_t *targets, int n_targets,
                        void *stream) {
    flag_targets_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, timed_out, targets, n_targets);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int decomp_path_blocks(int device) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, paths2_kernel, P2_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

static int dc_blocks(int device, const void *kern) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DC_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

int launch_decomp(const DecompLaunch &L, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(L.basis, 0, sizeof(uint64_t) * 2 * DB_COUNT, s);
    TriArgs A{L.g, L.tasks, L.t, L.basis, L.ctl, L.stats, (L.passes & DP_C5) ? 1 : 0};
    cudaMemsetAsync(L.t, 0, sizeof(int32_t) * size_t(L.g.nnz), s);
    cudaMemsetAsync(&L.ctl->work3, 0, sizeof(unsigned long long), s);
    tri_kernel<0><<<dc_blocks(device, (const void *)tri_kernel<0>), DC_WARPS * 32, 0, s>>>(A);
    mirror_kernel<<<dc_blocks(device, (const void *)mirror_kernel), DC_WARPS * 32, 0, s>>>(L.g, L.t,
                                                                                      L.stats);
    if (L.passes & DP_WHEEL) {
        WheelArgs w = L.wheel;
        w.g = L.g;
        w.t = L.t;
        w.basis = L.basis;
        w.ctl = L.ctl;
        w.stats = L.stats;
        if (launch_wheel(w, L.passes, s)) return -1;
    }
    if (L.passes & DP_LOCAL) {
        if (L.k4e) cudaMemsetAsync(L.k4e, 0, sizeof(uint32_t) * size_t(L.g.nnz), s);
        cudaMemsetAsync(&L.ctl->work3, 0, sizeof(unsigned long long), s);
        LocalArgs la = L.local;
        la.k4e = (L.passes & DP_K4E) ? L.k4e : nullptr;
        la.want_k5 = (L.passes & DP_K5) ? 1 : 0;
        la.stats = L.stats;
        if (launch_local(la, L.local_blocks, s)) return -1;
    }
    ve_kernel<<<dc_blocks(device, (const void *)ve_kernel), DC_WARPS * 32, 0, s>>>(
        L.g, L.t, (L.passes & DP_K4E) ? L.k4e : nullptr, L.basis, L.ctl, L.stats);
    if (L.passes & DP_TRI2) {
        cudaMemsetAsync(&L.ctl->work3, 0, sizeof(unsigned long long), s);
        tri_kernel<1><<<dc_blocks(device, (const void *)tri_kernel<1>), DC_WARPS * 32, 0, s>>>(A);
    }
    if (L.passes & DP_PATHS) {
        cudaMemsetAsync(&L.ctl->work3, 0, sizeof(unsigned long long), s);
        paths2_kernel<<<L.path_blocks, P2_THREADS, 0, s>>>(L.g, L.t, L.W, L.touched, L.basis, L.ctl,
                                                           (L.passes & DP_C5) ? 1 : 0, L.stats);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("decomposition kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

int launch_decomp_triangles(const DecompLaunch &L, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    cudaStream_t s = (cudaStream_t)stream;
    TriArgs A{L.g, L.tasks, L.t, L.basis, L.ctl, nullptr, 0};
    cudaMemsetAsync(L.t, 0, sizeof(int32_t) * size_t(L.g.nnz), s);
    cudaMemsetAsync(&L.ctl->work3, 0, sizeof(unsigned long long), s);
    tri_kernel<0><<<dc_blocks(device, (const void *)tri_kernel<0>), DC_WARPS * 32, 0, s>>>(A);
    mirror_kernel<<<dc_blocks(device, (const void *)mirror_kernel), DC_WARPS * 32, 0, s>>>(L.g, L.t,
                                                                                      nullptr);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("triangle pass launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

int launch_decomp_combine(const uint64_t *basis, const int32_t *targets, int n_targets,
                          uint64_t *counters, void *stream) {
    combine_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(basis, targets, n_targets, counters);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("decomposition combine launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

}  // namespace pm
