// Neighbourhood-graph pass (sm_103a): per-edge common-neighbour lists and
// the edge-induced counts of the 5-vertex patterns that need them.
//
// Common-neighbour lists: for every CSR slot s = (v, u) the list T_s holds,
// sorted, the positions in v's row of the vertices adjacent to both v and u.
// Read as the adjacency of u in the graph G_v induced on N(v), the lists of
// v's slots are G_v in v's own coordinates (positions 0..d_v-1), so counters
// over G_v's vertices are dense arrays indexed by position.  Their lengths
// are the per-edge triangle counts t_s (triangle pass), their offsets the
// exclusive scan of t; a list is filled by walking the shorter of the two
// rows and locating its members in the longer one (adjacency bitmap with a
// popcount rank index for hubs, binary search otherwise).
//
// 4-wheel (a centre joined to every vertex of a 4-cycle, 8 edges): every
// edge-induced copy has one centre c (the only vertex of degree 4 in it) and
// its rim is a 4-cycle of G_c.  With a the highest-ranked rim vertex and b
// the rim vertex opposite a, the copy is fixed by (c, a, b) and the pair of
// rim vertices x, y < a adjacent to a, b and c, so
//     W4 = sum_c sum_{a in N(c)} sum_{b in N(c), b < a} C(cnt_{c,a}[b], 2),
//     cnt_{c,a}[b] = #{x in N(c) n N(a) n N(b) : x < a},
// one task per slot (c, a) with its counters over the positions of N(c)
// below a's: for each x in T_(c,a) below a, +1 at every position of T_(c,x)
// below a.
//
// K2,3 and K2,3 plus an edge inside its 3-side (7 edges): with c_ab the
// number of common neighbours of a and b and e_ab the number of edges among
// them, every edge-induced K2,3 is a pair a > b with three of their common
// neighbours, and every K2,3+e a pair a > b (its two vertices of degree 3
// that are not adjacent in the pattern), an edge xy among their common
// neighbours and a third common neighbour z, so
//     K2,3 = sum_{a > b} C(c_ab, 3),   K2,3+e = sum_{a > b} e_ab (c_ab - 2).
// Per root a: walk A adds 1 to W[b] over the 2-paths a-w-b, b < a (any w);
// walk B adds 1 to E[b] over the "diamonds" with tips a > b, each edge xy of
// G_a once (x < y) and b in T_(x,y) below a, read in x's coordinates through
// the mirror position of a in x's row.
//
// K5 minus an edge (9 edges): every edge-induced copy is a triangle
// (x, y, z) plus two of its common neighbours, so with k_xyz the number of
// vertices adjacent to all three, K5-e = sum over triangles of C(k_xyz, 2).
// Each triangle is taken from its lowest-ranked vertex x and edge y < z of
// G_x above x: per slot (x, y), y > x, +1 at z for every w in T_(x,y) and
// z in T_(x,w) above y, then k_xyz is the count at each z of T_(x,y) above
// y.  The counters cover x's positions above y only (fewer than x's
// neighbours ranked above x, a few hundred on R-MAT graphs).
#include <algorithm>
#include <type_traits>

#include "devgraph.cuh"
#include "internal.hpp"

namespace pm {

constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 8;                        // scan items per thread
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;
constexpr int TL_WARPS = 8;                        // warps per block of the list builder
constexpr int W4_THREADS = 1024;
constexpr int W4_WARPS = W4_THREADS / 32;
constexpr int W4_WARP_CAP = 2048;                  // counter positions of a warp task
constexpr int W4_SMEM_WORDS = 32768;               // 128 KB: 65536 16-bit block counters
constexpr int64_t W4_BLOCK_CAP = 2 * int64_t(W4_SMEM_WORDS);
constexpr int K23_THREADS = 512;                   // two blocks (roots) per SM
constexpr int K5E_THREADS = 512;
constexpr int K5E_WARP_WORDS = 1024;               // 2048 16-bit counters per warp (64 KB per block)
constexpr int K23_WARP_CAP = 2048;                 // walk-B window of a warp item (positions)
constexpr int K23_SMEM_WORDS = 16384;              // 64 KB: 16 warps x 1024 words, or one block window

__device__ __forceinline__ u128 w_c2(uint64_t x) { return x >= 2 ? u128(x) * (x - 1) / 2 : 0; }

// Algorithmic bytes of a binary search over len elements (instrumented runs).
__device__ __forceinline__ uint64_t w_probe_bytes(int64_t len) {
    return 4ull * uint64_t(len > 1 ? 65 - __clzll(uint64_t(len)) : 1);
}

__device__ __forceinline__ void w_flush(uint64_t *basis, int idx, u128 v, int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(v), o);
        const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(v >> 64), o);
        v += (u128(hi) << 64) | lo;
    }
    if (lane == 0 && v != 0) add_u128(basis + 2 * idx, v);
}

__device__ __forceinline__ void w_flush_stat(unsigned long long *stats, uint64_t v, int lane) {
    if (!stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(stats, (unsigned long long)v);
}

// Deadline / stop check by one thread; returns non-zero to stop.
__device__ __forceinline__ int w_should_stop(Control *ctl, uint64_t deadline) {
    int stop = *(volatile int *)&ctl->status;
    if (!stop && deadline && global_ns() > deadline) {
        atomicExch(&ctl->status, 1);
        stop = 1;
    }
    return stop;
}

// Row of CSR slot s: the last v with rowptr[v] <= s, searched in [lo, hi).
__device__ __forceinline__ int32_t row_of_slot(const int64_t *rowptr, int64_t s, int64_t lo, int64_t hi) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(rowptr + mid) <= s) lo = mid;
        else hi = mid;
    }
    return int32_t(lo);
}

// Warp walk over up to 32 sorted lists at once, lane l holding
// T[base_l .. base_l + len_l), calling f(value) for each entry (with CUT,
// only for the entries below `bound`, the same for all lanes).  Lists
// longer than WL_LONG are walked one at a time by the whole warp (lanes
// stride over the entries, with CUT stopping at the first entry >= bound);
// the short ones (the common case: the common neighbours of a hub and a
// low-degree vertex) are cut by a binary search and then walked together,
// entry e of their concatenation going to lane e mod 32 (its list found by
// a binary search over the lanes' exclusive prefix sums), so short lists
// leave no lane idle and many loads are in flight at once.
constexpr int32_t WL_LONG = 64;

template <bool CUT, class F>
__device__ __forceinline__ void warp_lists(const int32_t *__restrict__ T, int64_t base, int32_t len,
                                           int32_t bound, int lane, Control *ctl, int64_t limit, F f) {
    unsigned longs = __ballot_sync(FULL, len > WL_LONG);
    while (longs) {
        const int l = __ffs(longs) - 1;
        longs &= longs - 1;
        const int64_t ob = __shfl_sync(FULL, base, l);
        const int32_t on = __shfl_sync(FULL, len, l);
        for (int32_t j = lane; j < on; j += 32) {
            if (!PM_DCHECK(ctl, ob + j < limit)) break;
            const int32_t v = __ldg(T + ob + j);
            if (CUT && v >= bound) break;
            f(v);
        }
    }
    int32_t cnt = 0;
    if (len > 0 && len <= WL_LONG) cnt = CUT ? lower_bound_dev(T + base, len, bound) : len;
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int32_t excl = incl - cnt;
    const int32_t total = __shfl_sync(FULL, incl, 31);
    for (int32_t e0 = 0; e0 < total; e0 += 32) {
        const int32_t e = e0 + lane;
        int lo = 0;                                  // last lane whose list starts at or before e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int32_t ex = __shfl_sync(FULL, excl, lo + step);
            if (ex <= e) lo += step;
        }
        const int64_t ob = __shfl_sync(FULL, base, lo);
        const int32_t oex = __shfl_sync(FULL, excl, lo);
        if (e < total && PM_DCHECK(ctl, ob + (e - oex) < limit)) f(__ldg(T + ob + (e - oex)));
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-slot triangle counts into list offsets.

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *s_warp, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < int(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;    // inclusive over warps
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const int64_t before = warp ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SC_THREADS) tsum_kernel(const int32_t *__restrict__ t, int64_t nnz,
                                                          int64_t *bsum) {
    __shared__ int64_t s_warp[32];
    const int64_t base = int64_t(blockIdx.x) * SC_TILE + int64_t(threadIdx.x) * SC_ITEMS;
    int64_t v = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++)
        if (base + i < nnz) v += __ldg(t + base + i);
    int64_t total;
    block_exclusive_scan(v, s_warp, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS) tscan_top_kernel(int64_t *bsum, int64_t nb) {
    __shared__ int64_t s_warp[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SC_THREADS) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, s_warp, total);
        if (i < nb) bsum[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SC_THREADS) tscan_kernel(const int32_t *__restrict__ t, int64_t nnz,
                                                           const int64_t *__restrict__ bsum,
                                                           int64_t *toff) {
    __shared__ int64_t s_warp[32];
    const int64_t base = int64_t(blockIdx.x) * SC_TILE + int64_t(threadIdx.x) * SC_ITEMS;
    int32_t x[SC_ITEMS];
    int64_t v = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        x[i] = base + i < nnz ? __ldg(t + base + i) : 0;
        v += x[i];
    }
    int64_t total;
    int64_t run = bsum[blockIdx.x] + block_exclusive_scan(v, s_warp, total);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        if (base + i < nnz) toff[base + i] = run;
        run += x[i];
        if (base + i == nnz - 1) toff[nnz] = run;
    }
}

// Popcount rank index of the hub bitmaps: rank[h][w] = set bits of hub h's
// bitmap in words 0..w-1 (one block per hub).
__global__ void __launch_bounds__(SC_THREADS) hub_rank_kernel(const uint32_t *__restrict__ bits,
                                                              int64_t words, int32_t *rank) {
    __shared__ int64_t s_warp[32];
    const uint32_t *b = bits + size_t(blockIdx.x) * size_t(words);
    int32_t *r = rank + size_t(blockIdx.x) * size_t(words);
    int64_t carry = 0;
    for (int64_t w0 = 0; w0 < words; w0 += SC_THREADS) {
        const int64_t i = w0 + threadIdx.x;
        const int64_t v = i < words ? __popc(__ldg(b + i)) : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, s_warp, total);
        if (i < words) r[i] = int32_t(carry + ex);
        carry += total;
    }
}

// ---------------------------------------------------------------------------
// Common-neighbour lists, one warp per slot, 32 consecutive slots per chunk.
__global__ void __launch_bounds__(TL_WARPS * 32) tlist_kernel(WheelArgs A) {
    const int lane = threadIdx.x & 31;
    const DevGraph &g = A.g;
    const int64_t nnz = g.nnz;
    const unsigned long long n_chunks = (unsigned long long)((nnz + 31) / 32);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t stat = 0;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&A.ctl->work3, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if (c >= n_chunks) break;
        const int64_t base = int64_t(c) * 32;
        int32_t vrow = 0;
        if (base + lane < nnz) vrow = row_of_slot(g.rowptr, base + lane, 0, g.n);
        for (int q = 0; q < 32; q++) {
            const int64_t s = base + q;
            if (s >= nnz) break;
            const int32_t ts = __ldg(A.t + s);
            const int32_t v = __shfl_sync(FULL, vrow, q);
            if (ts == 0) continue;
            const int32_t u = __ldg(g.col + s);
            const int64_t rowv = __ldg(g.rowptr + v), rowu = __ldg(g.rowptr + u);
            const int32_t dv = int32_t(__ldg(g.rowptr + v + 1) - rowv);
            const int32_t du = int32_t(__ldg(g.rowptr + u + 1) - rowu);
            int32_t *out = A.T + __ldg(A.toff + s);
            int32_t written = 0;
            if (du <= dv) {
                // members of N(u), located in v's row
                const int32_t hv = g.hub ? __ldg(g.hub + v) : -1;
                for (int32_t j0 = 0; j0 < du && written < ts; j0 += 32) {
                    const int32_t j = j0 + lane;
                    bool found = false;
                    int32_t pos = 0;
                    if (j < du) {
                        const int32_t w = __ldg(g.col + rowu + j);
                        if (hv >= 0) {
                            const size_t wi = size_t(hv) * size_t(g.words) + size_t(w >> 5);
                            const uint32_t word = __ldg(g.bits + wi);
                            found = (word >> (w & 31)) & 1u;
                            pos = __ldg(A.hub_rank + wi) + __popc(word & ((1u << (w & 31)) - 1u));
                        } else {
                            pos = lower_bound_dev(g.col + rowv, dv, w);
                            found = pos < dv && __ldg(g.col + rowv + pos) == w;
                        }
                    }
                    const unsigned m = __ballot_sync(FULL, found);
                    const int32_t k = written + __popc(m & lt);
                    if (found && k < ts && PM_DCHECK(A.ctl, out + k < A.T + A.T_len)) out[k] = pos;
                    written += __popc(m);
                    if (A.stats) stat += (j < du ? 4 : 0) + (j < du ? (hv >= 0 ? 8 : w_probe_bytes(dv)) : 0);
                }
            } else {
                // members of N(v) (by position), tested against N(u)
                for (int32_t p0 = 0; p0 < dv && written < ts; p0 += 32) {
                    const int32_t p = p0 + lane;
                    const bool found = p < dv && contains(g, u, __ldg(g.col + rowv + p));
                    const unsigned m = __ballot_sync(FULL, found);
                    const int32_t k = written + __popc(m & lt);
                    if (found && k < ts && PM_DCHECK(A.ctl, out + k < A.T + A.T_len)) out[k] = p;
                    written += __popc(m);
                    if (A.stats && p < dv) stat += 4 + (g.hub && __ldg(g.hub + u) >= 0 ? 4 : w_probe_bytes(du));
                }
            }
            if (A.stats && lane == 0) stat += 32 + 8 + 4ull * uint64_t(ts);
            if (lane == 0 && written != ts) atomicExch(&A.ctl->fault, 1);   // lists disagree with t
        }
    }
    w_flush_stat(A.stats, stat, lane);
}

// ---------------------------------------------------------------------------
// 4-wheels.  Block tasks: slots (c, a) whose position p_a in c's row is at
// least W4_WARP_CAP, with 16-bit counters for positions below p_a packed two
// to a shared-memory word (a count never exceeds p_a - 1 <= 65535), or 32-bit
// counters in a per-block global area above W4_BLOCK_CAP.  Warp tasks: the
// first W4_WARP_CAP slots of every row, one row per warp, with the warp's own
// 2048 16-bit counters.

template <bool SMEM>
__device__ __forceinline__ void w4_bump(uint32_t *cnt, int32_t pb) {
    if (SMEM) atomicAdd(cnt + (pb >> 1), (pb & 1) ? 65536u : 1u);
    else atomicAdd(cnt + pb, 1u);
}

// Walk of one block task: warps over the x below p_a, lanes over T_(c,x).
template <bool SMEM>
__device__ __forceinline__ uint64_t w4_block_walk(const WheelArgs &A, uint32_t *cnt, int64_t rowc,
                                                  const int32_t *X, int32_t nx, int32_t pa,
                                                  int warp, int lane) {
    uint64_t stat = 0;
    for (int32_t k = warp; k < nx; k += W4_WARPS) {
        const int64_t sx = rowc + __ldg(X + k);
        const int64_t b0 = __ldg(A.toff + sx);
        const int32_t len = int32_t(__ldg(A.toff + sx + 1) - b0);
        const int32_t *B = A.T + b0;
        for (int32_t j = lane; j < len; j += 32) {
            const int32_t pb = __ldg(B + j);
            if (A.stats) stat += 4;
            if (pb >= pa) break;
            if (PM_DCHECK(A.ctl, SMEM ? (pb >> 1) < W4_SMEM_WORDS : pb < A.gcnt_words)) w4_bump<SMEM>(cnt, pb);
        }
        if (A.stats && lane == 0) stat += 16;
    }
    return stat;
}

__global__ void __launch_bounds__(W4_THREADS, 1) w4_kernel(WheelArgs A) {
    extern __shared__ uint32_t sc[];
    __shared__ unsigned long long s_task;
    __shared__ int s_stop;
    __shared__ int32_t s_rows[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevGraph &g = A.g;
    Control *ctl = A.ctl;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    u128 acc = 0;
    uint64_t stat = 0;
    for (int i = tid; i < W4_SMEM_WORDS; i += W4_THREADS) sc[i] = 0;
    // first row of degree > W4_WARP_CAP (degrees do not decrease with the id)
    int64_t lo = 0, hi = g.n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(g.rowptr + mid + 1) - __ldg(g.rowptr + mid) > W4_WARP_CAP) hi = mid;
        else lo = mid + 1;
    }
    const int64_t h0 = lo;
    const int64_t base = __ldg(g.rowptr + h0);
    const int64_t nbig = g.nnz - base;
    uint32_t *gcnt = A.gcnt ? A.gcnt + size_t(blockIdx.x) * size_t(A.gcnt_words) : nullptr;
    __syncthreads();
    // block tasks, largest rows first, 32 slots per chunk
    const unsigned long long n_big_chunks = (unsigned long long)((nbig + 31) / 32);
    for (;;) {
        __syncthreads();   // the previous chunk's shared values are no longer read
        if (tid == 0) {
            s_task = atomicAdd(&ctl->work3, 1ull);
            s_stop = w_should_stop(ctl, deadline);
        }
        __syncthreads();
        const unsigned long long chunk = s_task;
        if (chunk >= n_big_chunks || s_stop) break;
        if (tid < 32) {
            const int64_t e = int64_t(chunk) * 32 + tid;
            s_rows[tid] = e < nbig ? row_of_slot(g.rowptr, g.nnz - 1 - e, h0, g.n) : -1;
        }
        __syncthreads();
        for (int q = 0; q < 32; q++) {
            const int32_t c = s_rows[q];
            if (c < 0) break;
            const int64_t s = g.nnz - 1 - (int64_t(chunk) * 32 + q);
            const int64_t rowc = __ldg(g.rowptr + c);
            const int32_t pa = int32_t(s - rowc);
            const int32_t ts = __ldg(A.t + s);
            if (pa < W4_WARP_CAP || ts < 2) continue;     // uniform; warp tasks take p_a < cap
            const int32_t *X = A.T + __ldg(A.toff + s);
            const int32_t nx = lower_bound_dev(X, ts, pa);
            if (nx < 2) continue;
            const bool smem = pa <= W4_BLOCK_CAP;
            if (smem) stat += w4_block_walk<true>(A, sc, rowc, X, nx, pa, warp, lane);
            else if (gcnt) stat += w4_block_walk<false>(A, gcnt, rowc, X, nx, pa, warp, lane);
            __syncthreads();
            if (smem) {
                for (int32_t w = tid; w < (pa + 1) / 2; w += W4_THREADS) {
                    const uint32_t v = sc[w];
                    if (v) {
                        acc += w_c2(v & 0xffffu) + w_c2(v >> 16);
                        sc[w] = 0;
                    }
                }
            } else if (gcnt) {
                for (int32_t w = tid; w < pa; w += W4_THREADS) {
                    const uint32_t v = gcnt[w];
                    if (v) {
                        acc += w_c2(v);
                        gcnt[w] = 0;
                    }
                }
            }
            if (A.stats && tid == 0) stat += 16 + w_probe_bytes(ts);
            __syncthreads();
        }
    }
    __syncthreads();
    // warp tasks: rows from the highest down, positions below W4_WARP_CAP
    uint32_t *wc = sc + warp * (W4_WARP_CAP / 2);
    for (int i = lane; i < W4_WARP_CAP / 2; i += 32) wc[i] = 0;
    __syncwarp();
    for (;;) {
        unsigned long long r = 0;
        int stop = 0;
        if (lane == 0) {
            r = atomicAdd(&ctl->work2, 1ull);
            stop = w_should_stop(ctl, deadline);
        }
        r = __shfl_sync(FULL, r, 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (r >= (unsigned long long)g.n || stop) break;
        const int32_t c = int32_t(g.n - 1 - int64_t(r));
        const int64_t rowc = __ldg(g.rowptr + c);
        const int32_t dc = int32_t(__ldg(g.rowptr + c + 1) - rowc);
        const int32_t np = dc < W4_WARP_CAP ? dc : W4_WARP_CAP;
        for (int32_t pa = 2; pa < np; pa++) {
            const int64_t s = rowc + pa;
            const int32_t ts = __ldg(A.t + s);
            if (ts < 2) continue;
            const int32_t *X = A.T + __ldg(A.toff + s);
            int32_t nx = 0;     // entries of X below pa
            for (int32_t k0 = 0; k0 < ts; k0 += 32) {
                const int32_t k = k0 + lane;
                const bool below = k < ts && __ldg(X + k) < pa;
                const unsigned m = __ballot_sync(FULL, below);
                nx += __popc(m);
                if (m != FULL) break;
            }
            if (nx < 2) continue;
            for (int32_t k = 0; k < nx; k++) {
                const int64_t sx = rowc + __ldg(X + k);
                const int64_t b0 = __ldg(A.toff + sx);
                const int32_t len = int32_t(__ldg(A.toff + sx + 1) - b0);
                const int32_t *B = A.T + b0;
                for (int32_t j = lane; j < len; j += 32) {
                    const int32_t pb = __ldg(B + j);
                    if (pb >= pa) break;
                    if (PM_DCHECK(ctl, (pb >> 1) < W4_WARP_CAP / 2)) atomicAdd(wc + (pb >> 1), (pb & 1) ? 65536u : 1u);
                }
                if (A.stats && lane == 0) stat += 16 + 4ull * uint64_t(len);
            }
            __syncwarp();
            for (int32_t w = lane; w < (pa + 1) / 2; w += 32) {
                const uint32_t v = wc[w];
                if (v) {
                    acc += w_c2(v & 0xffffu) + w_c2(v >> 16);
                    wc[w] = 0;
                }
            }
            __syncwarp();
            if (A.stats && lane == 0) stat += 16 + 4ull * uint64_t(nx);
        }
    }
    w_flush(A.basis, DB_W4, acc, lane);
    w_flush_stat(A.stats, stat, lane);
}

// Mirror positions: mpos[s] = position of v in u's row, for slot s = (v, u).
__global__ void __launch_bounds__(TL_WARPS * 32) mpos_kernel(WheelArgs A) {
    const int lane = threadIdx.x & 31;
    const DevGraph &g = A.g;
    const int64_t warps = int64_t(gridDim.x) * TL_WARPS;
    uint64_t stat = 0;
    for (int64_t v = int64_t(blockIdx.x) * TL_WARPS + (threadIdx.x >> 5); v < g.n; v += warps) {
        const int64_t row = __ldg(g.rowptr + v);
        const int32_t d = int32_t(__ldg(g.rowptr + v + 1) - row);
        for (int32_t j = lane; j < d; j += 32) {
            const int32_t u = __ldg(g.col + row + j);
            const int32_t hu = (g.hub && A.hub_rank) ? __ldg(g.hub + u) : -1;
            int32_t pos;
            if (hu >= 0) {
                const size_t wi = size_t(hu) * size_t(g.words) + size_t(v >> 5);
                pos = __ldg(A.hub_rank + wi) + __popc(__ldg(g.bits + wi) & ((1u << (v & 31)) - 1u));
                if (A.stats) stat += 4 + 4 + 8 + 4;
            } else {
                const int64_t ru = __ldg(g.rowptr + u);
                const int32_t du = int32_t(__ldg(g.rowptr + u + 1) - ru);
                pos = lower_bound_dev(g.col + ru, du, int32_t(v));
                if (A.stats) stat += 4 + 16 + w_probe_bytes(du) + 4;
            }
            A.mpos[row + j] = pos;
        }
    }
    w_flush_stat(A.stats, stat, lane);
}

__device__ __forceinline__ u128 w_c3(uint64_t x) { return x >= 3 ? u128(x) * (x - 1) * (x - 2) / 6 : 0; }

// Walk B of one neighbour x of root a (a at position mx of x's row): for
// each y > x in T_(x,a), +1 at the positions of T_(x,y) below mx.  With
// CNT != nullptr the counts go to 16-bit counters over x's positions
// (packed two to a word; a count never exceeds |T_(x,a)| <= 65535 here) and
// are added to E once per position afterwards; otherwise straight to E.
template <int STRIDE, class ET>
__device__ __forceinline__ uint64_t k23_walk_b(const WheelArgs &A, ET *E, uint32_t *cnt,
                                               int64_t rowx, const int32_t *Y, int32_t k0, int32_t ny,
                                               int32_t mx, int first, int lane) {
    uint64_t stat = 0;
    for (int32_t k = k0 + first; k < ny; k += STRIDE) {
        const int64_t sy = rowx + __ldg(Y + k);
        const int64_t b0 = __ldg(A.toff + sy);
        const int32_t nb = int32_t(__ldg(A.toff + sy + 1) - b0);
        for (int32_t j = lane; j < nb; j += 32) {
            const int32_t pb = __ldg(A.T + b0 + j);
            if (A.stats) stat += 4;
            if (pb >= mx) break;
            if (cnt) {
                if (PM_DCHECK(A.ctl, (pb >> 1) < K23_SMEM_WORDS)) atomicAdd(cnt + (pb >> 1), (pb & 1) ? 65536u : 1u);
            } else {
                const int32_t b = __ldg(A.g.col + rowx + pb);
                if (PM_DCHECK(A.ctl, b >= 0 && b < A.g.n)) atomicAdd(E + b, ET(1));
            }
        }
        if (A.stats && lane == 0) stat += 4 + 16;
    }
    return stat;
}

// Adds the packed 16-bit counts of positions [0, mx) of x's row to E and
// clears them (threads `first`, `first` + STRIDE, ...).
template <int STRIDE, class ET>
__device__ __forceinline__ uint64_t k23_flush(const WheelArgs &A, ET *E, uint32_t *cnt,
                                              int64_t rowx, int32_t mx, int first) {
    uint64_t stat = 0;
    for (int32_t w = first; w < (mx + 1) / 2; w += STRIDE) {
        const uint32_t v = cnt[w];
        if (!v) continue;
        if (v & 0xffffu) atomicAdd(E + __ldg(A.g.col + rowx + 2 * w), ET(v & 0xffffu));
        if (v >> 16) atomicAdd(E + __ldg(A.g.col + rowx + 2 * w + 1), ET(v >> 16));
        cnt[w] = 0;
        if (A.stats) stat += 4 * (((v & 0xffffu) != 0) + ((v >> 16) != 0)) + 8;
    }
    return stat;
}

// K2,3 and K2,3+e, one block per root (highest-ranked first), with the
// block's counters W (32-bit), E (64-bit) and touched list in global memory.
// Walk A: warps take neighbours w of the root from a shared counter.  Walk
// B: a warp takes each neighbour x whose window (a's position in x's row)
// fits its own 2048 16-bit counters; the whole block then takes the others
// one at a time with 32768 counters in shared memory (rows above that, or
// lists longer than 65535, add to E directly).  Two blocks share an SM, so
// 2 x SMs roots are in flight (most roots have few neighbours).
template <bool NARROW>
__global__ void __launch_bounds__(K23_THREADS, 2) k23_kernel(WheelArgs A) {
    // NARROW (largest degree below 65536): 16-bit 2-path and 32-bit diamond
    // counters (a root's c_ab <= 65535 and e_ab <= C(65535, 2) < 2^32), half
    // the scattered counter bytes of the 32/64-bit layout
    using ET = typename std::conditional<NARROW, unsigned int, unsigned long long>::type;
    extern __shared__ uint32_t sc[];
    __shared__ unsigned long long s_root;
    __shared__ int s_stop;
    __shared__ int s_nt;
    __shared__ int s_next[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevGraph &g = A.g;
    Control *ctl = A.ctl;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    uint32_t *W = A.kW + size_t(blockIdx.x) * size_t(g.n);          // NARROW: 16-bit halves
    uint16_t *W16 = reinterpret_cast<uint16_t *>(W);
    ET *E = reinterpret_cast<ET *>(A.kE + size_t(blockIdx.x) * size_t(g.n));
    int32_t *touched = A.ktouched + size_t(blockIdx.x) * size_t(g.n);
    uint32_t *wc = sc + warp * (K23_WARP_CAP / 2);
    u128 k23 = 0, k23e = 0;
    uint64_t stat = 0;
    for (int i = tid; i < K23_SMEM_WORDS; i += K23_THREADS) sc[i] = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_root = atomicAdd(&ctl->work3, 1ull);
            s_stop = w_should_stop(ctl, deadline);
            s_nt = 0;
            s_next[0] = 0;
            s_next[1] = 0;
        }
        __syncthreads();
        if (s_root >= (unsigned long long)g.n || s_stop) break;
        const int32_t a = int32_t(g.n - 1 - int64_t(s_root));
        const int64_t rowa = __ldg(g.rowptr + a);
        const int32_t da = int32_t(__ldg(g.rowptr + a + 1) - rowa);
        // walk A: 2-paths a-w-b, b < a (the entries of w's row before a)
        for (;;) {
            int32_t i = 0;
            if (lane == 0) i = atomicAdd(&s_next[0], 1);
            i = __shfl_sync(FULL, i, 0);
            if (i >= da) break;
            const int32_t w = __ldg(g.col + rowa + i);
            const int32_t m = __ldg(A.mpos + rowa + i);
            const int64_t roww = __ldg(g.rowptr + w);
            for (int32_t j = lane; j < m; j += 32) {
                const int32_t b = __ldg(g.col + roww + j);
                if (!PM_DCHECK(ctl, b >= 0 && b < g.n)) break;
                uint32_t old;
                if (NARROW) {
                    const int sh = 16 * (b & 1);
                    old = (atomicAdd(W + (b >> 1), 1u << sh) >> sh) & 0xffffu;
                } else {
                    old = atomicAdd(W + b, 1u);
                }
                if (old == 0) {
                    const int q = atomicAdd(&s_nt, 1);
                    if (PM_DCHECK(ctl, q < g.n)) touched[q] = b;
                }
            }
            if (A.stats && lane == 0) stat += 4 + 4 + 16 + 16ull * uint64_t(m);
        }
        // walk B, warp items: edges x < y of G_a, tips b < a in T_(x,y)
        for (;;) {
            int32_t i = 0;
            if (lane == 0) i = atomicAdd(&s_next[1], 1);
            i = __shfl_sync(FULL, i, 0);
            if (i >= da) break;
            const int32_t mx = __ldg(A.mpos + rowa + i);          // a's position in x's row
            if (mx > K23_WARP_CAP) continue;                       // block item
            const int32_t x = __ldg(g.col + rowa + i);
            const int64_t rowx = __ldg(g.rowptr + x);
            const int64_t y0 = __ldg(A.toff + rowx + mx);         // T_(x,a): the y in N(x) n N(a)
            const int32_t ny = int32_t(__ldg(A.toff + rowx + mx + 1) - y0);
            if (A.stats && lane == 0) stat += 4 + 4 + 16 + 16;
            if (ny == 0) continue;
            const int32_t dx = int32_t(__ldg(g.rowptr + x + 1) - rowx);
            const int32_t lox = lower_bound_dev(g.col + rowx, dx, x);    // positions of y > x
            const int32_t k0 = lower_bound_dev(A.T + y0, ny, lox);
            if (A.stats && lane == 0) stat += 8 + w_probe_bytes(dx) + w_probe_bytes(ny);
            if (k0 >= ny) continue;
            const bool agg = ny <= 65535;
            stat += k23_walk_b<1, ET>(A, E, agg ? wc : nullptr, rowx, A.T + y0, k0, ny, mx, 0, lane);
            if (agg) {
                __syncwarp();
                stat += k23_flush<32, ET>(A, E, wc, rowx, mx, lane);
                __syncwarp();
            }
        }
        __syncthreads();
        // walk B, block items: windows above K23_WARP_CAP, one at a time
        for (int32_t i = 0; i < da; i++) {
            const int32_t mx = __ldg(A.mpos + rowa + i);
            if (mx <= K23_WARP_CAP) continue;                      // uniform
            const int32_t x = __ldg(g.col + rowa + i);
            const int64_t rowx = __ldg(g.rowptr + x);
            const int64_t y0 = __ldg(A.toff + rowx + mx);
            const int32_t ny = int32_t(__ldg(A.toff + rowx + mx + 1) - y0);
            if (ny == 0) continue;
            const int32_t dx = int32_t(__ldg(g.rowptr + x + 1) - rowx);
            const int32_t lox = lower_bound_dev(g.col + rowx, dx, x);
            const int32_t k0 = lower_bound_dev(A.T + y0, ny, lox);
            if (k0 >= ny) continue;
            if (A.stats && tid == 0) stat += 4 + 4 + 16 + 16 + 8 + w_probe_bytes(dx) + w_probe_bytes(ny);
            const bool agg = ny <= 65535 && mx <= 2 * K23_SMEM_WORDS;
            stat += k23_walk_b<K23_THREADS / 32, ET>(A, E, agg ? sc : nullptr, rowx, A.T + y0, k0, ny, mx,
                                                     warp, lane);
            if (agg) {
                __syncthreads();
                stat += k23_flush<K23_THREADS, ET>(A, E, sc, rowx, mx, tid);
                __syncthreads();
            }
        }
        __syncthreads();
        const int nt = s_nt;
        for (int q = tid; q < nt; q += K23_THREADS) {
            const int32_t b = touched[q];
            const uint32_t w = NARROW ? uint32_t(W16[b]) : W[b];
            const unsigned long long e = E[b];
            k23 += w_c3(w);
            if (e) {
                if (w < 2) atomicExch(&ctl->fault, 1);
                else k23e += u128(e) * (w - 2);
                E[b] = 0;
            }
            if (NARROW) W16[b] = 0;
            else W[b] = 0;
            if (A.stats) stat += 4 + 4 + 8 + 4 + (e ? 8 : 0);
        }
    }
    w_flush(A.basis, DB_K23, k23, lane);
    w_flush(A.basis, DB_K23E, k23e, lane);
    w_flush_stat(A.stats, stat, lane);
}

size_t k23_smem_bytes() { return sizeof(uint32_t) * K23_SMEM_WORDS; }

int k23_blocks(int device) {
    cudaFuncSetAttribute(k23_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k23_smem_bytes()));
    cudaFuncSetAttribute(k23_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k23_smem_bytes()));
    int per_sm = 0, per_sm_n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k23_kernel<false>, K23_THREADS, k23_smem_bytes());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_n, k23_kernel<true>, K23_THREADS, k23_smem_bytes());
    per_sm = std::min(per_sm, per_sm_n);
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

// K5-e, one warp per slot (x, y) with y > x (32 consecutive slots per
// chunk), lanes over the w of T_(x,y); 16-bit counters over x's positions
// above y in the warp's own 1024 shared words (or, for up-degrees above 2048
// or lists above 65535, 32-bit counters in a per-warp global area).
__global__ void __launch_bounds__(K5E_THREADS) k5e_kernel(WheelArgs A) {
    extern __shared__ uint32_t sh[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DevGraph &g = A.g;
    Control *ctl = A.ctl;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const int64_t nnz = g.nnz;
    const unsigned long long n_chunks = (unsigned long long)((nnz + 31) / 32);
    uint32_t *wc = sh + warp * K5E_WARP_WORDS;
    uint32_t *gc = A.k5g ? A.k5g + (size_t(blockIdx.x) * (K5E_THREADS / 32) + size_t(warp)) * size_t(A.k5g_words)
                         : nullptr;
    for (int i = lane; i < K5E_WARP_WORDS; i += 32) wc[i] = 0;
    __syncwarp();
    u128 acc = 0;
    uint64_t stat = 0;
    while (true) {
        unsigned long long c = 0;
        int stop = 0;
        if (lane == 0) {
            c = atomicAdd(&ctl->work3, 1ull);
            stop = w_should_stop(ctl, deadline);
        }
        c = __shfl_sync(FULL, c, 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (c >= n_chunks || stop) break;
        const int64_t base = int64_t(c) * 32;
        int32_t xrow = 0;
        if (base + lane < nnz) xrow = row_of_slot(g.rowptr, base + lane, 0, g.n);
        for (int q = 0; q < 32; q++) {
            const int64_t s = base + q;
            if (s >= nnz) break;
            const int32_t x = __shfl_sync(FULL, xrow, q);
            const int32_t y = __ldg(g.col + s);
            const int32_t ts = __ldg(A.t + s);
            if (y < x || ts < 2) continue;
            const int64_t rowx = __ldg(g.rowptr + x);
            const int32_t dx = int32_t(__ldg(g.rowptr + x + 1) - rowx);
            const int32_t py = int32_t(s - rowx);
            const int32_t range = dx - py - 1;                  // positions py+1 .. dx-1
            const int64_t b0 = __ldg(A.toff + s);
            const int32_t *TY = A.T + b0;
            const bool smem = range <= 2 * K5E_WARP_WORDS && ts <= 65535;
            if (!smem && !gc) {
                if (lane == 0) atomicExch(&ctl->fault, 1);    // no counters for this slot
                continue;
            }
            // counts: every w of T_(x,y), every z of T_(x,w) above y (groups
            // of 32 w's, one per lane, walked together)
            for (int32_t k0 = 0; k0 < ts; k0 += 32) {
                const int32_t k = k0 + lane;
                int64_t base = 0;
                int32_t cnt = 0;
                if (k < ts) {
                    const int64_t sw = rowx + __ldg(TY + k);
                    const int64_t w0 = __ldg(A.toff + sw);
                    const int32_t nw = int32_t(__ldg(A.toff + sw + 1) - w0);
                    const int32_t j0 = lower_bound_dev(A.T + w0, nw, py + 1);
                    base = w0 + j0;
                    cnt = nw - j0;
                    if (A.stats) stat += 4 + 16 + w_probe_bytes(nw) + 4ull * uint64_t(cnt);
                }
                warp_lists<false>(A.T, base, cnt, 0, lane, ctl, A.T_len, [&](int32_t pz) {
                    const int32_t z = pz - py - 1;
                    if (!PM_DCHECK(ctl, z >= 0 && z < range)) return;
                    if (smem) atomicAdd(wc + (z >> 1), (z & 1) ? 65536u : 1u);
                    else atomicAdd(gc + z, 1u);
                });
            }
            __syncwarp();
            // C(k, 2) at each z of T_(x,y) above y
            for (int32_t k = lane; k < ts; k += 32) {
                const int32_t pz = __ldg(TY + k);
                if (pz <= py) continue;
                const int32_t z = pz - py - 1;
                const uint32_t v = smem ? ((wc[z >> 1] >> (16 * (z & 1))) & 0xffffu) : gc[z];
                acc += w_c2(v);
                if (A.stats) stat += 4;
            }
            __syncwarp();
            if (smem) {
                for (int32_t w = lane; w < (range + 1) / 2; w += 32) wc[w] = 0;
            } else {
                for (int32_t w = lane; w < range; w += 32) gc[w] = 0;
            }
            __syncwarp();
        }
    }
    w_flush(A.basis, DB_K5E, acc, lane);
    w_flush_stat(A.stats, stat, lane);
}

int64_t k5e_global_words(int64_t max_updeg, int64_t max_degree) {
    return (max_updeg > 2 * K5E_WARP_WORDS || max_degree > 65536) ? std::max<int64_t>(max_updeg, 1) : 0;
}

size_t k5e_smem_bytes() { return sizeof(uint32_t) * (K5E_THREADS / 32) * K5E_WARP_WORDS; }

int k5e_blocks(int device) {
    cudaFuncSetAttribute(k5e_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k5e_smem_bytes()));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k5e_kernel, K5E_THREADS, k5e_smem_bytes());
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

size_t w4_smem_bytes() { return sizeof(uint32_t) * W4_SMEM_WORDS; }

int w4_blocks(int device) {
    cudaFuncSetAttribute(w4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(w4_smem_bytes()));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, w4_kernel, W4_THREADS, w4_smem_bytes());
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

int64_t tscan_blocks(int64_t nnz) { return (nnz + SC_TILE - 1) / SC_TILE; }

int64_t w4_global_words(int64_t max_degree) { return max_degree > W4_BLOCK_CAP ? max_degree : 0; }

int launch_list_offsets(const WheelArgs &A, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nnz = A.g.nnz;
    if (nnz == 0) return 0;
    const int64_t nb = tscan_blocks(nnz);
    tsum_kernel<<<unsigned(nb), SC_THREADS, 0, s>>>(A.t, nnz, A.bsum);
    tscan_top_kernel<<<1, SC_THREADS, 0, s>>>(A.bsum, nb);
    tscan_kernel<<<unsigned(nb), SC_THREADS, 0, s>>>(A.t, nnz, A.bsum, A.toff);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("list offset scan launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

int launch_wheel(const WheelArgs &A, int passes, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    cudaStream_t s = (cudaStream_t)stream;
    if (A.g.nnz == 0) return 0;
    if (launch_list_offsets(A, stream)) return -1;
    if (A.g.hub && A.hub_rank && A.n_hubs > 0)
        hub_rank_kernel<<<unsigned(A.n_hubs), SC_THREADS, 0, s>>>(A.g.bits, A.g.words, A.hub_rank);
    cudaMemsetAsync(&A.ctl->work3, 0, sizeof(unsigned long long), s);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tlist_kernel, TL_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    tlist_kernel<<<device_sm_count(device) * per_sm, TL_WARPS * 32, 0, s>>>(A);
    if (passes & DP_K23E) {
        mpos_kernel<<<device_sm_count(device) * per_sm, TL_WARPS * 32, 0, s>>>(A);
        cudaMemsetAsync(&A.ctl->work3, 0, sizeof(unsigned long long), s);
        if (A.k23_narrow) {
            cudaFuncSetAttribute(k23_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k23_smem_bytes()));
            k23_kernel<true><<<A.k23_blocks, K23_THREADS, k23_smem_bytes(), s>>>(A);
        } else {
            cudaFuncSetAttribute(k23_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k23_smem_bytes()));
            k23_kernel<false><<<A.k23_blocks, K23_THREADS, k23_smem_bytes(), s>>>(A);
        }
    }
    if (passes & DP_K5E) {
        cudaMemsetAsync(&A.ctl->work3, 0, sizeof(unsigned long long), s);
        cudaFuncSetAttribute(k5e_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k5e_smem_bytes()));
        k5e_kernel<<<A.k5e_blocks, K5E_THREADS, k5e_smem_bytes(), s>>>(A);
    }
    if (passes & DP_W4) {
        if (A.gcnt) cudaMemsetAsync(A.gcnt, 0, sizeof(uint32_t) * size_t(A.gcnt_words) * size_t(A.w4_blocks), s);
        cudaMemsetAsync(&A.ctl->work3, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(&A.ctl->work2, 0, sizeof(unsigned long long), s);
        cudaFuncSetAttribute(w4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(w4_smem_bytes()));
        w4_kernel<<<A.w4_blocks, W4_THREADS, w4_smem_bytes(), s>>>(A);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("neighbourhood-graph kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

// Kernels launched by launch_wheel for a pass set.
int wheel_launches(const WheelArgs &A, int passes) {
    if (A.g.nnz == 0) return 0;
    return 4 + int(A.g.hub && A.hub_rank && A.n_hubs > 0) + 2 * int((passes & DP_K23E) != 0) +
           int((passes & DP_W4) != 0) + int((passes & DP_K5E) != 0);
}

}  // namespace pm
