// Clique counting kernel (sm_103a) for the rooted plans of the unlabeled
// 4- and 5-clique (edge- and vertex-induced counts coincide for cliques).
//
// An occurrence of K_k has a highest-ranked vertex a and a second-highest
// vertex b adjacent to it; its other k - 2 vertices form a K_{k-2} inside
//   S(a, b) = N(a) n N(b) n [0, b).
// A warp takes one task (a, b) at a time -- an oriented edge with b < a, the
// rooted plans' task space, so per-root counts stay exact -- builds S(a, b)
// once from the bound-cut slice of the shorter of the two adjacency rows,
// filtered by membership in the other row and compacted with __ballot_sync,
// and then counts
//   K4: the edges inside S: for x = S[i], |S[0, i) n N(x)|;
//   K5: the triangles inside S: for x = S[i], the edges inside the second
//       materialised set S[0, i) n N(x).
// The last intersections reuse the materialised set instead of re-reading
// N(a) and N(b) for every prefix.  For each x the cheaper side is taken:
// test the i earlier members in N(x) (one bit read when x has a hub
// bitmap, else a binary search in its row), or walk N(x) between S[0] and x
// and look each element up in S.  The work items of 32 consecutive members
// are flattened over the lanes with a warp prefix sum, so every lane has an
// item whatever the set sizes.  Sets longer than the per-warp shared buffer
// go to a per-warp global spill area of 2 x (largest degree) entries, which
// the host allocates whenever the largest degree exceeds the buffer.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "devgraph.cuh"
#include "internal.hpp"

namespace pm {

constexpr int CQ_WARPS = 8;      // warps per block
constexpr int CQ_CAP = 1024;     // shared entries per warp for each of the two sets

struct CliqueArgs {
    DevGraph g;
    DevTasks tasks;
    int k;                       // 4 or 5
    int counter;
    uint64_t *counters;
    Control *ctl;
    int32_t sample_stride;       // every stride-th 32-task chunk (autotuning)
    int32_t *spill;              // 2 * spill_len entries per warp, or nullptr
    int64_t spill_len;
    unsigned long long *stats;
    int32_t balanced;            // 1: strided chunks, weighted sides, per-task deadline checks
    uint64_t *deg_out;           // K4 only, nullable: 128-bit sum over 4-cliques of their degrees
};

// First index in s[0, len) whose value is >= key; s is written by this
// kernel, so it is read with plain loads.
__device__ __forceinline__ int32_t lower_bound_set(const int32_t *s, int32_t len, int32_t key) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = int32_t((uint32_t(lo) + uint32_t(hi)) >> 1);
        if (s[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool has_bitmap(const DevGraph &g, int32_t v) {
    return g.hub && __ldg(g.hub + v) >= 0;
}

// Walking side for x against the members S[0, i): the row range of N(x)
// inside [S[0], x).  Returns its length and start (index into col); deg
// receives |N(x)|.
__device__ __forceinline__ int32_t walk_range(const DevGraph &g, int32_t x, int32_t s0,
                                              int64_t &start, int32_t &deg) {
    const int64_t rb = __ldg(g.rowptr + x);
    const int32_t d = int32_t(__ldg(g.rowptr + x + 1) - rb);
    const int32_t plo = lower_bound_dev(g.col + rb, d, s0);
    const int32_t phi = plo + lower_bound_dev(g.col + rb + plo, d - plo, x);
    start = rb + plo;
    deg = d;
    return phi - plo;
}

__device__ __forceinline__ uint32_t bit_length(uint32_t v) { return 32u - uint32_t(__clz(v | 1u)); }

// Walk instead of test?  Plain: the shorter side.  Weighted (balanced
// mode): each side's item count times the depth of its binary searches --
// a test searches N(x) (degree d), a walk searches the i members.
__device__ __forceinline__ bool prefer_walk(int32_t len, int32_t i, int32_t d, bool weighted) {
    if (!weighted) return len < i;
    return uint64_t(len) * bit_length(uint32_t(i)) < uint64_t(i) * bit_length(uint32_t(d));
}

// Testing is chosen when x has a bitmap or few earlier members; otherwise
// the shorter of the two sides.
constexpr int32_t CQ_TEST_ALWAYS = 24;

// Edges inside the sorted set S[0, s): this lane's share of
// sum over i of |S[0, i) n N(S[i])|.
template <bool STATS, bool DEG = false>
__device__ uint64_t edges_within(const DevGraph &g, const int32_t *S, int32_t s, int lane,
                                 uint64_t &stat, bool weighted, uint64_t *dsum = nullptr) {
    uint64_t hits = 0;
    if (s < 2) return 0;
    const int32_t s0 = S[0];
    for (int32_t g0 = 0; g0 < s; g0 += 32) {
        const int32_t i = g0 + lane;
        int32_t x = 0, cost = 0, walk = 0;
        int64_t start = 0;
        if (i < s && i > 0) {
            x = S[i];
            cost = i;
            if (i > CQ_TEST_ALWAYS && !has_bitmap(g, x)) {
                int32_t d = 0;
                const int32_t len = walk_range(g, x, s0, start, d);
                if (prefer_walk(len, i, d, weighted)) {
                    walk = 1;
                    cost = len;
                }
            }
            if (STATS) stat += 8 + 4 * uint64_t(i + cost);
        }
        int32_t incl = cost;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int32_t total = __shfl_sync(FULL, incl, 31);
        const int32_t excl = incl - cost;
        for (int32_t t0 = 0; t0 < total; t0 += 32) {
            const int32_t t = t0 + lane;
            // owner: the first lane whose inclusive sum exceeds t
            int lo = 0, hi = 31;
#pragma unroll
            for (int step = 0; step < 5; step++) {
                const int mid = (lo + hi) >> 1;
                if (__shfl_sync(FULL, incl, mid) > t) hi = mid;
                else lo = mid + 1;
            }
            const int32_t xo = __shfl_sync(FULL, x, lo);
            const int32_t io = __shfl_sync(FULL, i, lo);
            const int32_t wo = __shfl_sync(FULL, walk, lo);
            const int64_t so = __shfl_sync(FULL, start, lo);
            const int32_t eo = __shfl_sync(FULL, excl, lo);
            if (t < total) {
                const int32_t j = t - eo;
                bool hit;
                int32_t y;
                if (!wo) {
                    y = S[j];
                    hit = contains(g, xo, y);
                } else {
                    y = __ldg(g.col + so + j);
                    const int32_t p = lower_bound_set(S, io, y);
                    hit = p < io && S[p] == y;
                }
                hits += hit ? 1 : 0;
                // DEG: the degrees of both endpoints of every edge found
                if (DEG && hit)
                    *dsum += uint64_t(__ldg(g.rowptr + xo + 1) - __ldg(g.rowptr + xo)) +
                             uint64_t(__ldg(g.rowptr + y + 1) - __ldg(g.rowptr + y));
            }
        }
    }
    return hits;
}

// D = S[0, i) n N(x) in ascending order; returns |D| (warp-uniform).
template <bool STATS>
__device__ int32_t restrict_set(const DevGraph &g, const int32_t *S, int32_t i, int32_t x,
                                int32_t *D, int lane, uint64_t &stat, bool weighted) {
    int32_t len = i, walk = 0;
    int64_t start = 0;
    if (i > CQ_TEST_ALWAYS && !has_bitmap(g, x)) {
        int32_t d = 0;
        const int32_t w = walk_range(g, x, S[0], start, d);
        if (prefer_walk(w, i, d, weighted)) {
            walk = 1;
            len = w;
        }
    }
    if (STATS && lane == 0) stat += 8 + 4 * uint64_t(i + len);
    int32_t cnt = 0;
    for (int32_t j0 = 0; j0 < len; j0 += 32) {
        const int32_t j = j0 + lane;
        int32_t y = 0;
        bool keep = false;
        if (j < len) {
            if (!walk) {
                y = S[j];
                keep = contains(g, x, y);
            } else {
                y = __ldg(g.col + start + j);
                const int32_t p = lower_bound_set(S, i, y);
                keep = p < i && S[p] == y;
            }
        }
        const uint32_t m = __ballot_sync(FULL, keep);
        if (keep) D[cnt + __popc(m & ((1u << lane) - 1))] = y;
        cnt += __popc(m);
    }
    __syncwarp();
    return cnt;
}

// Lane 0 reads the timer and the shared status; true (on every lane) once
// the deadline has expired or another warp has stopped the launch.
__device__ __forceinline__ bool cq_stop(Control *ctl, uint64_t deadline, int lane) {
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

template <bool STATS, bool DEG>
__global__ void __launch_bounds__(CQ_WARPS * 32)
clique_kernel(CliqueArgs A) {
    extern __shared__ __align__(16) int32_t cq_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const DevGraph &g = A.g;
    // per warp: S, and for the 5-clique the second set D
    const int per_warp = (A.k == 5 ? 2 : 1) * CQ_CAP;
    int32_t *sS = cq_smem + warp * per_warp;
    int32_t *sD = sS + CQ_CAP;
    const int64_t gw = int64_t(blockIdx.x) * CQ_WARPS + warp;
    int32_t *pS = A.spill ? A.spill + gw * 2 * A.spill_len : nullptr;
    int32_t *pD = A.spill ? pS + A.spill_len : nullptr;
    Control *ctl = A.ctl;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    const int64_t ntasks = A.tasks.ntasks[TASKS_LOWER];
    const int64_t *off = A.tasks.off[TASKS_LOWER];
    const unsigned long long stride =
        (unsigned long long)(A.sample_stride > 1 ? A.sample_stride : 1);
    const unsigned long long n_chunks = (unsigned long long)((ntasks + 31) / 32);
    const unsigned long long n_sampled = (n_chunks + stride - 1) / stride;
    uint64_t hits = 0, stat = 0;
    u128 degsum = 0;
    bool alive = true;
    while (alive) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(&ctl->work3, 1ull);
        w = __shfl_sync(FULL, w, 0);
        if (w >= n_sampled || cq_stop(ctl, deadline, lane)) break;
        // this lane's task of the chunk: root by binary search over the offsets.
        // Plain mode: chunk c holds tasks 32c .. 32c + 31 (one root's
        // neighbours side by side); balanced mode: tasks c + j * n_chunks, so
        // the tasks between one hub and its hub neighbours, adjacent in the
        // hub's row, go to different chunks.  Either way every task is in
        // exactly one chunk, and the tasks past the end are a suffix of lanes.
        const int64_t c = int64_t(w * stride);
        const int64_t e = A.balanced ? c + int64_t(lane) * int64_t(n_chunks) : c * 32 + lane;
        // (lower-neighbour tasks index a's row from its start, so the index of b
        // in N(a) is |N(a) n [0, b)|)
        int32_t a = -1, b = -1, ia = 0;
        if (e < ntasks) {
            int64_t lo = 0, hi = A.tasks.nroots;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(off + mid) <= e) lo = mid;
                else hi = mid;
            }
            a = A.tasks.roots ? __ldg(A.tasks.roots + lo) : int32_t(g.n - 1 - lo);
            ia = int32_t(e - __ldg(off + lo));
            b = __ldg(g.col + __ldg(g.rowptr + a) + ia);
        }
        for (int q = 0; q < 32 && alive; q++) {
            const int32_t ra = __shfl_sync(FULL, a, q);
            const int32_t rb = __shfl_sync(FULL, b, q);
            const int32_t la = __shfl_sync(FULL, ia, q);
            if (ra < 0) break;                       // tasks past the end are at the tail
            if (A.balanced && q > 0 && cq_stop(ctl, deadline, lane)) {
                alive = false;
                break;
            }
            const int64_t rowa = __ldg(g.rowptr + ra);
            const int64_t rowb = __ldg(g.rowptr + rb);
            int32_t lb = 0;
            if (lane == 0) lb = lower_bound_dev(g.col + rowb, int32_t(__ldg(g.rowptr + rb + 1) - rowb), rb);
            lb = __shfl_sync(FULL, lb, 0);
            if (STATS && lane == 0) stat += 16 + 4 * uint64_t(la + lb);
            const int32_t n = la <= lb ? la : lb;
            if (n < A.k - 2) continue;
            const int64_t src = la <= lb ? rowa : rowb;
            const int32_t other = la <= lb ? rb : ra;
            int32_t *S = n <= CQ_CAP ? sS : pS;
            int32_t s = 0;
            __syncwarp();                            // every lane is done with the last task's sets
            for (int32_t j0 = 0; j0 < n; j0 += 32) {
                const int32_t j = j0 + lane;
                int32_t x = 0;
                bool keep = false;
                if (j < n) {
                    x = __ldg(g.col + src + j);
                    keep = contains(g, other, x);
                }
                const uint32_t m = __ballot_sync(FULL, keep);
                if (keep) S[s + __popc(m & ((1u << lane) - 1))] = x;
                s += __popc(m);
            }
            __syncwarp();
            if (A.k == 4) {
                if (DEG) {
                    uint64_t ds = 0;
                    const uint64_t h = edges_within<STATS, true>(g, S, s, lane, stat, A.balanced != 0, &ds);
                    hits += h;
                    const uint64_t dab = uint64_t(__ldg(g.rowptr + ra + 1) - rowa) +
                                         uint64_t(__ldg(g.rowptr + rb + 1) - rowb);
                    degsum += u128(h) * dab + ds;
                } else {
                    hits += edges_within<STATS>(g, S, s, lane, stat, A.balanced != 0);
                }
                continue;
            }
            for (int32_t i = 2; i < s; i++) {
                if ((i & 63) == 0 && cq_stop(ctl, deadline, lane)) {
                    alive = false;
                    break;
                }
                int32_t *D = i <= CQ_CAP ? sD : pD;
                const int32_t c2 = restrict_set<STATS>(g, S, i, S[i], D, lane, stat, A.balanced != 0);
                if (c2 >= 2) hits += edges_within<STATS>(g, D, c2, lane, stat, A.balanced != 0);
                __syncwarp();
            }
        }
    }
    u128 acc = hits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(acc), o);
        const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(acc >> 64), o);
        acc += (u128(hi) << 64) | lo;
    }
    if (lane == 0 && acc != 0) add_u128(A.counters + 2 * int64_t(A.counter), acc);
    if (DEG) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(degsum), o);
            const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(degsum >> 64), o);
            degsum += (u128(hi) << 64) | lo;
        }
        if (lane == 0 && degsum != 0) add_u128(A.deg_out, degsum);
    }
    if (STATS) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) stat += __shfl_xor_sync(FULL, stat, o);
        if (lane == 0 && stat) atomicAdd(A.stats, (unsigned long long)stat);
    }
}

static size_t clique_smem(int k) {
    return size_t(CQ_WARPS) * (k == 5 ? 2 : 1) * CQ_CAP * sizeof(int32_t);
}

template <bool STATS, bool DEG = false>
static int clique_blocks_for(int device, int k) {
    auto kern = clique_kernel<STATS, DEG>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(clique_smem(5)));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CQ_WARPS * 32, clique_smem(k));
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

int64_t clique_warps(int device) {
    int most = 0;
    for (int k = 4; k <= 5; k++) {
        most = std::max(most, clique_blocks_for<false>(device, k));
        most = std::max(most, clique_blocks_for<true>(device, k));
        most = std::max(most, clique_blocks_for<false, true>(device, k));
    }
    return int64_t(most) * CQ_WARPS;
}

int64_t clique_spill_len(int64_t max_degree) { return max_degree > CQ_CAP ? max_degree : 0; }

int launch_clique(const DevGraph &g, const DevTasks &tasks, int k, int counter,
                  uint64_t *counters, int32_t *spill, int64_t spill_len, int sample_stride,
                  Control *ctl, unsigned long long *stats, void *stream, uint64_t *deg_out) {
    int device = 0;
    cudaGetDevice(&device);
    cudaStream_t s = (cudaStream_t)stream;
    CliqueArgs A;
    A.g = g;
    A.tasks = tasks;
    A.k = k;
    A.counter = counter;
    A.counters = counters;
    A.ctl = ctl;
    A.sample_stride = sample_stride;
    A.spill = spill;
    A.spill_len = spill_len;
    A.stats = stats;
    A.deg_out = deg_out;
    // balanced scheduling is opt-in until it has been timed against the
    // plain one (PM_CLIQUE_BALANCED=1)
    const char *bal = std::getenv("PM_CLIQUE_BALANCED");
    A.balanced = (bal && bal[0] == '1') ? 1 : 0;
    cudaMemsetAsync(&ctl->work3, 0, sizeof(unsigned long long), s);
    if (deg_out && k == 4) {
        const int blocks = clique_blocks_for<false, true>(device, k);
        clique_kernel<false, true><<<blocks, CQ_WARPS * 32, clique_smem(k), s>>>(A);
    } else if (stats) {
        const int blocks = clique_blocks_for<true>(device, k);
        clique_kernel<true, false><<<blocks, CQ_WARPS * 32, clique_smem(k), s>>>(A);
    } else {
        const int blocks = clique_blocks_for<false>(device, k);
        clique_kernel<false, false><<<blocks, CQ_WARPS * 32, clique_smem(k), s>>>(A);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("clique kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

}  // namespace pm
