// Matching kernels (sm_103a): counting and MNI-domain collection over a
// shared queue of (plan, oriented-edge chunk) tasks, plus the MNI morph
// reduction.
//
// Work decomposition.  A task chunk is one plan and 32 consecutive oriented
// edges (root, v) with v < root, roots taken highest-ranked first so hub work
// starts early.  Warps pull chunks from one global counter (persistent grid,
// one launch for every plan of every matched pattern).
//
// Set operations.  A level's candidate set is never materialised: it is the
// bounded slice of the smallest intersected adjacency list, cut by two binary
// searches to the (gt, lt) id window, and filtered 32 elements at a time, one
// per lane (membership in the other intersected lists and absence from the
// differenced lists by binary search; injectivity and label tests).  Survivors
// come from __ballot_sync and are walked in order, which gives the nested
// depth-first enumeration with O(levels) state per warp and no scratch.
// The last `tail` levels are counted as C(|C|, tail); when C is one adjacency
// range minus known vertices, |C| comes from binary searches alone, and the
// lanes of the warp each finish a different prefix in parallel.
//
// Aggregation.  Counts accumulate per lane in 128 bits, are summed across the
// warp, and are added to the pattern's 128-bit counter with a carry into the
// high word, so totals are exact modulo 2^128.  MNI domains are n-bit bitsets
// per (matched pattern, column) set with atomicOr, skipping words whose bit is
// already set.
#include <climits>
#include <cstdio>

#include "internal.hpp"

namespace pm {

typedef unsigned __int128 u128;

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS_PER_BLOCK = 8;
constexpr int CHUNK = 32;

struct WarpState {
    int64_t base[PLAN_KMAX];
    int32_t len[PLAN_KMAX];
    int32_t pos[PLAN_KMAX];
    int32_t cstart[PLAN_KMAX];
    uint32_t mask[PLAN_KMAX];
    int32_t src[PLAN_KMAX];
};

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int64_t lower_bound_dev(const int32_t *__restrict__ a, int64_t len,
                                                   int32_t key) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains(const DevGraph &g, int32_t v, int32_t x) {
    const int64_t b = __ldg(g.rowptr + v), e = __ldg(g.rowptr + v + 1);
    const int32_t *a = g.col + b;
    const int64_t len = e - b;
    const int64_t p = lower_bound_dev(a, len, x);
    return p < len && __ldg(a + p) == x;
}

__device__ __forceinline__ u128 binom(int64_t c, int r) {
    if (r == 0) return 1;
    if (c < r) return 0;
    u128 res = 1;
    for (int i = 0; i < r; i++) res = res * u128(uint64_t(c - i)) / u128(uint64_t(i + 1));
    return res;
}

// m[] holds bound vertices for levels < L in registers; every access uses a
// compile-time index so the array never leaves registers.
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
    int64_t base;
    int32_t len;
    int32_t src;
    int32_t lo, hi;   // open id window (lo, hi)
};

// Candidate slice of level `lv` given the bound prefix.
__device__ __forceinline__ Slice make_slice(const DevGraph &g, const DevLevel &lv, const Bound &m) {
    Slice s;
    int32_t hi = INT_MAX, lo = -1;
    int best = -1;
    int64_t bestd = LLONG_MAX, bestb = 0;
#pragma unroll
    for (int j = 0; j < PLAN_KMAX; j++) {
        if ((lv.lt >> j) & 1) hi = min(hi, m.v[j]);
        if ((lv.gt >> j) & 1) lo = max(lo, m.v[j]);
        if ((lv.isect >> j) & 1) {
            const int64_t b = __ldg(g.rowptr + m.v[j]);
            const int64_t d = __ldg(g.rowptr + m.v[j] + 1) - b;
            if (d < bestd) { bestd = d; best = j; bestb = b; }
        }
    }
    if (best < 0) {   // no intersected list: cannot happen for levels >= 1
        s.base = 0; s.len = 0; s.src = 0; s.lo = lo; s.hi = hi;
        return s;
    }
    const int32_t *a = g.col + bestb;
    const int64_t a0 = lo < 0 ? 0 : lower_bound_dev(a, bestd, lo + 1);
    const int64_t a1 = hi == INT_MAX ? bestd : lower_bound_dev(a, bestd, hi);
    s.base = bestb + a0;
    s.len = a1 > a0 ? int32_t(a1 - a0) : 0;
    s.src = best;
    s.lo = lo;
    s.hi = hi;
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

// |C| for a scanned final stage, computed by the whole warp (same on all lanes).
__device__ __forceinline__ int64_t scan_count(const DevGraph &g, const DevLevel &lv, const Bound &m,
                                              int lane) {
    const Slice s = make_slice(g, lv, m);
    int64_t c = 0;
    for (int32_t off = 0; off < s.len; off += 32) {
        const int32_t i = off + lane;
        bool ok = false;
        if (i < s.len) ok = admissible(g, lv, s.src, m, __ldg(g.col + s.base + i));
        c += __popc(__ballot_sync(FULL, ok));
    }
    return c;
}

__device__ __forceinline__ void set_bit(uint32_t *bits, int32_t x) {
    uint32_t *w = bits + (x >> 5);
    const uint32_t b = 1u << (x & 31);
    if (!(*(volatile uint32_t *)w & b)) atomicOr(w, b);
}

// MNI: record the tail candidate set (all lanes cooperate) and the prefix.
__device__ void record_domains(const DevGraph &g, const DevPlan &P, const Bound &m, int lane,
                               uint32_t *bitsets, int64_t words) {
    const DevLevel &lv = P.lv[P.n_enum];
    const Slice s = make_slice(g, lv, m);
    int64_t c = 0;
    if (P.tail > 1) {
        for (int32_t off = 0; off < s.len; off += 32) {
            const int32_t i = off + lane;
            bool ok = i < s.len && admissible(g, lv, s.src, m, __ldg(g.col + s.base + i));
            c += __popc(__ballot_sync(FULL, ok));
        }
        if (c < P.tail) return;
    }
    uint32_t *tail_bits = bitsets + int64_t(P.dom_base + lv.column) * words;
    bool any = false;
    for (int32_t off = 0; off < s.len; off += 32) {
        const int32_t i = off + lane;
        bool ok = false;
        int32_t x = 0;
        if (i < s.len) {
            x = __ldg(g.col + s.base + i);
            ok = admissible(g, lv, s.src, m, x);
        }
        if (ok) set_bit(tail_bits, x);
        any |= __any_sync(FULL, ok);
    }
    if (P.tail == 0) any = true;
    if (any && lane < P.n_enum) {
        const int32_t v = m.get(lane);
        set_bit(bitsets + int64_t(P.dom_base + P.lv[lane].column) * words, v);
    }
}

template <bool DOMAINS>
__device__ u128 run_dfs(const DevGraph &g, const DevPlan &P, WarpState &S, Bound m, int lane,
                        uint32_t *bitsets, int64_t words, uint64_t deadline, int *status) {
    u128 acc = 0;
    const int last = P.n_enum - 1;
    if (P.n_enum == 2) {
        if (DOMAINS) {
            record_domains(g, P, m, lane, bitsets, words);
        } else if (P.tail == 0) {
            if (lane == 0) acc += 1;
        } else {
            const int64_t c = scan_count(g, P.lv[2], m, lane);
            if (lane == 0) acc += binom(c, P.tail);
        }
        return acc;
    }
    auto setup = [&](int L) {
        const Slice s = make_slice(g, P.lv[L], m);
        if (lane == 0) {
            S.base[L] = s.base;
            S.len[L] = s.len;
            S.pos[L] = 0;
            S.mask[L] = 0;
            S.src[L] = s.src;
        }
        __syncwarp();
    };
    int L = 2;
    setup(L);
    uint32_t iter = 0;
    while (L >= 2) {
        if (deadline && ((++iter & 1023u) == 0)) {
            uint64_t t = 0;
            if (lane == 0) t = global_ns();
            t = __shfl_sync(FULL, t, 0);
            if (t > deadline) {
                if (lane == 0) atomicExch(status, 1);
                return acc;
            }
        }
        const uint32_t mk = S.mask[L];
        if (mk == 0) {
            const int32_t pos = S.pos[L], len = S.len[L];
            if (pos >= len) {
                L--;
                continue;
            }
            const int32_t i = pos + lane;
            bool ok = false;
            int32_t x = 0;
            if (i < len) {
                x = __ldg(g.col + S.base[L] + i);
                ok = admissible(g, P.lv[L], S.src[L], m, x);
            }
            if (!DOMAINS && L == last && P.closed) {
                // lanes finish different prefixes in parallel
                if (ok) {
                    Bound mm = m;
                    mm.set(L, x);
                    acc += binom(closed_count(g, P.lv[L + 1], mm), P.tail);
                }
                __syncwarp();
                if (lane == 0) S.pos[L] = pos + 32;
                __syncwarp();
                continue;
            }
            const uint32_t b = __ballot_sync(FULL, ok);
            __syncwarp();
            if (lane == 0) {
                S.mask[L] = b;
                S.cstart[L] = pos;
                S.pos[L] = pos + 32;
            }
            __syncwarp();
            continue;
        }
        const int bit = __ffs(mk) - 1;
        const int32_t x = __ldg(g.col + S.base[L] + S.cstart[L] + bit);
        __syncwarp();
        if (lane == 0) S.mask[L] = mk & (mk - 1);
        __syncwarp();
        m.set(L, x);
        if (L == last) {
            if (DOMAINS) {
                record_domains(g, P, m, lane, bitsets, words);
            } else if (P.tail == 0) {
                if (lane == 0) acc += 1;
            } else {
                const int64_t c = scan_count(g, P.lv[L + 1], m, lane);
                if (lane == 0) acc += binom(c, P.tail);
            }
        } else {
            L++;
            setup(L);
        }
    }
    return acc;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int mask) {
    const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(v), mask);
    const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(v >> 64), mask);
    return (u128(hi) << 64) | lo;
}

__device__ __forceinline__ void add_u128(uint64_t *counter, u128 v) {
    const unsigned long long lo = (unsigned long long)(uint64_t)v;
    unsigned long long hi = (unsigned long long)(uint64_t)(v >> 64);
    const unsigned long long old = atomicAdd((unsigned long long *)counter, lo);
    if (old + lo < old) hi += 1;
    if (hi) atomicAdd((unsigned long long *)counter + 1, hi);
}

template <bool DOMAINS>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32)
match_kernel(DevGraph g, const DevPlan *__restrict__ plans, int nplans, DevTasks tasks,
             uint64_t *counters, uint32_t *bitsets, int64_t words, Control *ctl) {
    __shared__ WarpState warp_state[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31;
    unsigned long long *work = &ctl->work;
    int *status = &ctl->status;
    const uint64_t deadline = *(volatile unsigned long long *)&ctl->deadline;
    WarpState &S = warp_state[threadIdx.x >> 5];
    const unsigned long long n_echunks = (unsigned long long)((tasks.ntasks + CHUNK - 1) / CHUNK);
    const unsigned long long total = n_echunks * (unsigned long long)nplans;
    while (true) {
        unsigned long long c = 0;
        int stop = 0;
        if (lane == 0) {
            c = atomicAdd(work, 1ull);
            stop = *(volatile int *)status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(status, 1);
                stop = 1;
            }
        }
        c = __shfl_sync(FULL, c, 0);
        stop = __shfl_sync(FULL, stop, 0);
        if (c >= total || stop) break;
        const DevPlan &P = plans[c % nplans];
        const int64_t e = int64_t(c / nplans) * CHUNK + lane;
        int32_t root = -1, v1 = -1;
        if (e < tasks.ntasks) {
            // root index: last i with off[i] <= e
            int64_t lo = 0, hi = tasks.nroots;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(tasks.off + mid) <= e) lo = mid;
                else hi = mid;
            }
            root = tasks.roots ? __ldg(tasks.roots + lo) : int32_t(g.n - 1 - lo);
            v1 = __ldg(g.col + __ldg(g.rowptr + root) + (e - __ldg(tasks.off + lo)));
            if (P.lv[0].label >= 0 && __ldg(g.labels + root) != uint8_t(P.lv[0].label)) root = -1;
            if (P.lv[1].label >= 0 && __ldg(g.labels + v1) != uint8_t(P.lv[1].label)) root = -1;
        }
        u128 acc = 0;
        if (!DOMAINS && P.k == 2) {
            acc = root >= 0 ? 1 : 0;
        } else if (!DOMAINS && P.n_enum == 2 && P.closed) {
            if (root >= 0) {
                Bound m;
#pragma unroll
                for (int i = 0; i < PLAN_KMAX; i++) m.v[i] = 0;
                m.v[0] = root;
                m.v[1] = v1;
                acc = binom(closed_count(g, P.lv[2], m), P.tail);
            }
        } else {
            uint32_t tm = __ballot_sync(FULL, root >= 0);
            while (tm) {
                const int j = __ffs(tm) - 1;
                tm &= tm - 1;
                Bound m;
#pragma unroll
                for (int i = 0; i < PLAN_KMAX; i++) m.v[i] = 0;
                m.v[0] = __shfl_sync(FULL, root, j);
                m.v[1] = __shfl_sync(FULL, v1, j);
                if (DOMAINS && P.k == 2) {
                    if (lane < 2) {
                        const int32_t v = m.v[lane];
                        set_bit(bitsets + int64_t(P.dom_base + P.lv[lane].column) * words, v);
                    }
                    continue;
                }
                acc += run_dfs<DOMAINS>(g, P, S, m, lane, bitsets, words, deadline, status);
            }
        }
        if (!DOMAINS) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += shfl_xor_u128(acc, off);
            if (lane == 0 && acc != 0) add_u128(counters + 2 * int64_t(P.counter), acc);
        }
    }
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

int device_sm_count(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return sms;
}

__global__ void arm_kernel(Control *ctl, uint64_t budget_ns) {
    ctl->work = 0;
    ctl->status = 0;
    ctl->deadline = budget_ns ? global_ns() + budget_ns : 0;
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

template <bool DOMAINS>
static int launch_match(const DevGraph &g, const DevPlan *d_plans, int nplans, const DevTasks &tasks,
                        uint64_t *d_counters, uint32_t *d_bitsets, int64_t words, Control *d_ctl,
                        void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    const int sms = device_sm_count(device);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, match_kernel<DOMAINS>,
                                                  WARPS_PER_BLOCK * 32, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t chunks = ((tasks.ntasks + CHUNK - 1) / CHUNK) * int64_t(nplans);
    int64_t blocks = int64_t(sms) * per_sm;
    const int64_t need = (chunks + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    if (need < blocks) blocks = need > 0 ? need : 1;
    match_kernel<DOMAINS><<<unsigned(blocks), WARPS_PER_BLOCK * 32, 0, (cudaStream_t)stream>>>(
        g, d_plans, nplans, tasks, d_counters, d_bitsets, words, d_ctl);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("match kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

int launch_count(const DevGraph &g, const DevPlan *d_plans, int nplans, const DevTasks &tasks,
                 uint64_t *d_counters, Control *d_ctl, void *stream) {
    return launch_match<false>(g, d_plans, nplans, tasks, d_counters, nullptr, 0, d_ctl, stream);
}

int launch_domains(const DevGraph &g, const DevPlan *d_plans, int nplans, const DevTasks &tasks,
                   uint32_t *d_bitsets, int64_t words, Control *d_ctl, void *stream) {
    return launch_match<true>(g, d_plans, nplans, tasks, nullptr, d_bitsets, words, d_ctl, stream);
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
