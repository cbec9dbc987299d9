// Device helpers shared by the counting kernels: the global timer, binary
// search in a sorted adjacency row, adjacency membership (hub bitmap or
// binary search), and the exact 128-bit counter update.
#pragma once

#include <cstdint>

#include "plan.hpp"

namespace pm {

typedef unsigned __int128 u128;

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First index in a[0, len) whose value is >= key.
__device__ __forceinline__ int32_t lower_bound_dev(const int32_t *__restrict__ a, int32_t len,
                                                   int32_t key) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = int32_t((uint32_t(lo) + uint32_t(hi)) >> 1);
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains(const DevGraph &g, int32_t v, int32_t x) {
    if (g.hub) {
        const int32_t h = __ldg(g.hub + v);
        if (h >= 0) return (__ldg(g.bits + int64_t(h) * g.words + (x >> 5)) >> (x & 31)) & 1u;
    }
    const int64_t b = __ldg(g.rowptr + v);
    const int32_t len = int32_t(__ldg(g.rowptr + v + 1) - b);
    const int32_t *a = g.col + b;
    const int32_t p = lower_bound_dev(a, len, x);
    return p < len && __ldg(a + p) == x;
}

// Bounds checks of the PM_DEBUG build: an index derived from data must
// satisfy `cond` for the access that follows; otherwise the control block's
// fault word becomes 2 (reported by the host as an error) and the caller
// skips the access.  Without PM_DEBUG the check compiles to `true`.
#ifdef PM_DEBUG
#define PM_DCHECK(ctl, cond) ((cond) ? true : (atomicExch(&(ctl)->fault, 2), false))
#else
#define PM_DCHECK(ctl, cond) true
#endif

__device__ __forceinline__ void add_u128(uint64_t *counter, u128 v) {
    const unsigned long long lo = (unsigned long long)(uint64_t)v;
    unsigned long long hi = (unsigned long long)(uint64_t)(v >> 64);
    const unsigned long long old = atomicAdd((unsigned long long *)counter, lo);
    if (old + lo < old) hi += 1;
    if (hi) atomicAdd((unsigned long long *)counter + 1, hi);
}

}  // namespace pm
