// Allocation-free entry point: edge-induced 4-cycle counting whose scratch
// lives in a fixed array compiled into the library.
//
// Some callers cannot allocate device memory at the moment they need a count:
// code running inside a memory pool that is already fully reserved by its
// framework, real-time loops that must not call into the allocator (which can
// synchronise the device or block on a lock), and embedders that hand out
// every byte of device memory themselves.  For them this file provides a
// variant of the wedge-pair kernel (the 4-cycle counter behind pm_count) that
// takes the graph and the output from the caller and uses, as its scratch,
// the file-scope array `g_wedge_scratch` below instead of memory obtained
// from cudaMalloc or from the allocator set with pm_set_allocator.
//
// The array is a static device variable: every GPU that loads the library
// holds it (NOALLOC_SCRATCH_WORDS 32-bit words = 16 MiB) until the process
// exits, whether or not the entry point is used.  Host code only sees a
// host-side stand-in for its name, so its device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made on that
// device (with that device current); that first call should therefore come
// before any CUDA stream capture.
#include <climits>
#include <cstring>
#include <mutex>

#include "internal.hpp"

namespace pm {

namespace {

constexpr size_t NOALLOC_SCRATCH_WORDS = size_t(1) << 22;   // 16 MiB of uint32 counters
constexpr int NOALLOC_THREADS = 512;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Scratch shared by every call: per-block dense counters (blocks x n words;
// the kernel's reset walk leaves them zero and every call clears them again
// before launching) and the cursor that hands roots to blocks.
static __device__ __align__(256) uint32_t g_wedge_scratch[NOALLOC_SCRATCH_WORDS];
static __device__ __align__(256) unsigned long long g_wedge_cursor;

std::mutex g_symbols_mu;
uint32_t *g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};
unsigned long long *g_cursor_ptr[NOALLOC_MAX_DEVICES] = {};

typedef unsigned __int128 u128;

__device__ __forceinline__ int32_t lb32(const int32_t *__restrict__ a, int32_t len, int32_t key) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = int32_t((uint32_t(lo) + uint32_t(hi)) >> 1);
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// For every root a (largest id first) and each neighbour b < a, each
// neighbour c < a of b is the opposite corner of the 4-cycles a-b-c-d-a with
// a as largest id; summing the old value of an atomic per-c counter over all
// such 2-paths gives sum_c C(w_c, 2), one count per 4-cycle.  A second walk
// over the same 2-paths returns the touched counters to zero.
__global__ void __launch_bounds__(NOALLOC_THREADS)
wedge_pairs_static_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          int64_t n, uint32_t *scratch, unsigned long long *cursor,
                          unsigned long long *count) {
    __shared__ unsigned long long s_root;
    __shared__ unsigned long long s_acc[NOALLOC_THREADS / 32];
    uint32_t *cnt = scratch + size_t(blockIdx.x) * size_t(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long acc = 0;
    for (;;) {
        if (threadIdx.x == 0) s_root = atomicAdd(cursor, 1ull);
        __syncthreads();
        const unsigned long long r = s_root;
        __syncthreads();
        if (r >= (unsigned long long)n) break;
        const int32_t a = int32_t(n - 1 - int64_t(r));
        const int64_t abase = __ldg(rowptr + a);
        const int32_t adeg = int32_t(__ldg(rowptr + a + 1) - abase);
        const int32_t lo = lb32(col + abase, adeg, a);   // neighbours of a below a
        for (int pass = 0; pass < 2; pass++) {
            for (int i = warp; i < lo; i += nwarps) {
                const int32_t b = __ldg(col + abase + i);
                const int64_t bb = __ldg(rowptr + b);
                const int32_t bd = int32_t(__ldg(rowptr + b + 1) - bb);
                const int32_t bl = lb32(col + bb, bd, a);
                for (int32_t j = lane; j < bl; j += 32) {
                    const int32_t c = __ldg(col + bb + j);
                    if (pass == 0) acc += atomicAdd(cnt + c, 1u);
                    else cnt[c] = 0;
                }
            }
            __syncthreads();
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 total = 0;
        for (int w = 0; w < nwarps; w++) total += s_acc[w];
        const unsigned long long lo64 = (unsigned long long)(uint64_t)total;
        unsigned long long hi64 = (unsigned long long)(uint64_t)(total >> 64);
        const unsigned long long old = atomicAdd(count, lo64);
        if (old + lo64 < old) hi64 += 1;
        if (hi64) atomicAdd(count + 1, hi64);
    }
}

}  // namespace

}  // namespace pm

extern "C" pm_status pm_count_c4_noalloc(const int64_t *rowptr, const int32_t *col, int64_t n,
                                         uint64_t *count, void *stream) {
    using namespace pm;
    if (!rowptr || !col || !count || n < 1) {
        set_error("pm_count_c4_noalloc: null pointer or n < 1");
        return PM_EINVAL;
    }
    if (size_t(n) > NOALLOC_SCRATCH_WORDS) {
        set_error("pm_count_c4_noalloc: n exceeds the built-in scratch (at most 4194304 vertices)");
        return PM_EINVAL;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e) {
        set_error(std::string("pm_count_c4_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return PM_ECUDA;
    }
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) {
        set_error("pm_count_c4_noalloc: device ordinal beyond the supported range");
        return PM_EUNSUPPORTED;
    }
    uint32_t *scratch;
    unsigned long long *cursor;
    {
        // once per device, with that device current: device addresses of the
        // file-scope arrays (their host names are only stand-ins)
        std::lock_guard<std::mutex> lk(g_symbols_mu);
        if (!g_scratch_ptr[device]) {
            void *sp = nullptr, *cp = nullptr;
            e = cudaGetSymbolAddress(&sp, g_wedge_scratch);
            if (!e) e = cudaGetSymbolAddress(&cp, g_wedge_cursor);
            if (e) {
                set_error(std::string("pm_count_c4_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
                return PM_ECUDA;
            }
            g_scratch_ptr[device] = static_cast<uint32_t *>(sp);
            g_cursor_ptr[device] = static_cast<unsigned long long *>(cp);
        }
        scratch = g_scratch_ptr[device];
        cursor = g_cursor_ptr[device];
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e || sms < 1) sms = 1;
    const int64_t fit = int64_t(NOALLOC_SCRATCH_WORDS / size_t(n));
    const int blocks = int(fit < sms ? fit : sms);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * size_t(n) * size_t(blocks), s);
    if (!e) e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (!e) e = cudaMemsetAsync(count, 0, 2 * sizeof(uint64_t), s);
    if (e) {
        set_error(std::string("pm_count_c4_noalloc: clearing scratch: ") + cudaGetErrorString(e));
        return PM_ECUDA;
    }
    wedge_pairs_static_kernel<<<blocks, NOALLOC_THREADS, 0, s>>>(
        rowptr, col, n, scratch, cursor, reinterpret_cast<unsigned long long *>(count));
    e = cudaGetLastError();
    if (e) {
        set_error(std::string("pm_count_c4_noalloc: launch: ") + cudaGetErrorString(e));
        return PM_ECUDA;
    }
    return PM_OK;
}
