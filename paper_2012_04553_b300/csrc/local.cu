// Out-neighbourhood adjacency bitmaps (sm_103a): cliques counted from each
// vertex's neighbours ranked above it.
//
// Every clique has exactly one lowest-ranked vertex v, and its other
// vertices lie in M = N(v) n (v, n) (at most a few hundred vertices on
// R-MAT graphs even when v's degree is in the tens of thousands, because
// vertices are ranked by degree).  For each v this pass builds the adjacency
// matrix of the graph induced on M as bit rows (row i has bit j when
// M[i] ~ M[j]) and counts on it with AND and popcount:
//   4-cliques with lowest vertex v = triangles of M: for i < j adjacent,
//       popc(R_i & R_j) over the members above j;
//   5-cliques = 4-cliques of M: for each such triangle (i, j, k), popc of
//       R_i & R_j & R_k above k;
//   4-cliques per edge (edge-induced K4 count of each edge's common
//       neighbourhood): an edge (M[i], M[j]) of M lies in popc(R_i & R_j)
//       4-cliques with lowest vertex v, an edge (v, M[i]) in the number of
//       triangles of M through i; added to the edge's slot in the row of its
//       lower-ranked endpoint.
// Rows are built by walking each member's own higher neighbours (a
// coalesced read of its row) and locating them in M by binary search in
// registers or shared memory, instead of a binary search in a global row
// per member pair.  Neighbourhoods of at most 32 members take one warp with
// one row per lane; larger ones a block with the rows in shared memory (or,
// above LC_SMEM_S members, in a per-block global area).
#include "devgraph.cuh"
#include "internal.hpp"

namespace pm {

constexpr int LC_THREADS = 512;
constexpr int LC_WARPS = LC_THREADS / 32;
constexpr int LC_SMEM_S = 704;                       // members whose rows fit shared memory
constexpr int LC_PITCH_MAX = ((LC_SMEM_S + 31) / 32) | 1;

// Algorithmic bytes of a row walk (instrumented runs): row offsets, the
// search for its end, 4 B per element read.
__device__ __forceinline__ uint64_t walk_bytes(int64_t from, int64_t to, int64_t row_len) {
    return 16 + 4ull * uint64_t(row_len > 1 ? 65 - __clzll(uint64_t(row_len)) : 1) +
           4ull * uint64_t(to - from);
}

__device__ __forceinline__ void lc_flush_stat(unsigned long long *stats, uint64_t v, int lane) {
    if (!stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(stats, (unsigned long long)v);
}

__device__ __forceinline__ int32_t lc_lowdeg(const LocalArgs &A, int32_t v) {
    const int64_t r = A.g.n - 1 - v;
    return int32_t(__ldg(A.low_off + r + 1) - __ldg(A.low_off + r));
}

__device__ __forceinline__ void lc_flush(uint64_t *basis, int idx, u128 v, int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(FULL, uint64_t(v), o);
        const uint64_t hi = __shfl_xor_sync(FULL, uint64_t(v >> 64), o);
        v += (u128(hi) << 64) | lo;
    }
    if (lane == 0 && v != 0) add_u128(basis + 2 * idx, v);
}

// End (exclusive, index into col) of x's neighbours in (x, last]: the walk
// that locates x's higher neighbours in M stops at M's last member.
__device__ __forceinline__ int64_t walk_end(const DevGraph &g, int32_t x, int64_t from, int32_t last) {
    const int64_t e = __ldg(g.rowptr + x + 1);
    return from + lower_bound_dev(g.col + from, int32_t(e - from), last + 1);
}

// Vertices with 3..32 higher neighbours: one warp each, lane i holding M[i]
// and row i.
__global__ void __launch_bounds__(LC_THREADS) local_warp_kernel(LocalArgs A) {
    const int lane = threadIdx.x & 31;
    const DevGraph &g = A.g;
    const uint64_t deadline = *(volatile unsigned long long *)&A.ctl->deadline;
    const int64_t warps = int64_t(gridDim.x) * LC_WARPS;
    u128 k4 = 0, k5 = 0;
    uint64_t stat = 0;
    uint32_t tick = 0;
    for (int64_t v = int64_t(blockIdx.x) * LC_WARPS + (threadIdx.x >> 5); v < g.n; v += warps) {
        if (((++tick) & 255u) == 0) {
            int stop = 0;
            if (lane == 0) {
                stop = *(volatile int *)&A.ctl->status;
                if (!stop && deadline && global_ns() > deadline) {
                    atomicExch(&A.ctl->status, 1);
                    stop = 1;
                }
            }
            if (__shfl_sync(FULL, stop, 0)) break;
        }
        const int64_t rowv = __ldg(g.rowptr + v);
        const int32_t lowv = lc_lowdeg(A, int32_t(v));
        const int32_t s = int32_t(__ldg(g.rowptr + v + 1) - rowv) - lowv;
        if (s < 3 || s > 32) continue;
        const int32_t Mi = lane < s ? __ldg(g.col + rowv + lowv + lane) : INT_MAX;
        const int32_t last = __shfl_sync(FULL, Mi, s - 1);
        if (A.stats && lane == 0) stat += 16 + 4ull * uint64_t(s);
        uint32_t U = 0;                                   // members above lane adjacent to M[lane]
        for (int i = 0; i < s; i++) {
            const int32_t x = __shfl_sync(FULL, Mi, i);
            const int64_t from = __ldg(g.rowptr + x) + lc_lowdeg(A, x);
            const int64_t to = walk_end(g, x, from, last);
            if (A.stats && lane == 0) stat += walk_bytes(from, to, __ldg(g.rowptr + x + 1) - from);
            uint32_t bits = 0;
            for (int64_t p0 = from; p0 < to; p0 += 32) {
                const int64_t p = p0 + lane;
                const int32_t y = p < to ? __ldg(g.col + p) : INT_MAX;
                int lo = 0, hi = s;
#pragma unroll
                for (int it = 0; it < 6; it++) {
                    const int mid = (lo + hi) >> 1;
                    const int32_t mm = __shfl_sync(FULL, Mi, mid & 31);
                    if (lo < hi) {
                        if (mm < y) lo = mid + 1;
                        else hi = mid;
                    }
                }
                const int32_t at = __shfl_sync(FULL, Mi, lo & 31);
                if (p < to && lo < s && at == y) bits |= 1u << lo;
            }
            bits = __reduce_or_sync(FULL, bits);
            if (lane == i) U = bits;
        }
        uint32_t R = U;                                   // symmetric row
        for (int c = 0; c < s; c++) {
            const uint32_t col_c = __ballot_sync(FULL, (U >> c) & 1u);
            if (lane == c) R |= col_c;
        }
        // triangles of M (i < j < k: k in U_i & U_j) and its 4-cliques
        // (l in U_i & U_j & U_k); the loops are warp-uniform so that every
        // shuffle has all lanes
        uint32_t tri_i = 0;                               // 2 x triangles of M through lane
        for (int j = 0; j < s; j++) {
            const uint32_t Uj = __shfl_sync(FULL, U, j);
            const uint32_t Rj = __shfl_sync(FULL, R, j);
            if ((R >> j) & 1u) tri_i += __popc(R & Rj);
            const uint32_t C = ((U >> j) & 1u) ? (U & Uj) : 0u;
            k4 += __popc(C);
            if (A.want_k5 && __any_sync(FULL, __popc(C) > 1)) {
                for (int k = j + 1; k < s; k++) {
                    const uint32_t Uk = __shfl_sync(FULL, U, k);
                    if ((C >> k) & 1u) k5 += __popc(C & Uk);
                }
            }
        }
        if (A.k4e) {
            if (lane < s && tri_i) atomicAdd(A.k4e + rowv + lowv + lane, tri_i / 2);
            if (A.stats && lane < s && tri_i) stat += 8;
            // edges (M[i], M[j]), i < j, at their slot in M[i]'s row
            for (int i = 0; i < s; i++) {
                const int32_t x = __shfl_sync(FULL, Mi, i);
                const uint32_t Ri = __shfl_sync(FULL, R, i);
                const int64_t from = __ldg(g.rowptr + x) + lc_lowdeg(A, x);
                const int64_t to = walk_end(g, x, from, last);
                if (A.stats && lane == 0) stat += walk_bytes(from, to, __ldg(g.rowptr + x + 1) - from);
                for (int64_t p0 = from; p0 < to; p0 += 32) {
                    const int64_t p = p0 + lane;
                    const int32_t y = p < to ? __ldg(g.col + p) : INT_MAX;
                    int lo = 0, hi = s;
#pragma unroll
                    for (int it = 0; it < 6; it++) {
                        const int mid = (lo + hi) >> 1;
                        const int32_t mm = __shfl_sync(FULL, Mi, mid & 31);
                        if (lo < hi) {
                            if (mm < y) lo = mid + 1;
                            else hi = mid;
                        }
                    }
                    const int32_t at = __shfl_sync(FULL, Mi, lo & 31);
                    const uint32_t Rj = __shfl_sync(FULL, R, lo & 31);
                    if (p < to && lo < s && at == y) {
                        const uint32_t c = __popc(Ri & Rj);
                        if (c) atomicAdd(A.k4e + p, c);
                        if (A.stats && c) stat += 8;
                    }
                }
            }
        }
    }
    lc_flush(A.basis, DB_K4, k4, lane);
    if (A.want_k5) lc_flush(A.basis, DB_K5, k5, lane);
    lc_flush_stat(A.stats, stat, lane);
}

// Vertices with more than 32 higher neighbours: one block each (taken from a
// shared counter), rows in shared memory.
__global__ void __launch_bounds__(LC_THREADS) local_block_kernel(LocalArgs A) {
    extern __shared__ __align__(16) uint32_t lc_smem[];
    __shared__ unsigned long long s_v;
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevGraph &g = A.g;
    const uint64_t deadline = *(volatile unsigned long long *)&A.ctl->deadline;
    // shared layout: rows (LC_SMEM_S x LC_PITCH_MAX), members, per-member
    // triangle sums, per-warp candidate sets C (32 words)
    uint32_t *srows = lc_smem;
    int32_t *smem_M = reinterpret_cast<int32_t *>(srows + LC_SMEM_S * LC_PITCH_MAX);
    uint32_t *tsum = reinterpret_cast<uint32_t *>(smem_M + LC_SMEM_S);
    uint32_t *Cbuf = tsum + LC_SMEM_S;
    uint32_t *Cw = Cbuf + 33 * warp;
    u128 k4 = 0, k5 = 0;
    uint64_t stat = 0;
    for (;;) {
        if (tid == 0) {
            s_v = atomicAdd(&A.ctl->work3, 1ull);
            int stop = *(volatile int *)&A.ctl->status;
            if (!stop && deadline && global_ns() > deadline) {
                atomicExch(&A.ctl->status, 1);
                stop = 1;
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_v >= (unsigned long long)g.n || s_stop) break;
        const int32_t v = int32_t(g.n - 1 - int64_t(s_v));
        const int64_t rowv = __ldg(g.rowptr + v);
        const int32_t lowv = lc_lowdeg(A, v);
        const int32_t s = int32_t(__ldg(g.rowptr + v + 1) - rowv) - lowv;
        if (s <= 32) {
            __syncthreads();
            continue;
        }
        const bool inshared = s <= LC_SMEM_S;
        const int pitch = ((s + 31) / 32) | 1;
        const int W = (s + 31) / 32;
        // neighbourhoods above LC_SMEM_S members: this block's global area
        uint32_t *rows = inshared ? srows : A.grows + size_t(blockIdx.x) * size_t(A.grow_words);
        int32_t *M = inshared ? smem_M : A.gmem + size_t(blockIdx.x) * size_t(A.max_s);
        uint32_t *ts = inshared ? tsum : A.gts + size_t(blockIdx.x) * size_t(A.max_s);
        for (int i = tid; i < s; i += blockDim.x) {
            M[i] = __ldg(g.col + rowv + lowv + i);
            ts[i] = 0;
        }
        for (int64_t w = tid; w < int64_t(s) * pitch; w += blockDim.x) rows[w] = 0;
        __syncthreads();
        const int32_t last = M[s - 1];
        if (A.stats && tid == 0) stat += 16 + 4ull * uint64_t(s);
        // build: warp per member row, symmetric bits
        for (int i = warp; i < s; i += LC_WARPS) {
            const int32_t x = M[i];
            const int64_t from = __ldg(g.rowptr + x) + lc_lowdeg(A, x);
            const int64_t to = walk_end(g, x, from, last);
            if (A.stats && lane == 0) stat += walk_bytes(from, to, __ldg(g.rowptr + x + 1) - from);
            for (int64_t p = from + lane; p < to; p += 32) {
                const int32_t y = __ldg(g.col + p);
                int lo = i + 1, hi = s;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (M[mid] < y) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < s && M[lo] == y) {
                    atomicOr(rows + size_t(i) * pitch + (lo >> 5), 1u << (lo & 31));
                    atomicOr(rows + size_t(lo) * pitch + (i >> 5), 1u << (i & 31));
                }
            }
        }
        __syncthreads();
        // count: warp per row i; j over the members above i adjacent to i
        for (int i = warp; i < s; i += LC_WARPS) {
            const uint32_t *Ri = rows + size_t(i) * pitch;
            for (int wj = (i + 1) >> 5; wj < W; wj++) {
                uint32_t wordj = Ri[wj];
                if (wj == ((i + 1) >> 5)) wordj &= ~0u << ((i + 1) & 31);
                while (wordj) {
                    const int j = wj * 32 + (__ffs(wordj) - 1);
                    wordj &= wordj - 1;
                    const uint32_t *Rj = rows + size_t(j) * pitch;
                    // C = R_i & R_j above j
                    uint32_t c = 0;
                    const int w0 = (j + 1) >> 5;
                    for (int w = lane; w < W; w += 32) {
                        uint32_t word = w >= w0 ? (Ri[w] & Rj[w]) : 0u;
                        if (w == w0) word &= ~0u << ((j + 1) & 31);
                        if (j + 1 >= s) word = 0;
                        Cw[w] = word;
                        c += __popc(word);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
                    if (lane == 0) k4 += c;
                    __syncwarp();
                    if (A.want_k5 && c > 1) {
                        // k over the set bits of C, one per lane
                        for (int wk = w0; wk < W; wk++) {
                            uint32_t wordk = Cw[wk];
                            const int nk = __popc(wordk);
                            for (int b0 = 0; b0 < nk; b0 += 32) {
                                if (b0 + lane < nk) {
                                    const int k = wk * 32 + (__fns(wordk, 0, b0 + lane + 1));
                                    const uint32_t *Rk = rows + size_t(k) * pitch;
                                    const int w1 = (k + 1) >> 5;
                                    uint32_t cc = 0;
                                    for (int w = w1; w < W; w++) {
                                        uint32_t word = Cw[w] & Rk[w];
                                        if (w == w1) word &= ~0u << ((k + 1) & 31);
                                        cc += __popc(word);
                                    }
                                    if (k + 1 >= s) cc = 0;
                                    k5 += cc;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (A.k4e) {
            // per edge (M[i], M[j]): popc(R_i & R_j) at its slot in M[i]'s row;
            // per member the sum over its edges (twice its triangles in M)
            for (int i = warp; i < s; i += LC_WARPS) {
                const int32_t x = M[i];
                const uint32_t *Ri = rows + size_t(i) * pitch;
                const int64_t from = __ldg(g.rowptr + x) + lc_lowdeg(A, x);
                const int64_t to = walk_end(g, x, from, last);
                if (A.stats && lane == 0) stat += walk_bytes(from, to, __ldg(g.rowptr + x + 1) - from);
                for (int64_t p = from + lane; p < to; p += 32) {
                    const int32_t y = __ldg(g.col + p);
                    int lo = i + 1, hi = s;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (M[mid] < y) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < s && M[lo] == y) {
                        const uint32_t *Rj = rows + size_t(lo) * pitch;
                        uint32_t c = 0;
                        for (int w = 0; w < W; w++) c += __popc(Ri[w] & Rj[w]);
                        if (c) {
                            atomicAdd(A.k4e + p, c);
                            atomicAdd(ts + i, c);
                            atomicAdd(ts + lo, c);
                            if (A.stats) stat += 8;
                        }
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < s; i += blockDim.x)
                if (ts[i]) {
                    atomicAdd(A.k4e + rowv + lowv + i, ts[i] / 2);
                    if (A.stats) stat += 8;
                }
        }
        __syncthreads();
    }
    lc_flush(A.basis, DB_K4, k4, lane);
    if (A.want_k5) lc_flush(A.basis, DB_K5, k5, lane);
    lc_flush_stat(A.stats, stat, lane);
}

size_t local_smem_bytes() {
    return sizeof(uint32_t) * (size_t(LC_SMEM_S) * LC_PITCH_MAX + 2 * LC_SMEM_S + 33 * LC_WARPS);
}

int local_blocks(int device) {
    cudaFuncSetAttribute(local_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(local_smem_bytes()));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_block_kernel, LC_THREADS,
                                                  local_smem_bytes());
    if (per_sm < 1) per_sm = 1;
    return device_sm_count(device) * per_sm;
}

int64_t local_grow_words(int64_t max_s) {
    if (max_s <= LC_SMEM_S) return 0;
    return max_s * (((max_s + 31) / 32) | 1);
}

int launch_local(const LocalArgs &A0, int blocks, void *stream) {
    int device = 0;
    cudaGetDevice(&device);
    cudaStream_t s = (cudaStream_t)stream;
    LocalArgs A = A0;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_warp_kernel, LC_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    local_warp_kernel<<<device_sm_count(device) * per_sm, LC_THREADS, 0, s>>>(A);
    cudaMemsetAsync(&A.ctl->work3, 0, sizeof(unsigned long long), s);
    cudaFuncSetAttribute(local_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(local_smem_bytes()));
    local_block_kernel<<<blocks, LC_THREADS, local_smem_bytes(), s>>>(A);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("local bitmap kernel launch: ") + cudaGetErrorString(err));
        return -1;
    }
    return 0;
}

}  // namespace pm
