// Graph preparation (host) and upload: clean an undirected edge list, order
// vertices by (degree, caller id), build a CSR with sorted rows, and copy it
// to the device.  Every step is O(m) bucketing plus per-row sorts, spread
// over the host's cores.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "internal.hpp"

namespace pm {

namespace {

template <class F>
void parallel_for(int64_t n, F f, int64_t grain = 4096, int64_t min_parallel = 100000) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < min_parallel) nt = 1;
    std::vector<std::thread> th;
    std::atomic<int64_t> next{0};
    auto body = [&]() {
        for (;;) {
            int64_t b = next.fetch_add(grain);
            if (b >= n) break;
            int64_t e = std::min(n, b + grain);
            for (int64_t i = b; i < e; i++) f(i);
        }
    };
    for (unsigned t = 1; t < nt; t++) th.emplace_back(body);
    body();
    for (auto &t : th) t.join();
}

// An array of k entries left uninitialised, for buffers whose every entry is
// written by a parallel pass: the threads that fill it touch its pages first,
// instead of one thread zeroing it beforehand.
template <class T>
std::unique_ptr<T[]> raw_array(size_t k) {
    return std::unique_ptr<T[]>(new T[k]);
}

// Sorts a[0..d) of ids in [0, 2^bits) ascending: short rows by comparison,
// long ones by least-significant-digit radix sort on 8-bit digits (one
// stable counting pass per digit, alternating with a scratch row: on the
// stack up to 4096 entries, on the heap above).
void sort_ids(int32_t *a, int64_t d, int bits) {
    if (d < 128) {
        std::sort(a, a + d);
        return;
    }
    int32_t local[4096];
    std::unique_ptr<int32_t[]> heap;
    if (d > 4096) heap = raw_array<int32_t>(size_t(d));
    int32_t *from = a, *to = heap ? heap.get() : local;
    for (int shift = 0; shift < bits; shift += 8) {
        int64_t cnt[257] = {0};
        for (int64_t i = 0; i < d; i++) cnt[((uint32_t(from[i]) >> shift) & 255u) + 1]++;
        for (int b = 0; b < 256; b++) cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < d; i++) to[cnt[(uint32_t(from[i]) >> shift) & 255u]++] = from[i];
        std::swap(from, to);
    }
    if (from != a) std::copy(from, from + d, a);
}

// Bits needed for ids in [0, n).
int id_bits(int64_t n) {
    int b = 1;
    while (b < 31 && (int64_t(1) << b) < n) b++;
    return b;
}

// f(t) on threads t = 0 .. nt-1 (the calling thread runs t = 0).
template <class F>
void run_threads(unsigned nt, F f) {
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; t++) th.emplace_back(f, t);
    f(0u);
    for (auto &x : th) x.join();
}

// Argument and edge checks shared by pm_load_graph and pm_prepare_csr.
pm_status check_input(const char *who, int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst) {
    if (n < 1 || n > INT32_MAX || m_raw < 0 || (m_raw > 0 && (!src || !dst))) {
        set_error(std::string(who) + ": invalid argument");
        return PM_EINVAL;
    }
    for (int64_t i = 0; i < m_raw; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) {
            set_error(std::string(who) + ": edge " + std::to_string(i) + " has a vertex id outside [0, n)");
            return PM_EINVAL;
        }
    }
    return PM_OK;
}

// The host CSR of a prepared graph: rows in internal ids, each sorted, and
// the task offsets of the three task spaces.
struct HostCsr {
    std::vector<int64_t> rowptr;
    std::unique_ptr<int32_t[]> col;
    int64_t nnz = 0;
    std::vector<int64_t> off[3];
};

// Steps 1-5 of graph preparation on checked input: fills the host fields of
// g (counts, new_id, lowdeg, labels, task totals) and h.  May throw
// std::bad_alloc.
pm_status prepare_host(const char *who, int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                       const uint8_t *labels, pm_graph *g, HostCsr &h) {
    g->n = n;
    g->labeled = labels != nullptr;
    // 1. bucket both directions by source, dropping self-loops: each
    //    thread counts its slice of the edges per vertex, the counts are
    //    scanned per vertex across threads, and each thread fills its own
    //    part of every row (no shared cursors: hub rows would serialise
    //    them); the order inside a row does not matter, rows are sorted next
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    while (nt > 1 && (m_raw < int64_t(nt) * 65536 ||
                      int64_t(nt) * n > std::min(m_raw, int64_t(1) << 25))) nt /= 2;   // counters <= edges
    const int64_t slice = (m_raw + nt - 1) / nt;
    auto tc = raw_array<int64_t>(size_t(nt) * size_t(n));   // thread t's counts, then cursors
    std::vector<int64_t> tloops(nt, 0);
    run_threads(nt, [&](unsigned t) {
        int64_t *c = tc.get() + size_t(t) * size_t(n);
        std::fill(c, c + n, int64_t(0));
        const int64_t b = int64_t(t) * slice, e = std::min(m_raw, b + slice);
        for (int64_t i = b; i < e; i++) {
            if (src[i] == dst[i]) { tloops[t]++; continue; }
            c[src[i]]++;
            c[dst[i]]++;
        }
    });
    int64_t loops = 0;
    for (unsigned t = 0; t < nt; t++) loops += tloops[t];
    std::vector<int64_t> rp(n + 1, 0);
    parallel_for(n, [&](int64_t v) {     // raw degree: the threads' counts summed
        int64_t d = 0;
        for (unsigned t = 0; t < nt; t++) d += tc[size_t(t) * size_t(n) + size_t(v)];
        rp[v + 1] = d;
    });
    for (int64_t v = 0; v < n; v++) rp[v + 1] += rp[v];
    auto adj = raw_array<int32_t>(size_t(rp[n]));   // every entry written by the fill
    {
        // per-thread write positions: thread t fills row v after the entries
        // of threads 0 .. t-1, so each row keeps the input order of its edges
        parallel_for(n, [&](int64_t v) {
            int64_t pos = rp[v];
            for (unsigned t = 0; t < nt; t++) {
                int64_t &c = tc[size_t(t) * size_t(n) + size_t(v)];
                const int64_t k = c;
                c = pos;
                pos += k;
            }
        });
        run_threads(nt, [&](unsigned t) {
            int64_t *c = tc.get() + size_t(t) * size_t(n);
            const int64_t b = int64_t(t) * slice, e = std::min(m_raw, b + slice);
            for (int64_t i = b; i < e; i++) {
                if (src[i] == dst[i]) continue;
                adj[c[src[i]]++] = dst[i];
                adj[c[dst[i]]++] = src[i];
            }
        });
    }
    // 2. sort and deduplicate each row
    std::vector<int64_t> deg(n);
    const int bits = id_bits(n);
    parallel_for(n, [&](int64_t v) {
        int32_t *b = adj.get() + rp[v], *e = adj.get() + rp[v + 1];
        sort_ids(b, e - b, bits);
        deg[v] = std::unique(b, e) - b;
    }, 256);
    int64_t nnz = 0, maxd = 0;
    for (int64_t v = 0; v < n; v++) { nnz += deg[v]; maxd = std::max(maxd, deg[v]); }
    g->m = nnz / 2;
    g->self_loops = loops;
    g->duplicates = (m_raw - loops) - g->m;
    g->max_degree = maxd;
    // 3. order by (degree, id): counting sort on degree, stable in id
    std::vector<int64_t> cnt(maxd + 2, 0);
    for (int64_t v = 0; v < n; v++) cnt[deg[v] + 1]++;
    for (int64_t d = 0; d <= maxd; d++) cnt[d + 1] += cnt[d];
    g->new_id.assign(n, 0);
    std::vector<int32_t> old_of(n);
    for (int64_t v = 0; v < n; v++) {
        int64_t r = cnt[deg[v]]++;
        g->new_id[v] = int32_t(r);
        old_of[r] = int32_t(v);
    }
    // 4. CSR in internal ids, rows sorted
    std::vector<int64_t> &rowptr = h.rowptr;
    rowptr.assign(n + 1, 0);
    for (int64_t r = 0; r < n; r++) rowptr[r + 1] = rowptr[r] + deg[old_of[r]];
    h.col = raw_array<int32_t>(size_t(nnz));   // every row written below
    int32_t *col = h.col.get();
    g->lowdeg.assign(n, 0);
    parallel_for(n, [&](int64_t i) {
        const int64_t r = n - 1 - i;   // the longest rows (highest ranks) first, spread over threads
        const int64_t v = old_of[r];
        int32_t *o = col + rowptr[r];
        const int64_t d = deg[v];
        for (int64_t j = 0; j < d; j++) o[j] = g->new_id[adj[rp[v] + j]];
        sort_ids(o, d, bits);
        g->lowdeg[r] = int32_t(std::lower_bound(o, o + d, int32_t(r)) - o);
    }, 64);
    if (labels) {
        g->labels.resize(n);
        for (int64_t r = 0; r < n; r++) g->labels[r] = labels[old_of[r]];
    }
    // 5. task offsets for the implicit root list n-1, ..., 0, per task
    //    space: lower neighbours, higher neighbours, all neighbours
    std::vector<int64_t> *off = h.off;
    for (int sp = 0; sp < 3; sp++) off[sp].assign(n + 1, 0);
    for (int64_t i = 0; i < n; i++) {
        const int64_t r = n - 1 - i;
        const int64_t d = rowptr[r + 1] - rowptr[r];
        off[0][i + 1] = off[0][i] + g->lowdeg[r];
        off[1][i + 1] = off[1][i] + (d - g->lowdeg[r]);
        off[2][i + 1] = off[2][i] + d;
        g->max_updeg = std::max<int64_t>(g->max_updeg, d - g->lowdeg[r]);
    }
    for (int sp = 0; sp < 3; sp++) g->ntasks[sp] = off[sp][n];
    if (nnz >= (int64_t(1) << 32)) {
        set_error(std::string(who) + ": more than 2^32 - 1 adjacency entries");
        return PM_EUNSUPPORTED;
    }
    h.nnz = nnz;
    return PM_OK;
}

}  // namespace

pm_status build_graph(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                      const uint8_t *labels, int device, void *stream, pm_graph **out) {
    if (!out) {
        set_error("pm_load_graph: invalid argument");
        return PM_EINVAL;
    }
    pm_status st = check_input("pm_load_graph", n, m_raw, src, dst);
    if (st != PM_OK) return st;
    auto *g = new (std::nothrow) pm_graph();
    if (!g) return PM_ENOMEM;
    g->device = device;
    try {
        HostCsr h;
        st = prepare_host("pm_load_graph", n, m_raw, src, dst, labels, g, h);
        if (st != PM_OK) {
            delete g;
            return st;
        }
        const std::vector<int64_t> &rowptr = h.rowptr;
        const int32_t *col = h.col.get();
        const int64_t nnz = h.nnz;
        const std::vector<int64_t> *off = h.off;

        // 6. upload
        int prev = 0;
        cudaGetDevice(&prev);
        if (cudaSetDevice(device) != cudaSuccess) {
            set_error("pm_load_graph: cudaSetDevice failed");
            delete g;
            return PM_ECUDA;
        }
        cudaStream_t s = (cudaStream_t)stream;
        const size_t b_rp = sizeof(int64_t) * (n + 1), b_col = sizeof(int32_t) * std::max<int64_t>(nnz, 1);
        g->d_rowptr = (int64_t *)dev_alloc(b_rp, device);
        g->d_col = (int32_t *)dev_alloc(b_col, device);
        for (int sp = 0; sp < 3; sp++) g->d_off[sp] = (int64_t *)dev_alloc(b_rp, device);
        if (labels) g->d_labels = (uint8_t *)dev_alloc(n, device);
        if (!g->d_rowptr || !g->d_col || !g->d_off[0] || !g->d_off[1] || !g->d_off[2] ||
            (labels && !g->d_labels)) {
            set_error("pm_load_graph: device allocation failed");
            pm_free_graph(g);
            cudaSetDevice(prev);
            return PM_ENOMEM;
        }
        g->bytes = 4 * b_rp + b_col + (labels ? n : 0);
        cudaError_t e1 = cudaMemcpyAsync(g->d_rowptr, rowptr.data(), b_rp, cudaMemcpyHostToDevice, s);
        cudaError_t e2 = nnz ? cudaMemcpyAsync(g->d_col, col, sizeof(int32_t) * nnz,
                                               cudaMemcpyHostToDevice, s) : cudaSuccess;
        cudaError_t e3 = cudaSuccess;
        for (int sp = 0; sp < 3 && !e3; sp++)
            e3 = cudaMemcpyAsync(g->d_off[sp], off[sp].data(), b_rp, cudaMemcpyHostToDevice, s);
        cudaError_t e4 = labels ? cudaMemcpyAsync(g->d_labels, g->labels.data(), n,
                                                  cudaMemcpyHostToDevice, s) : cudaSuccess;
        // 7. adjacency bitmaps for the highest-degree vertices: every vertex of
        //    degree >= PM_HUB_MIN_DEGREE (environment, default 1024), highest
        //    first, within 256 MiB of bitmaps; built on the device from the
        //    uploaded CSR, behind the copies on the same stream
        cudaError_t e6 = cudaSuccess;
        if (!(e1 || e2 || e3 || e4)) {
            int64_t min_degree = 1024;
            if (const char *env = std::getenv("PM_HUB_MIN_DEGREE")) min_degree = std::max(1L, std::atol(env));
            const int64_t words = (n + 31) / 32;
            const int64_t cap = std::max<int64_t>(0, (int64_t(256) << 20) / (4 * words));
            int64_t nh = 0;
            for (int64_t r = n - 1; r >= 0 && nh < cap; r--) {
                if (rowptr[r + 1] - rowptr[r] < min_degree) break;   // ids ascend by degree
                nh++;
            }
            if (nh > 0) {
                const size_t n_bits = size_t(nh) * size_t(words);
                g->d_hub = (int32_t *)dev_alloc(sizeof(int32_t) * n, device);
                g->d_bits = (uint32_t *)dev_alloc(sizeof(uint32_t) * n_bits, device);
                if (!g->d_hub || !g->d_bits) {
                    cudaStreamSynchronize(s);   // the copies read host buffers of this frame
                    set_error("pm_load_graph: device allocation failed (hub bitmaps)");
                    pm_free_graph(g);
                    cudaSetDevice(prev);
                    return PM_ENOMEM;
                }
                g->n_hubs = nh;
                g->hub_words = words;
                g->bytes += sizeof(int32_t) * n + sizeof(uint32_t) * n_bits;
                e6 = cudaError_t(launch_hub_bitmaps(g->d_rowptr, g->d_col, n, nh, words, g->d_hub, g->d_bits, s));
            }
        }
        cudaError_t e5 = cudaStreamSynchronize(s);
        cudaSetDevice(prev);
        if (e1 || e2 || e3 || e4 || e5 || e6) {
            const cudaError_t first = e1 ? e1 : e2 ? e2 : e3 ? e3 : e4 ? e4 : e6 ? e6 : e5;
            set_error(std::string("pm_load_graph: upload failed: ") + cudaGetErrorString(first));
            pm_free_graph(g);
            return PM_ECUDA;
        }
    } catch (const std::bad_alloc &) {
        set_error("pm_load_graph: host allocation failed");
        pm_free_graph(g);
        return PM_ENOMEM;
    }
    *out = g;
    return PM_OK;
}

pm_status prepare_csr(int64_t n, int64_t m_raw, const int32_t *src, const int32_t *dst,
                      int64_t *rowptr, int32_t *col, int32_t *new_id, int64_t *lowdeg) {
    if (!rowptr || !col) {
        set_error("pm_prepare_csr: invalid argument");
        return PM_EINVAL;
    }
    pm_status st = check_input("pm_prepare_csr", n, m_raw, src, dst);
    if (st != PM_OK) return st;
    try {
        pm_graph g;   // host fields only: nothing on a device
        HostCsr h;
        st = prepare_host("pm_prepare_csr", n, m_raw, src, dst, nullptr, &g, h);
        if (st != PM_OK) return st;
        std::copy(h.rowptr.begin(), h.rowptr.end(), rowptr);
        std::copy(h.col.get(), h.col.get() + h.nnz, col);
        if (new_id) std::copy(g.new_id.begin(), g.new_id.end(), new_id);
        if (lowdeg) std::copy(g.lowdeg.begin(), g.lowdeg.end(), lowdeg);
    } catch (const std::bad_alloc &) {
        set_error("pm_prepare_csr: host allocation failed");
        return PM_ENOMEM;
    }
    return PM_OK;
}

}  // namespace pm
