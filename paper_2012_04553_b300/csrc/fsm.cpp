// Frequent subgraph mining with MNI support (Section 2, "Frequent Subgraph
// Mining"): level-wise over the number of edges.  Level 1 holds every labeled
// edge whose labels occur in the graph; level j+1 holds the connected labeled
// patterns obtained by adding one edge (between two existing vertices, or to
// a new vertex of any present label) to a frequent level-j pattern and whose
// every connected one-edge-smaller subpattern is frequent.  MNI support is
// anti-monotone (a pattern's support never exceeds a subpattern's), so the
// pruning loses no frequent pattern.  Each level's candidates are planned and
// counted with pm_plan / pm_support, so the level's MNI domains come from the
// GPU and, when morphing is enabled, from vertex-induced superpatterns
// (Theorem 3.2).
#include <algorithm>
#include <map>
#include <set>
#include <vector>

#include "internal.hpp"

namespace pm {

namespace {

// Connected subpatterns with one edge fewer (an endpoint left isolated is dropped).
std::vector<Pat> one_edge_smaller(const Pat &p) {
    std::vector<Pat> out;
    for (int a = 0; a < p.k; a++)
        for (int b = a + 1; b < p.k; b++) {
            if (!p.adjacent(a, b)) continue;
            Pat q = p;
            q.adj[a] &= uint8_t(~(1u << b));
            q.adj[b] &= uint8_t(~(1u << a));
            if (q.n_edges() == 0) continue;
            // drop isolated vertices
            std::vector<int> keep;
            for (int v = 0; v < q.k; v++)
                if (q.adj[v]) keep.push_back(v);
            Pat r;
            r.k = int(keep.size());
            r.vi = false;
            for (int i = 0; i < r.k; i++) {
                r.lab[i] = q.lab[keep[i]];
                for (int j = 0; j < r.k; j++)
                    if (q.adjacent(keep[i], keep[j])) r.adj[i] |= uint8_t(1u << j);
            }
            if (r.connected()) out.push_back(r);
        }
    return out;
}

pm_pattern to_abi(const Pat &q) {
    pm_pattern r{};
    r.k = q.k;
    r.edge_mask = q.mask();
    for (int u = 0; u < PM_MAX_K; u++) r.label[u] = u < q.k ? q.lab[u] : -1;
    r.induced = PM_EDGE_INDUCED;
    return r;
}

}  // namespace

}  // namespace pm

using namespace pm;

extern "C" pm_status pm_fsm(const pm_graph *g, int32_t max_edges, uint64_t threshold,
                            pm_morph_mode mode, void *stream, double timeout_s,
                            pm_pattern *out, uint64_t *support, uint8_t *frequent, int32_t cap,
                            int32_t *n_out) {
    if (!g || !n_out || max_edges < 1 || max_edges > 5 || cap < 0 ||
        (cap > 0 && (!out || !support))) {
        set_error("pm_fsm: bad argument (max_edges must be 1..5)");
        return PM_EINVAL;
    }
    if (!g->labeled) {
        set_error("pm_fsm: the graph has no vertex labels");
        return PM_EINVAL;
    }
    std::vector<int8_t> labels;
    {
        std::set<int> present(g->labels.begin(), g->labels.end());
        for (int l : present)
            if (l <= 127) labels.push_back(int8_t(l));
    }
    std::vector<Pat> cand;
    for (size_t i = 0; i < labels.size(); i++)
        for (size_t j = i; j < labels.size(); j++) {
            Pat p;
            p.k = 2;
            p.add_edge(0, 1);
            p.lab[0] = labels[i];
            p.lab[1] = labels[j];
            cand.push_back(p);
        }
    std::vector<std::pair<Pat, uint64_t>> results;
    std::vector<uint8_t> flags;
    for (int level = 1; level <= max_edges && !cand.empty(); level++) {
        std::vector<pm_pattern> q;
        for (const Pat &p : cand) q.push_back(to_abi(p));
        pm_query_plan *plan = nullptr;
        pm_status st = pm_plan(g, q.data(), int32_t(q.size()), PM_OP_SUPPORT, mode, &plan);
        if (st != PM_OK) return st;
        std::vector<uint64_t> sup(q.size());
        std::vector<uint8_t> fr(q.size());
        st = pm_support(plan, stream, timeout_s, threshold, sup.data(), fr.data(), nullptr);
        pm_free_plan(plan);
        if (st != PM_OK) return st;
        std::set<Key> frequent_keys;
        std::vector<Pat> freq;
        for (size_t i = 0; i < cand.size(); i++) {
            results.push_back({cand[i], sup[i]});
            flags.push_back(fr[i]);
            if (fr[i]) {
                frequent_keys.insert(canonical(cand[i]));
                freq.push_back(cand[i]);
            }
        }
        if (level == max_edges) break;
        // extend every frequent pattern by one edge, then prune
        std::map<Key, Pat> next;
        for (const Pat &f : freq) {
            for (int a = 0; a < f.k; a++)
                for (int b = a + 1; b < f.k; b++) {
                    if (f.adjacent(a, b)) continue;
                    Pat c = f;
                    c.add_edge(a, b);
                    next.emplace(canonical(c), c);
                }
            if (f.k < 6) {
                for (int a = 0; a < f.k; a++)
                    for (int8_t l : labels) {
                        Pat c = f;
                        c.k = f.k + 1;
                        c.lab[f.k] = l;
                        c.add_edge(a, f.k);
                        next.emplace(canonical(c), c);
                    }
            }
        }
        cand.clear();
        for (auto &kv : next) {
            bool ok = true;
            for (const Pat &s : one_edge_smaller(kv.second))
                if (!frequent_keys.count(canonical(s))) { ok = false; break; }
            if (ok) cand.push_back(kv.second);
        }
    }
    *n_out = int32_t(results.size());
    if (int64_t(results.size()) > cap) {
        set_error("pm_fsm: output capacity too small (n_out holds the size needed)");
        return PM_EOVERFLOW;
    }
    for (size_t i = 0; i < results.size(); i++) {
        out[i] = to_abi(results[i].first);
        support[i] = results[i].second;
        if (frequent) frequent[i] = flags[i];
    }
    return PM_OK;
}
