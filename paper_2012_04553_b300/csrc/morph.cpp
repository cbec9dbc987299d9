// Morph selection, morph transform coefficients and matching-plan compilation.
//
// Counting (sum aggregation, permute operator = identity, Section 3.2.3):
//  * an edge-induced query p^E becomes its vertex-induced superpatterns
//    (Theorem 3.1): count(p^E) = sum_q c(p, q) count(q^V), q = p included;
//  * a vertex-induced query p^V becomes edge-induced superpatterns.  Applying
//    Corollary 3.1 recursively until only cliques remain gives, in closed
//    form, count(p^V) = sum_q (-1)^(e(q) - e(p)) c(p, q) count(q^E): the
//    signed coefficients are the Moebius function of the "spanning copy"
//    order, the inverse of the Theorem 3.1 matrix.
// MNI (union aggregation, permute operator = column permutation): only the
// edge-from-vertex direction exists (a union has no inverse, Section 3.2.3):
//  D_{p^E}[u] = D_{p^V}[u]  u  U_q U_{f in phi(p^E, q^E)} D_{q^V}[f(u)].
#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <numeric>
#include <string>

#include "internal.hpp"

namespace pm {

namespace {

struct MatchedSet {
    std::map<Key, int> index;
    std::vector<Pat> pats;
    int add(const Pat &p) {
        Pat c = canonical_form(p);
        Key key = canonical(c);
        auto it = index.find(key);
        if (it != index.end()) return it->second;
        int id = int(pats.size());
        index[key] = id;
        pats.push_back(c);
        return id;
    }
};

// superpatterns() of an edge-induced pattern depends only on its class, so
// the result is cached by canonical key (serving re-plans the same patterns
// for every batch).
std::mutex g_super_mu;
std::map<Key, std::vector<Super>> g_super_cache;

std::vector<Super> cached_superpatterns(const Pat &pe) {
    const Key key = canonical(pe);
    {
        std::lock_guard<std::mutex> lk(g_super_mu);
        auto it = g_super_cache.find(key);
        if (it != g_super_cache.end()) return it->second;
    }
    std::vector<Super> v = superpatterns(pe);
    std::lock_guard<std::mutex> lk(g_super_mu);
    g_super_cache.emplace(key, v);
    return v;
}

// Column (orbit index, orbits numbered by smallest member) of every vertex.
std::vector<int> columns_of(const Pat &p, int *n_columns) {
    std::vector<Perm> aut = automorphisms(p);
    std::vector<int> orb = orbit_of(p, aut);
    std::vector<int> col(p.k, -1), rep_col(p.k, -1);
    int nc = 0;
    for (int u = 0; u < p.k; u++) {
        if (rep_col[orb[u]] < 0) rep_col[orb[u]] = nc++;
        col[u] = rep_col[orb[u]];
    }
    if (n_columns) *n_columns = nc;
    return col;
}

}  // namespace

// For every query column, the matched bitsets (matched pattern, column)
// whose union is the column's MNI domain (Theorem 3.2).
void fill_mni_sources(MorphPlan &out) {
    const std::vector<Pat> &queries = out.queries;
    {
        out.mni_sources.assign(queries.size(), {});
        out.query_columns.assign(queries.size(), {});
        for (size_t i = 0; i < queries.size(); i++) {
            Pat p = queries[i];
            if (p.is_clique()) p.vi = false;
            int nqc = 0;
            std::vector<int> qcol = columns_of(p, &nqc);
            out.query_columns[i] = qcol;
            out.mni_sources[i].assign(nqc, {});
            std::vector<int> rep(nqc, -1);
            for (int u = 0; u < p.k; u++)
                if (rep[qcol[u]] < 0) rep[qcol[u]] = u;
            // Every matched pattern this query draws on, with the maps phi(p^E, q^E)
            Pat pe = p;
            pe.vi = false;
            for (const Term &t : out.terms[i]) {
                const Pat &q = out.matched[t.matched];
                Pat qe = q;
                qe.vi = false;
                std::vector<Perm> fs = (q.vi || q.is_clique()) && !p.vi ? embeddings(pe, qe)
                                                                         : embeddings(p, q);
                for (int c = 0; c < nqc; c++) {
                    auto &dst = out.mni_sources[i][c];
                    for (const Perm &f : fs) {
                        std::pair<int, int> src{t.matched, out.matched_orbit[t.matched][f[rep[c]]]};
                        if (std::find(dst.begin(), dst.end(), src) == dst.end()) dst.push_back(src);
                    }
                }
            }
        }
    }
}

namespace {

// Cost-based selection (Section 4.1, "pattern morphing optimizer").  A
// count is "known" as a signed combination of matched patterns.  For a
// vertex-induced count there are two ways: match p^V, or match p^E and
// subtract c(p, q) * (known vertex-induced count) for every non-isomorphic
// superpattern q (Corollary 3.1, applied recursively).  For an edge-induced
// count: match p^E, or add c(p, q) * (known vertex-induced count) over all
// superpatterns q, p included (Theorem 3.1).  MNI has no subtraction
// (Section 3.2.3), so its vertex-induced domains are always matched
// directly.  Each choice minimises the summed cost of the patterns it adds
// to those already selected (patterns shared between queries cost once).
struct CostSelector {
    pm_op op;
    const std::function<double(const Pat &)> &cost;
    std::map<Key, double> cost_memo;
    std::set<Key> selected;                                  // patterns committed so far
    std::map<Key, Pat> pats;
    std::map<Key, std::map<Key, int64_t>> known_v;           // memo: combination per pattern class

    double c(const Pat &q) {
        const Key k = canonical(q);
        auto it = cost_memo.find(k);
        if (it != cost_memo.end()) return it->second;
        const double v = cost(q);
        cost_memo[k] = v;
        return v;
    }
    static void add(std::map<Key, int64_t> &acc, const std::map<Key, int64_t> &x, int64_t f) {
        for (auto &kv : x) acc[kv.first] += f * kv.second;
    }
    // cost of the patterns of a combination that are not selected yet
    double marginal(const std::map<Key, int64_t> &combo) {
        double t = 0;
        for (auto &kv : combo)
            if (kv.second != 0 && !selected.count(kv.first)) t += c(pats[kv.first]);
        return t;
    }
    std::map<Key, int64_t> single(const Pat &q) {
        Pat n = canonical_form(q);
        const Key k = canonical(n);
        pats[k] = n;
        return {{k, 1}};
    }
    std::map<Key, int64_t> vertex_induced(const Pat &p) {
        Pat pv = p;
        pv.vi = !p.is_clique();
        const Key key = canonical(pv);
        auto it = known_v.find(key);
        if (it != known_v.end()) return it->second;
        std::map<Key, int64_t> direct = single(pv);
        std::map<Key, int64_t> best = direct;
        if (!p.is_clique() && op == PM_OP_COUNT) {
            Pat pe = p;
            pe.vi = false;
            std::map<Key, int64_t> via = single(pe);
            for (const Super &s : cached_superpatterns(pe)) {
                if (canonical(s.q) == key) continue;          // p itself
                add(via, vertex_induced(s.q), -s.coef);
            }
            if (marginal(via) < marginal(direct)) best = via;
        }
        known_v[key] = best;
        return best;
    }
    std::map<Key, int64_t> edge_induced(const Pat &p) {
        Pat pe = p;
        pe.vi = false;
        std::map<Key, int64_t> direct = single(pe);
        if (p.is_clique()) return direct;
        std::map<Key, int64_t> via;
        for (const Super &s : cached_superpatterns(pe)) add(via, vertex_induced(s.q), s.coef);
        return marginal(via) < marginal(direct) ? via : direct;
    }
    void commit(const std::map<Key, int64_t> &combo) {
        for (auto &kv : combo)
            if (kv.second != 0) selected.insert(kv.first);
    }
};

}  // namespace

pm_status morph_select(const std::vector<Pat> &queries, pm_op op, pm_morph_mode mode,
                       MorphPlan &out, std::string *why,
                       const std::function<double(const Pat &)> *cost) {
    if (mode == PM_MORPH_COST) {
        if (!cost) {
            if (why) *why = "cost-based morph selection needs a graph to measure costs on";
            return PM_EINVAL;
        }
        CostSelector sel{op, *cost};
        MatchedSet ms;
        out.queries = queries;
        out.terms.assign(queries.size(), {});
        for (size_t i = 0; i < queries.size(); i++) {
            Pat p = queries[i];
            if (p.is_clique()) p.vi = false;
            std::map<Key, int64_t> combo = p.vi ? sel.vertex_induced(p) : sel.edge_induced(p);
            sel.commit(combo);
            for (auto &kv : combo)
                if (kv.second != 0) out.terms[i].push_back({ms.add(sel.pats[kv.first]), kv.second});
        }
        out.matched = ms.pats;
        out.matched_columns.assign(out.matched.size(), 0);
        out.matched_orbit.assign(out.matched.size(), {});
        for (size_t j = 0; j < out.matched.size(); j++)
            out.matched_orbit[j] = columns_of(out.matched[j], &out.matched_columns[j]);
        if (op == PM_OP_SUPPORT) fill_mni_sources(out);
        return PM_OK;
    }
    MatchedSet ms;
    out.queries = queries;
    out.terms.assign(queries.size(), {});
    std::vector<std::vector<std::pair<int, std::vector<int>>>> mni_raw(queries.size());
    // mni_raw[query] = list of (matched id, f-image of each query column rep)
    for (size_t i = 0; i < queries.size(); i++) {
        Pat p = queries[i];
        if (p.is_clique()) p.vi = false;
        bool morph = (mode == PM_MORPH_NAIVE) && !p.is_clique();
        if (op == PM_OP_SUPPORT && p.vi) morph = false;   // no vertex-from-edge MNI rule
        if (!morph) {
            int id = ms.add(p);
            out.terms[i].push_back({id, 1});
            continue;
        }
        const int e_p = p.n_edges();
        Pat pe = p;
        pe.vi = false;
        for (const Super &s : cached_superpatterns(pe)) {
            if (!p.vi) {
                // Theorem 3.1: p^E from vertex-induced superpatterns
                Pat q = s.q;
                q.vi = !q.is_clique();
                int id = ms.add(q);
                out.terms[i].push_back({id, s.coef});
            } else {
                // Corollary 3.1, recursively: p^V from edge-induced superpatterns
                Pat q = s.q;
                q.vi = false;
                int id = ms.add(q);
                int64_t sign = ((q.n_edges() - e_p) & 1) ? -1 : 1;
                out.terms[i].push_back({id, sign * s.coef});
            }
        }
    }
    out.matched = ms.pats;
    // Merge repeated terms.
    for (auto &t : out.terms) {
        std::map<int, int64_t> acc;
        for (const Term &x : t) acc[x.matched] += x.coef;
        t.clear();
        for (auto &kv : acc)
            if (kv.second != 0) t.push_back({kv.first, kv.second});
    }
    out.matched_columns.assign(out.matched.size(), 0);
    out.matched_orbit.assign(out.matched.size(), {});
    for (size_t j = 0; j < out.matched.size(); j++)
        out.matched_orbit[j] = columns_of(out.matched[j], &out.matched_columns[j]);

    if (op == PM_OP_SUPPORT) fill_mni_sources(out);
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Plan compilation.

namespace {

// Visiting order from the root: repeatedly the unvisited vertex with the most
// edges into the visited set, then most anti-edges (vertex-induced), then
// highest pattern degree, then smallest id.
std::vector<int> matching_order(const Pat &p, int root) {
    std::vector<int> order{root};
    uint32_t visited = 1u << root;
    while (int(order.size()) < p.k) {
        int best = -1;
        int bs[3] = {-1, -1, -1};
        for (int w = 0; w < p.k; w++) {
            if ((visited >> w) & 1) continue;
            int e = __builtin_popcount(p.adj[w] & visited);
            if (e == 0) continue;
            int a = p.vi ? __builtin_popcount(~p.adj[w] & visited & ~(1u << w)) : 0;
            int d = __builtin_popcount(p.adj[w]);
            int s[3] = {e, a, d};
            if (best < 0 || std::lexicographical_compare(bs, bs + 3, s, s + 3)) {
                best = w;
                std::copy(s, s + 3, bs);
            }
        }
        order.push_back(best);
        visited |= 1u << best;
    }
    return order;
}

bool same_common(const DevLevel &a, const DevLevel &b, uint8_t tail_bits) {
    return a.isect == b.isect && a.diff == b.diff && a.lt == b.lt && a.neq == b.neq &&
           a.label == b.label && (a.gt & ~tail_bits) == (b.gt & ~tail_bits);
}

}  // namespace

// One plan: `order[0]` is the root; `H` is the group whose symmetry the
// ordering constraints break (the root's stabiliser for rooted plans, the
// whole automorphism group for free plans); rooted plans bound every vertex
// below the root.
static DevPlan build_plan(const Pat &p, const std::vector<int> &order, std::vector<Perm> H,
                          bool rooted, int counter, int dom_base,
                          const std::vector<int> &column_of_vertex, bool counting) {
    int n_columns = 0;
    for (int c : column_of_vertex) n_columns = std::max(n_columns, c + 1);
    std::vector<int> level_of(p.k);
    for (int i = 0; i < p.k; i++) level_of[order[i]] = i;
    DevPlan plan{};
    plan.k = p.k;
    plan.counter = counter;
    plan.dom_base = dom_base;
    plan.n_columns = n_columns;
    for (int i = 0; i < p.k; i++) {
        int u = order[i];
        DevLevel &lv = plan.lv[i];
        lv.vertex = uint8_t(u);
        lv.label = p.lab[u];
        lv.column = uint8_t(column_of_vertex.empty() ? 0 : column_of_vertex[u]);
        if (i == 0) continue;
        if (rooted) lv.lt = 1;   // every non-root vertex ranks below the root
        for (int j = 0; j < i; j++) {
            int w = order[j];
            if (p.adjacent(u, w)) lv.isect |= uint8_t(1u << j);
            else if (p.vi) lv.diff |= uint8_t(1u << j);
        }
    }
    // Symmetry breaking (Grochow & Kellis): in matching order, v's image is
    // the smallest over v's orbit under H, then H shrinks to v's stabiliser.
    for (int i = rooted ? 1 : 0; i < p.k; i++) {
        int v = order[i];
        uint32_t orbit = 0;
        for (const Perm &s : H) orbit |= 1u << s[v];
        for (int w = 0; w < p.k; w++) {
            if (w == v || !((orbit >> w) & 1)) continue;
            // image of v below image of w; w comes later in the order
            plan.lv[level_of[w]].gt |= uint8_t(1u << i);
        }
        std::vector<Perm> H2;
        for (const Perm &s : H)
            if (s[v] == v) H2.push_back(s);
        H.swap(H2);
    }
    // Injectivity not implied by adjacency or ordering.
    for (int i = 1; i < p.k; i++) {
        DevLevel &lv = plan.lv[i];
        uint8_t implied = lv.isect | lv.lt | lv.gt;
        for (int j = 0; j < i; j++)
            if (!((implied >> j) & 1)) lv.neq |= uint8_t(1u << j);
    }
    // Longest totally ordered tail with one shared candidate set.
    int tail = 0;
    if (p.k >= 3) {
        tail = 1;
        for (int r = p.k - 2; r >= 2; r--) {
            int t0 = p.k - r;
            uint8_t tail_bits = uint8_t(((1u << p.k) - 1) & ~((1u << t0) - 1));
            bool ok = true;
            for (int t = t0; t < p.k && ok; t++) {
                const DevLevel &lv = plan.lv[t];
                if (!same_common(lv, plan.lv[t0], tail_bits)) ok = false;
                if ((lv.isect | lv.diff | lv.lt | lv.neq) & tail_bits) ok = false;
                uint8_t before = uint8_t(((1u << t) - 1) & tail_bits);
                if ((lv.gt & tail_bits) != before) ok = false;
            }
            if (ok) { tail = r; break; }
        }
    }
    plan.tail = tail;
    plan.n_enum = p.k - tail;
    const DevLevel &f = plan.lv[plan.n_enum < p.k ? plan.n_enum : p.k - 1];
    plan.closed = tail > 0 && __builtin_popcount(f.isect) == 1 && f.diff == 0 && f.label < 0;
    // Independent pair of closed leaves at the end (counting plans only).
    if (counting && tail == 1 && p.k >= 4 && p.k < PLAN_KMAX) {
        const int L1 = p.k - 2, L2 = p.k - 1;
        const DevLevel &a = plan.lv[L1], &b = plan.lv[L2];
        const uint8_t bit1 = uint8_t(1u << L1);
        auto closed_level = [](const DevLevel &x) {
            return __builtin_popcount(x.isect) == 1 && x.diff == 0 && x.label < 0;
        };
        if (closed_level(a) && closed_level(b) && !((b.isect | b.diff | b.lt | b.gt) & bit1)) {
            DevLevel B = b;
            B.neq &= uint8_t(~bit1);
            DevLevel M{};
            M.isect = a.isect | B.isect;
            M.lt = a.lt | B.lt;
            M.gt = a.gt | B.gt;
            M.neq = uint8_t((a.neq | B.neq) & ~(a.isect | B.isect | M.lt | M.gt));
            M.label = -1;
            plan.lv[L2] = B;
            plan.lv[p.k] = M;
            plan.pair = 1;
            plan.tail = 2;
            plan.n_enum = p.k - 2;
            plan.closed = 1;
        }
    }
    // second-level candidates per chunk before the rest is deferred: deeper
    // plans do more work per candidate, so they split finer
    plan.split = plan.n_enum <= 2 ? 4096 : std::max(32, 1024 >> (2 * (plan.n_enum - 3)));
    // task space: rooted plans take (root, lower neighbour); free plans take
    // (root, higher neighbour) when symmetry orders them, else both directions
    if (rooted) plan.task_space = TASKS_LOWER;
    else plan.task_space = (plan.lv[1].gt & 1) ? TASKS_UPPER : TASKS_BOTH;
    return plan;
}

// Unlabeled edge-induced 4-cycle: every vertex of degree 2, four edges.
static bool is_plain_c4(const Pat &p) {
    if (p.k != 4 || p.vi || p.labeled() || p.n_edges() != 4) return false;
    for (int u = 0; u < 4; u++)
        if (__builtin_popcount(p.adj[u]) != 2) return false;
    return true;
}

std::vector<DevPlan> compile_plans(const Pat &p, int counter, int dom_base,
                                   const std::vector<int> &column_of_vertex, bool counting) {
    std::vector<Perm> aut = automorphisms(p);
    std::vector<int> orb = orbit_of(p, aut);
    std::vector<DevPlan> plans;
    for (int root = 0; root < p.k; root++) {
        if (orb[root] != root) continue;   // one plan per orbit, at its smallest vertex
        std::vector<Perm> H;
        for (const Perm &s : aut)
            if (s[root] == root) H.push_back(s);
        plans.push_back(build_plan(p, matching_order(p, root), H, true, counter, dom_base,
                                   column_of_vertex, counting));
    }
    // the 4-cycle's single rooted plan is counted by the wedge kernel (its
    // levels still describe the same occurrences: root, two lower neighbours
    // and the opposite vertex)
    if (counting && is_plain_c4(p) && plans.size() == 1) plans[0].kind = PLAN_WEDGE_PAIRS;
    // the unlabeled 4- and 5-clique's single rooted plan runs in the clique kernel
    if (counting && (p.k == 4 || p.k == 5) && p.is_clique() && !p.labeled() && plans.size() == 1)
        plans[0].kind = PLAN_CLIQUE;
    return plans;
}

DevPlan compile_free_plan(const Pat &p, int counter, int dom_base,
                          const std::vector<int> &column_of_vertex, bool counting) {
    // root at a vertex of highest pattern degree (most intersections early)
    int root = 0;
    for (int u = 1; u < p.k; u++)
        if (__builtin_popcount(p.adj[u]) > __builtin_popcount(p.adj[root])) root = u;
    return build_plan(p, matching_order(p, root), automorphisms(p), false, counter, dom_base,
                      column_of_vertex, counting);
}

// Patterns whose edge-induced count the decomposition kernels produce
// (decomp.cu), by canonical class: the representative edge masks in
// lexicographic pair order.
int decomp_formula(const Pat &p) {
    if ((p.vi && !p.is_clique()) || p.labeled() || (p.k != 4 && p.k != 5)) return -1;
    // (a clique's edge- and vertex-induced counts coincide)
    static const std::map<Key, int> table = [] {
        const int8_t none[KMAX] = {-1, -1, -1, -1, -1, -1, -1, -1};
        const struct { int k; uint32_t mask; int f; } rows[] = {
            {4, 7, DF_STAR3}, {4, 13, DF_P4}, {4, 15, DF_PAW}, {4, 31, DF_DIAMOND},
            {5, 15, DF_STAR4}, {5, 29, DF_FORK}, {5, 58, DF_P5}, {5, 31, DF_CRICKET},
            {5, 59, DF_BULL}, {5, 185, DF_LOLLIPOP}, {5, 62, DF_BANNER}, {5, 220, DF_C5},
            {5, 63, DF_KITE}, {5, 187, DF_DART}, {5, 207, DF_BOWTIE}, {5, 221, DF_HOUSE},
            {5, 127, DF_BOOK}, {5, 223, DF_GEM}, {5, 191, DF_K4PENDANT},
            {4, 63, DF_K4}, {5, 1023, DF_K5}, {5, 255, DF_K5P3},
            {5, 495, DF_W4}, {5, 126, DF_K23}, {5, 254, DF_K23E}, {5, 511, DF_K5E}};
        std::map<Key, int> m;
        for (const auto &r : rows) m[canonical(Pat::from_mask(r.k, r.mask, none, false))] = r.f;
        return m;
    }();
    Pat q = p;
    q.vi = false;
    auto it = table.find(canonical(q));
    return it == table.end() ? -1 : it->second;
}

int decomp_passes(int f) {
    switch (f) {
        case DF_P5: case DF_BANNER: case DF_HOUSE: return DP_PATHS;
        case DF_C5: return DP_PATHS | DP_C5;
        case DF_DART: case DF_GEM: return DP_TRI2 | DP_LOCAL;
        case DF_K4: return DP_LOCAL;
        case DF_K5: return DP_LOCAL | DP_K5;
        case DF_K4PENDANT: case DF_K5P3: return DP_LOCAL | DP_K4E;
        case DF_W4: return DP_W4;
        case DF_K23: case DF_K23E: return DP_K23E;
        case DF_K5E: return DP_K5E;
        default: return 0;
    }
}

}  // namespace pm
