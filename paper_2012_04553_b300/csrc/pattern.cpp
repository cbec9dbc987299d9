// Pattern algebra (see pattern.hpp).  Automorphisms and embeddings are found
// by backtracking over vertex images with adjacency, label and degree
// pruning; canonical forms take the least (labels, edge mask) over the
// relabelings that order vertices by an isomorphism invariant (k <= 8).
#include "pattern.hpp"

#include <algorithm>
#include <map>
#include <numeric>

namespace pm {

int Pat::n_edges() const {
    int e = 0;
    for (int v = 0; v < k; v++) e += __builtin_popcount(adj[v]);
    return e / 2;
}

bool Pat::connected() const {
    if (k == 0) return false;
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
        uint32_t next = 0;
        for (int v = 0; v < k; v++)
            if ((frontier >> v) & 1) next |= adj[v];
        next &= ~seen;
        seen |= next;
        frontier = next;
    }
    return seen == (1u << k) - 1;
}

bool Pat::labeled() const {
    for (int v = 0; v < k; v++)
        if (lab[v] >= 0) return true;
    return false;
}

uint32_t Pat::mask() const {
    uint32_t m = 0;
    int bit = 0;
    for (int a = 0; a < k; a++)
        for (int b = a + 1; b < k; b++, bit++)
            if (adjacent(a, b)) m |= 1u << bit;
    return m;
}

Pat Pat::from_mask(int k, uint32_t mask, const int8_t *lab, bool vi) {
    Pat p;
    p.k = k;
    p.vi = vi;
    int bit = 0;
    for (int a = 0; a < k; a++)
        for (int b = a + 1; b < k; b++, bit++)
            if ((mask >> bit) & 1) p.add_edge(a, b);
    for (int v = 0; v < k; v++) p.lab[v] = lab ? lab[v] : -1;
    return p;
}

// Apply relabeling perm (perm[u] = new name of u).
static Pat relabel(const Pat &p, const Perm &perm) {
    Pat q;
    q.k = p.k;
    q.vi = p.vi;
    for (int u = 0; u < p.k; u++) {
        q.lab[perm[u]] = p.lab[u];
        for (int w = u + 1; w < p.k; w++)
            if (p.adjacent(u, w)) q.add_edge(perm[u], perm[w]);
    }
    return q;
}

static uint64_t pack_labels(const Pat &p) {
    uint64_t x = 0;
    for (int v = 0; v < p.k; v++) x = (x << 8) | uint8_t(p.lab[v] + 1);
    return x;
}

// Vertex invariant for canonical labelling: label, then degree (higher
// first), then the multiset of neighbour degrees.  Isomorphisms preserve it,
// so taking the least (labels, mask) only over the relabelings that number
// vertices in ascending invariant order (every order of equal-invariant
// vertices tried) is still a class function, and it tries far fewer than k!
// relabelings unless the pattern is vertex-transitive.
static uint64_t vertex_invariant(const Pat &p, int v, const int *deg) {
    uint64_t code = 0;
    for (int u = 0; u < p.k; u++)
        if (p.adjacent(v, u)) code += uint64_t(1) << (3 * (deg[u] - 1));
    return (uint64_t(uint8_t(p.lab[v] + 1)) << 48) | (uint64_t(7 - deg[v]) << 40) | code;
}

Pat canonical_form(const Pat &p) {
    const int k = p.k;
    int deg[KMAX];
    uint64_t inv[KMAX];
    int order[KMAX];
    for (int v = 0; v < k; v++) deg[v] = __builtin_popcount(p.adj[v]);
    for (int v = 0; v < k; v++) {
        inv[v] = vertex_invariant(p, v, deg);
        order[v] = v;
    }
    std::sort(order, order + k, [&](int a, int b) { return inv[a] != inv[b] ? inv[a] < inv[b] : a < b; });
    int gb[KMAX + 1], ng = 0;      // group boundaries in `order`
    for (int i = 0; i < k; i++)
        if (i == 0 || inv[order[i]] != inv[order[i - 1]]) gb[ng++] = i;
    gb[ng] = k;
    Pat best;
    bool have = false;
    uint64_t best_l = 0;
    uint32_t best_m = 0;
    for (;;) {
        Perm perm{};
        for (int i = 0; i < k; i++) perm[order[i]] = uint8_t(i);
        Pat q = relabel(p, perm);
        const uint64_t l = pack_labels(q);
        const uint32_t m = q.mask();
        if (!have || l < best_l || (l == best_l && m < best_m)) {
            best = q; best_l = l; best_m = m; have = true;
        }
        // next combination of within-group orders (odometer, last group fastest)
        int g = ng - 1;
        while (g >= 0 && !std::next_permutation(order + gb[g], order + gb[g + 1])) g--;
        if (g < 0) break;
    }
    if (best.is_clique()) best.vi = false;
    return best;
}

Key canonical(const Pat &p) {
    Pat c = canonical_form(p);
    Key key;
    key.a = (uint64_t(c.k) << 40) | (uint64_t(c.vi) << 32) | c.mask();
    key.b = pack_labels(c);
    return key;
}

// Backtracking: images for vertices 0..k-1 of p in q, injective.
static void extend(const Pat &p, const Pat &q, bool keep_anti, int u, Perm &f, uint32_t used,
                   std::vector<Perm> &out) {
    if (u == p.k) {
        out.push_back(f);
        return;
    }
    for (int x = 0; x < q.k; x++) {
        if ((used >> x) & 1) continue;
        if (p.lab[u] != q.lab[x]) continue;
        bool ok = true;
        for (int w = 0; w < u && ok; w++) {
            bool pe = p.adjacent(u, w), qe = q.adjacent(x, f[w]);
            if (pe && !qe) ok = false;
            if (keep_anti && !pe && qe) ok = false;
        }
        if (!ok) continue;
        f[u] = uint8_t(x);
        extend(p, q, keep_anti, u + 1, f, used | (1u << x), out);
    }
}

std::vector<Perm> embeddings(const Pat &p, const Pat &q) {
    std::vector<Perm> out;
    if (p.k != q.k) return out;
    Perm f{};
    // anti-edges of p must land on anti-edges of q (q's non-edges when q is
    // vertex-induced; an edge-induced q has none, so nothing can land there)
    bool keep_anti = p.vi;
    if (p.vi && !q.vi && !p.is_clique()) return out;
    extend(p, q, keep_anti, 0, f, 0, out);
    return out;
}

std::vector<Perm> automorphisms(const Pat &p) {
    Pat e = p;
    e.vi = false;
    return embeddings(e, e);   // bijective edge-preserving maps of p onto itself
}

std::vector<int> orbit_of(const Pat &p, const std::vector<Perm> &aut) {
    std::vector<int> orb(p.k);
    for (int u = 0; u < p.k; u++) {
        int best = u;
        for (const Perm &s : aut) best = std::min(best, int(s[u]));
        orb[u] = best;
    }
    return orb;
}

std::vector<Super> superpatterns(const Pat &p) {
    std::vector<std::pair<int, int>> free_pairs;
    for (int a = 0; a < p.k; a++)
        for (int b = a + 1; b < p.k; b++)
            if (!p.adjacent(a, b)) free_pairs.push_back({a, b});
    Pat pe = p;
    pe.vi = false;
    const int64_t n_aut = int64_t(automorphisms(pe).size());
    std::map<Key, size_t> index;
    std::vector<Super> out;
    const uint32_t n_sub = 1u << free_pairs.size();
    for (uint32_t s = 0; s < n_sub; s++) {
        Pat q = pe;
        for (size_t i = 0; i < free_pairs.size(); i++)
            if ((s >> i) & 1) q.add_edge(free_pairs[i].first, free_pairs[i].second);
        q.vi = true;
        Key key = canonical(q);
        if (index.count(key)) continue;
        Pat qc = canonical_form(q);
        qc.vi = true;
        Pat qe = qc;
        qe.vi = false;
        int64_t n_emb = int64_t(embeddings(pe, qe).size());
        index[key] = out.size();
        out.push_back({qc, n_emb / n_aut});
    }
    return out;
}

}  // namespace pm
