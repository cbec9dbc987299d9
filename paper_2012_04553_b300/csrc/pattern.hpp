// Pattern algebra on the host: small graphs (k <= 8) with labels and
// anti-edges, their automorphisms, canonical forms, subgraph isomorphisms
// between patterns and the superpatterns used by morphing.
//
// Definitions (Jamshidi & Vora, Section 2 and Section 3.2.1):
//  * a pattern is a simple connected graph, optionally vertex-labeled; the
//    vertex-induced form has an anti-edge on every non-adjacent pair, the
//    edge-induced form none (cliques are both);
//  * phi(p, q) is the set of injective maps V(p) -> V(q) that keep edges,
//    anti-edges and labels; with |p| = |q| they are permutations;
//  * a non-isomorphic superpattern q of p has the same vertex count (the
//    paper morphs only between equal sizes) and contains p.
#pragma once

#include <array>
#include <cstdint>
#include <vector>

namespace pm {

constexpr int KMAX = 8;

using Perm = std::array<uint8_t, KMAX>;

struct Pat {
    int k = 0;
    uint8_t adj[KMAX] = {};     // adjacency bitmask per vertex
    int8_t lab[KMAX] = {-1, -1, -1, -1, -1, -1, -1, -1};
    bool vi = false;            // vertex-induced (anti-edges on all non-adjacent pairs)

    bool adjacent(int a, int b) const { return (adj[a] >> b) & 1; }
    void add_edge(int a, int b) { adj[a] |= uint8_t(1u << b); adj[b] |= uint8_t(1u << a); }
    int n_edges() const;
    bool is_clique() const { return n_edges() == k * (k - 1) / 2; }
    bool connected() const;
    bool labeled() const;
    uint32_t mask() const;                      // lexicographic pair order
    static Pat from_mask(int k, uint32_t mask, const int8_t *lab, bool vi);
};

// Canonical key (k, induced flag, labels and edge mask minimised over the
// relabelings that number vertices in ascending order of an isomorphism
// invariant: a class function).  Cliques are keyed as edge-induced since
// both forms coincide.
struct Key {
    uint64_t a = 0, b = 0;
    bool operator<(const Key &o) const { return a != o.a ? a < o.a : b < o.b; }
    bool operator==(const Key &o) const { return a == o.a && b == o.b; }
};

Key canonical(const Pat &p);
// The canonical representative itself (vertex numbering of the minimum).
Pat canonical_form(const Pat &p);

// Label- and edge-preserving permutations of p (the same group for p^E and p^V).
std::vector<Perm> automorphisms(const Pat &p);
// orbit[u] = smallest vertex in u's orbit under automorphisms(p).
std::vector<int> orbit_of(const Pat &p, const std::vector<Perm> &aut);

// All bijections f (|p| = |q|) with f(E(p)) in E(q), labels kept, and, if p
// is vertex-induced, f(A(p)) in A(q).
std::vector<Perm> embeddings(const Pat &p, const Pat &q);

struct Super {
    Pat q;            // vertex-induced superpattern (p's labels kept), canonical numbering
    int64_t coef;     // c(p, q) = |phi(p^E, q^E)| / |Aut(p^E)|: distinct spanning copies of p in q
};
// Every superpattern class of p on p's vertex count, p itself included
// (first), each with its coefficient.
std::vector<Super> superpatterns(const Pat &p);

}  // namespace pm
