"""Oracle pattern algebra: patterns, isomorphisms, morph coefficients, morph rules.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this package; the library never does.

Everything here is the plain definition written out with itertools, for
patterns of at most 8 vertices:

* A pattern (Section 2, "Pattern Semantics") is a simple connected graph on
  vertices 0..k-1 with optional vertex labels (-1 = any label).  Its
  edge-induced form p^E has no anti-edges; its vertex-induced form p^V has an
  anti-edge on every non-adjacent pair.
* phi(p, q) (Section 3.2.1) is the set of injective maps V(p) -> V(q) that send
  edges to edges and anti-edges to anti-edges (and keep labels); Aut(p) is
  phi(p, p).
* q is a non-isomorphic superpattern of p (Section 3.2.1) when p embeds in q,
  q is not isomorphic to p, and q has the same number of vertices (the paper
  morphs only between patterns of equal vertex count, Section 3.1 Discussion).
* Theorem 3.1 / 3.2 (E from V) and Corollary 3.1 applied recursively
  (V from E) are implemented on integer counts and on MNI domains.

Counts are numbers of distinct subgraphs: |matches| / |Aut(p)| (the paper's
coefficients count "unique" matches, e.g. three 4-cycles in a 4-clique,
Section 3.1), so the morph coefficient is c(p, q) = |phi(p^E, q^E)| / |Aut(p)|.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np


def pairs(k):
    """All vertex pairs (a, b), a < b, in lexicographic order."""
    return [(a, b) for a in range(k) for b in range(a + 1, k)]


def mask_to_edges(k, mask):
    return frozenset(pr for i, pr in enumerate(pairs(k)) if mask >> i & 1)


def edges_to_mask(k, edges):
    idx = {pr: i for i, pr in enumerate(pairs(k))}
    m = 0
    for a, b in edges:
        m |= 1 << idx[(min(a, b), max(a, b))]
    return m


class Pattern:
    """k vertices, an edge set, labels (tuple, -1 = any) and induced flag."""

    __slots__ = ("k", "edges", "labels", "vertex_induced")

    def __init__(self, k, edges, labels=None, vertex_induced=False):
        self.k = k
        self.edges = frozenset((min(a, b), max(a, b)) for a, b in edges)
        self.labels = tuple(labels) if labels is not None else (-1,) * k
        self.vertex_induced = bool(vertex_induced)
        assert len(self.labels) == k

    @staticmethod
    def from_mask(k, mask, labels=None, vertex_induced=False):
        return Pattern(k, mask_to_edges(k, mask), labels, vertex_induced)

    @property
    def mask(self):
        return edges_to_mask(self.k, self.edges)

    @property
    def is_clique(self):
        return len(self.edges) == self.k * (self.k - 1) // 2

    @property
    def anti_edges(self):
        if not self.vertex_induced:
            return frozenset()
        return frozenset(pr for pr in pairs(self.k) if pr not in self.edges)

    def with_induced(self, vertex_induced):
        return Pattern(self.k, self.edges, self.labels, vertex_induced)

    def connected(self):
        seen, stack = {0}, [0]
        while stack:
            v = stack.pop()
            for a, b in self.edges:
                for x, y in ((a, b), (b, a)):
                    if x == v and y not in seen:
                        seen.add(y)
                        stack.append(y)
        return len(seen) == self.k

    def relation(self):
        """k x k matrix: +1 edge, -1 anti-edge, 0 unconstrained pair."""
        r = [[0] * self.k for _ in range(self.k)]
        for a, b in self.edges:
            r[a][b] = r[b][a] = 1
        for a, b in self.anti_edges:
            r[a][b] = r[b][a] = -1
        return r

    def __repr__(self):
        kind = "V" if self.vertex_induced else "E"
        lab = "" if all(x < 0 for x in self.labels) else f", labels={self.labels}"
        return f"Pattern(k={self.k}, edges={sorted(self.edges)}{lab}, {kind})"


def _respects(p, q, f):
    """f (tuple, f[u] = image of u) sends E(p) into E(q), A(p) into A(q), labels equal."""
    qa = q.anti_edges
    for a, b in p.edges:
        if (min(f[a], f[b]), max(f[a], f[b])) not in q.edges:
            return False
    for a, b in p.anti_edges:
        if (min(f[a], f[b]), max(f[a], f[b])) not in qa:
            return False
    for u in range(p.k):
        if p.labels[u] != q.labels[f[u]]:
            return False
    return True


def phi(p, q):
    """All subgraph isomorphisms from pattern p into pattern q (injective maps)."""
    return [f for f in itertools.permutations(range(q.k), p.k) if _respects(p, q, f)]


def automorphisms(p):
    return phi(p, p)


def orbits(p):
    """Orbits of V(p) under its (label-preserving) automorphism group."""
    auts = automorphisms(p)
    seen, out = set(), []
    for u in range(p.k):
        if u in seen:
            continue
        orb = sorted({f[u] for f in auts})
        seen.update(orb)
        out.append(orb)
    return out


def canonical(p):
    """Canonical key: lexicographically least (labels, sorted edges) over relabelings."""
    return _canonical(p.k, tuple(sorted(p.edges)), p.labels, p.vertex_induced)


@lru_cache(maxsize=None)
def _canonical(k, edge_tuple, labels_in, vertex_induced):
    p = Pattern(k, edge_tuple, labels_in, vertex_induced)
    best = None
    for perm in itertools.permutations(range(p.k)):
        # perm[u] = new name of u
        labels = [None] * p.k
        for u in range(p.k):
            labels[perm[u]] = p.labels[u]
        edges = tuple(sorted((min(perm[a], perm[b]), max(perm[a], perm[b])) for a, b in p.edges))
        key = (p.k, tuple(labels), edges, p.vertex_induced)
        if best is None or key < best:
            best = key
    return best


def from_canonical(key):
    k, labels, edges, vi = key
    return Pattern(k, edges, labels, vi)


def isomorphic(p, q):
    return canonical(p) == canonical(q)


@lru_cache(maxsize=None)
def unlabeled_canonical_table(k):
    """Canonical mask for every edge mask on k vertices: min over all vertex
    permutations of the permuted mask (numpy over all masks at once)."""
    prs = pairs(k)
    idx = {pr: i for i, pr in enumerate(prs)}
    npairs = len(prs)
    masks = np.arange(1 << npairs, dtype=np.int64)
    bits = (masks[:, None] >> np.arange(npairs)) & 1
    best = masks.copy()
    for perm in itertools.permutations(range(k)):
        dest = np.array([idx[(min(perm[a], perm[b]), max(perm[a], perm[b]))] for a, b in prs], dtype=np.int64)
        permuted = (bits << dest[None, :]).sum(axis=1)
        np.minimum(best, permuted, out=best)
    return best


def connected_classes(k):
    """One representative (the canonical mask) per isomorphism class of connected
    unlabeled graphs on k vertices, sorted by (edge count, mask)."""
    table = unlabeled_canonical_table(k)
    reps = sorted(set(int(x) for x in np.unique(table)))
    out = [m for m in reps if Pattern.from_mask(k, m).connected()]
    return sorted(out, key=lambda m: (bin(m).count("1"), m))


def all_classes(k):
    """Every isomorphism class (connected or not) of unlabeled graphs on k vertices."""
    table = unlabeled_canonical_table(k)
    return sorted(set(int(x) for x in np.unique(table)))


def superpatterns(p):
    """Non-isomorphic superpatterns of p on the same vertices, p included, as
    vertex-induced patterns carrying p's labels (one per class)."""
    return [from_canonical(key) for key in
            _superpattern_keys(p.k, tuple(sorted(p.edges)), p.labels)]


@lru_cache(maxsize=None)
def _superpattern_keys(k, edge_tuple, labels):
    p = Pattern(k, edge_tuple, labels, False)
    return tuple(canonical(q) for q in _superpatterns(p))


def _superpatterns(p):
    """Built by adding edges to p in p's own numbering, one per class."""
    free = [pr for pr in pairs(p.k) if pr not in p.edges]
    seen = {}
    for r in range(len(free) + 1):
        for extra in itertools.combinations(free, r):
            q = Pattern(p.k, p.edges | set(extra), p.labels, True)
            key = canonical(q)
            if key not in seen:
                seen[key] = q
    return list(seen.values())


def coefficient(p, q):
    """c(p, q) = number of distinct copies of p^E spanning q = |phi(p^E, q^E)| / |Aut(p^E)|."""
    pe, qe = p.with_induced(False), q.with_induced(False)
    n_phi = len(phi(pe, qe))
    n_aut = len(automorphisms(pe))
    assert n_phi % n_aut == 0
    return n_phi // n_aut


# ---------------------------------------------------------------------------
# Morph rules on counts.  `count_V` / `count_E` are callables Pattern -> int.

def count_E_from_V(p, count_V):
    """Theorem 3.1/3.2 with counting (lambda = size, (+) = sum, permute = identity):
    count(p^E) = count(p^V) + sum over superpatterns q of c(p, q) * count(q^V)."""
    total = 0
    for q in superpatterns(p):
        total += coefficient(p, q) * count_V(q)
    return total


def count_V_from_E(p, count_E, _memo=None):
    """Corollary 3.1 applied recursively until cliques:
    count(p^V) = count(p^E) - sum over non-isomorphic superpatterns q of
    c(p, q) * count(q^V), each count(q^V) expanded the same way."""
    memo = {} if _memo is None else _memo
    key = canonical(p.with_induced(True))
    if key in memo:
        return memo[key]
    value = count_E(p.with_induced(False))
    if not p.is_clique:
        for q in superpatterns(p):
            if isomorphic(q, p.with_induced(True)):
                continue
            value -= coefficient(p, q) * count_V_from_E(q, count_E, memo)
    memo[key] = value
    return value


def mni_E_from_V(p, domains_V):
    """Theorem 3.2 with MNI tables: the domain of vertex u of p^E is the union
    of the domain of u in p^V and, for every superpattern q and every
    f in phi(p^E, q^E), the domain of f(u) in q^V.  `domains_V(q)` returns one
    set (or boolean array) of data vertices per vertex of q^V."""
    pe = p.with_induced(False)
    out = [None] * p.k
    for q in superpatterns(p):
        dq = domains_V(q)
        for f in phi(pe, q.with_induced(False)):
            for u in range(p.k):
                out[u] = dq[f[u]].copy() if out[u] is None else (out[u] | dq[f[u]])
    return out


def mni_support(p, domains):
    """MNI support: one column per orbit of Aut(p) holding the images of its
    vertices over all matches; the support is the smallest column size."""
    sizes = []
    for orb in orbits(p):
        col = domains[orb[0]].copy()
        for u in orb[1:]:
            col = col | domains[u]
        sizes.append(int(np.count_nonzero(col)) if isinstance(col, np.ndarray) else len(col))
    return min(sizes)


# ---------------------------------------------------------------------------
# Brute force on tiny graphs (n <= 12): ground truth from the definitions.

def brute_force_vertex_induced(n, edge_set, k, labels=None):
    """Histogram {canonical key: count} of G[S] over all k-subsets S (connected
    or not), as vertex-induced patterns carrying S's labels."""
    hist = {}
    for S in itertools.combinations(range(n), k):
        loc = {v: i for i, v in enumerate(S)}
        es = [(loc[a], loc[b]) for a, b in itertools.combinations(S, 2) if (a, b) in edge_set]
        lab = [labels[v] for v in S] if labels is not None else None
        key = canonical(Pattern(k, es, lab, True))
        hist[key] = hist.get(key, 0) + 1
    return hist


def brute_force_edge_induced(n, edge_set, k, labels=None):
    """Histogram {canonical key: count} over edge subsets F whose endpoints are
    exactly k vertices and whose graph (V(F), F) is connected."""
    hist = {}
    for S in itertools.combinations(range(n), k):
        loc = {v: i for i, v in enumerate(S)}
        es = [(loc[a], loc[b]) for a, b in itertools.combinations(S, 2) if (a, b) in edge_set]
        lab = [labels[v] for v in S] if labels is not None else None
        for r in range(k - 1, len(es) + 1):
            for F in itertools.combinations(es, r):
                touched = {x for e in F for x in e}
                if len(touched) != k:
                    continue
                p = Pattern(k, F, lab, False)
                if not p.connected():
                    continue
                key = canonical(p)
                hist[key] = hist.get(key, 0) + 1
    return hist


def brute_force_matches(n, edge_set, p, labels=None):
    """Every match of p (Section 2): injective maps respecting edges, anti-edges, labels."""
    out = []
    anti = p.anti_edges
    for img in itertools.permutations(range(n), p.k):
        ok = all((min(img[a], img[b]), max(img[a], img[b])) in edge_set for a, b in p.edges)
        ok = ok and all((min(img[a], img[b]), max(img[a], img[b])) not in edge_set for a, b in anti)
        if ok and labels is not None:
            ok = all(p.labels[u] < 0 or p.labels[u] == labels[img[u]] for u in range(p.k))
        if ok:
            out.append(img)
    return out
