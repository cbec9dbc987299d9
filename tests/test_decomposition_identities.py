"""CPU check of the counting identities the decomposition kernels evaluate,
each written out here in plain Python over adjacency sets and compared with
the oracle's direct edge-induced counts (an independent matcher) on small
random graphs: the 22 local identities of the 4- and 5-vertex patterns
(`local_counts`), and those of the neighbourhood-graph patterns:

* 4-wheel = sum_c sum_{a in N(c)} sum_{b in N(c), b < a} C(x_cab, 2),
  x_cab = #{x in N(c) n N(a) n N(b) : x < a}  (rims are 4-cycles of G[N(c)]);
* K2,3 = sum_{a > b} C(c_ab, 3) and K2,3 plus an edge in its 3-side =
  sum_{a > b} e_ab (c_ab - 2), with c_ab the common neighbours of a and b and
  e_ab the edges among them;
* K5 minus an edge = sum over triangles of C(k, 2), k the vertices adjacent
  to all three.

A wrong term in any of them (a dropped restriction, an off-by-one in the
"- 2", a missing binomial) changes the value on these graphs."""
from itertools import combinations
from math import comb

import numpy as np
import pytest

import oracle
from oracle import algebra
from pm_inputs import gnp_edges, rmat_edges

W4, K23, K23E, K5E = 495, 126, 254, 511


def adjacency(n, s, d):
    adj = [set() for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def wheel(adj):
    total = 0
    for c, nc in enumerate(adj):
        for a in nc:
            for b in nc:
                if b < a:
                    x = sum(1 for v in nc & adj[a] & adj[b] if v < a)
                    total += comb(x, 2)
    return total


def k23_pair_sums(adj):
    k23 = k23e = 0
    for a, b in combinations(range(len(adj)), 2):
        common = adj[a] & adj[b]
        c = len(common)
        e = sum(1 for x, y in combinations(sorted(common), 2) if y in adj[x])
        k23 += comb(c, 3)
        if e:
            k23e += e * (c - 2)
    return k23, k23e


def k5_minus_edge(adj):
    total = 0
    for x in range(len(adj)):
        for y in adj[x]:
            if y <= x:
                continue
            for z in adj[x] & adj[y]:
                if z <= y:
                    continue
                total += comb(len(adj[x] & adj[y] & adj[z]), 2)
    return total


def graphs():
    s, d = gnp_edges(18, 0.45, 901)
    yield "gnp18", 18, s, d
    s, d = gnp_edges(26, 0.3, 902)
    yield "gnp26", 26, s, d
    s, d = rmat_edges(5, 6, seed=903)
    yield "rmat5", 32, s, d


@pytest.mark.parametrize("name,n,s,d", list(graphs()), ids=lambda x: x if isinstance(x, str) else "")
def test_identities_match_the_oracle(name, n, s, d):
    og = oracle.prepare_graph(n, s, d)
    adj = adjacency(n, np.asarray(s), np.asarray(d))
    want = {m: oracle.count(og, algebra.Pattern.from_mask(5, m)) for m in (W4, K23, K23E, K5E)}
    assert any(v > 0 for v in want.values())
    k23, k23e = k23_pair_sums(adj)
    assert wheel(adj) == want[W4]
    assert k23 == want[K23]
    assert k23e == want[K23E]
    assert k5_minus_edge(adj) == want[K5E]


def test_identities_on_complete_graph():
    """K_7: every identity against the closed form C(7,5) * 5! / |Aut(p)|."""
    n = 7
    adj = [set(range(n)) - {v} for v in range(n)]
    closed = {m: comb(n, 5) * 120 // len(algebra.automorphisms(algebra.Pattern.from_mask(5, m)))
              for m in (W4, K23, K23E, K5E)}
    k23, k23e = k23_pair_sums(adj)
    assert (wheel(adj), k23, k23e, k5_minus_edge(adj)) == (closed[W4], closed[K23], closed[K23E], closed[K5E])


def c(x, k):
    return comb(x, k) if x >= k >= 0 else 0


def local_counts(adj):
    """The identities over per-vertex, per-edge, per-triangle and rooted
    2-path quantities that the decomposition evaluates for the other
    unlabeled edge-induced 4- and 5-vertex patterns (d degree, t_e triangles
    on edge e, t_v triangles at v, S_v the sum of the neighbours' degrees,
    W_a[c] 2-paths a-b-c with b, c below a in (degree, id) order, k4_e
    4-cliques on edge e)."""
    n = len(adj)
    deg0 = [len(a) for a in adj]
    order = sorted(range(n), key=lambda v: (deg0[v], v))
    rank = {v: i for i, v in enumerate(order)}
    N = [sorted(rank[x] for x in adj[order[i]]) for i in range(n)]
    A = [set(x) for x in N]
    d = [len(x) for x in N]
    t = {(u, v): len(A[u] & A[v]) for u in range(n) for v in N[u]}
    tv = [sum(t[(u, v)] for v in N[u]) // 2 for u in range(n)]
    S = [sum(d[x] for x in N[u]) for u in range(n)]
    und = [(u, v) for u in range(n) for v in N[u] if u < v]
    tri = [(a, b, x) for a in range(n) for b in N[a] if b < a for x in N[b] if x < b and x in A[a]]
    T = len(tri)
    k4e = {(u, v): sum(1 for x, y in combinations(sorted(A[u] & A[v]), 2) if y in A[x]) for (u, v) in und}
    K4 = sum(k4e.values()) // 6
    DE = sum(c(t[e], 2) for e in und)
    C4 = banner2 = house = c5 = 0
    for a in range(n):
        W = {}
        low = [b for b in N[a] if b < a]
        for b in low:
            for x in N[b]:
                if x < a:
                    W[x] = W.get(x, 0) + 1
        C4 += sum(c(w, 2) for w in W.values())
        for b in low:
            for x in N[b]:
                if x < a:
                    w = W[x]
                    banner2 += (w - 1) * (2 * d[b] + d[a] + d[x] - 8)
                    house += (w - 1) * (t[(a, b)] + t[(b, x)])
        c5 += sum(W[x] * sum(W.get(y, 0) for y in N[x] if y < x) for x in W)
        c5 -= sum(sum(1 for x in N[b] if x < a) * W.get(b, 0) for b in low)
        c5 += sum(W.get(b, 0) for b in low) // 2
    c5 -= sum(sum(1 for y in N[v] if y > a) for (a, b, x) in tri for v in (a, b, x))
    S1 = [sum(d[x] - 1 for x in N[v]) for v in range(n)]
    S2 = [sum((d[x] - 1) ** 2 for x in N[v]) for v in range(n)]
    return {
        (4, 7): sum(c(x, 3) for x in d),
        (4, 13): sum((d[u] - 1) * (d[v] - 1) for (u, v) in und) - 3 * T,
        (4, 15): sum(tv[v] * (d[v] - 2) for v in range(n)),
        (4, 31): DE,
        (4, 63): K4,
        (5, 15): sum(c(x, 4) for x in d),
        (5, 29): sum(c(d[v] - 1, 2) * (S[v] - d[v]) - 2 * tv[v] * (d[v] - 2) for v in range(n)),
        (5, 58): sum((S1[v] ** 2 - S2[v]) // 2 for v in range(n)) - 4 * C4
                 - 2 * sum(tv[v] * d[v] for v in range(n)) + 9 * T,
        (5, 31): sum(tv[v] * c(d[v] - 2, 2) for v in range(n)),
        (5, 59): sum(t[e] * ((d[e[0]] - 2) * (d[e[1]] - 2) - t[e] + 1) for e in und),
        (5, 185): sum(tv[u] * (S[u] - d[u] + 4) for u in range(n))
                  - sum(t[(u, v)] * (d[v] + t[(u, v)]) for u in range(n) for v in N[u]),
        (5, 62): banner2 // 2 - 2 * DE,
        (5, 220): c5,
        (5, 63): sum(c(t[e], 2) * (d[e[0]] + d[e[1]] - 6) for e in und),
        (5, 187): sum((t[(u, v)] - 1) * d[w] + (t[(v, w)] - 1) * d[u] + (t[(u, w)] - 1) * d[v] for (u, v, w) in tri)
                  - 2 * sum(t[e] * (t[e] - 1) for e in und) - 12 * K4,
        (5, 207): sum(c(x, 2) for x in tv) - 2 * DE,
        (5, 221): house - 4 * DE,
        (5, 127): sum(c(t[e], 3) for e in und),
        (5, 223): sum((t[(h, y)] - 1) * (t[(h, z)] - 1) for (a, b, x) in tri
                      for (h, y, z) in ((a, b, x), (b, a, x), (x, a, b))) - 12 * K4,
        (5, 191): sum(k4e[(u, v)] * (d[u] + d[v]) for (u, v) in und) // 3 - 12 * K4,
        (5, 255): sum(k4e[e] * (t[e] - 2) for e in und),
    }


@pytest.mark.parametrize("name,n,s,d", list(graphs()), ids=lambda x: x if isinstance(x, str) else "")
def test_local_identities_match_the_oracle(name, n, s, d):
    og = oracle.prepare_graph(n, s, d)
    got = local_counts(adjacency(n, np.asarray(s), np.asarray(d)))
    for (k, m), v in got.items():
        assert v == oracle.count(og, algebra.Pattern.from_mask(k, m)), (k, m)
