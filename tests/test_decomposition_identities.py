"""CPU check of the counting identities the decomposition kernels evaluate
for the neighbourhood-graph patterns, each written out here in plain Python
over adjacency sets and compared with the oracle's direct edge-induced
counts (an independent matcher) on small random graphs:

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
