"""Pins for the oracle's MNI support and level-wise FSM (Section 2, Frequent
Subgraph Mining), CPU only.

* MNI support: one column per automorphism orbit of the (labeled) pattern,
  the column holding the images of all of the orbit's vertices, support =
  the smallest column.  Checked on hand-countable domains and on domains
  collected from a symmetry-broken subset of matches, where the orbit union
  differs from every single vertex's image set.
* FSM: brute force over every connected labeled subgraph of the data graph
  with 1..3 edges (so every pattern with support >= 1 is seen, without any
  level-wise generation), each support computed from brute-force matches;
  the oracle's frequent sets at every level and its candidate supports must
  equal it at several thresholds (anti-monotonicity makes the level-wise
  frequent sets exact)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import algebra
from oracle.algebra import Pattern
from pm_inputs import gnp_edges, uniform_ints


def brute_orbits(p):
    """Orbits of the label-preserving automorphisms, by trying every permutation."""
    auts = []
    for f in itertools.permutations(range(p.k)):
        if all((min(f[a], f[b]), max(f[a], f[b])) in p.edges for a, b in p.edges) and \
                all(p.labels[u] == p.labels[f[u]] for u in range(p.k)):
            auts.append(f)
    orbs, seen = [], set()
    for u in range(p.k):
        if u not in seen:
            o = sorted({f[u] for f in auts})
            seen.update(o)
            orbs.append(o)
    return orbs


def brute_support(p, maps):
    """min over orbit columns of |{m(u) : m a match, u in the orbit}|."""
    if not maps:
        return 0
    return min(len({m[u] for m in maps for u in orb}) for orb in brute_orbits(p))


def test_mni_support_orbit_columns_hand_checked():
    # labeled wedge: leaves labeled 0 (one orbit {0, 2}), centre labeled 1
    wedge = Pattern(3, [(0, 1), (1, 2)], labels=(0, 1, 0))
    dom = [np.zeros(30, bool) for _ in range(3)]
    dom[0][[10, 11]] = True
    dom[1][[20, 21, 22, 23]] = True
    dom[2][[12]] = True
    # columns {10, 11, 12} (size 3) and {20..23} (size 4): support 3
    # (per-vertex columns would give 1, the largest column 4)
    assert algebra.mni_support(wedge, dom) == 3
    # an unlabeled path on 3 vertices has the same orbits; a triangle has one column
    tri = Pattern(3, [(0, 1), (1, 2), (0, 2)])
    assert algebra.mni_support(tri, dom) == 7
    # all three vertices in different orbits when every label differs
    path = Pattern(3, [(0, 1), (1, 2)], labels=(0, 1, 2))
    assert algebra.mni_support(path, dom) == 1


def test_mni_support_on_symmetry_broken_matches():
    """K_{5,3}: five centres labeled 1, three leaves labeled 0; pattern = the
    labeled wedge 0-1-0.  Keeping only the matches with image(0) < image(2)
    (one per automorphic pair) gives leaf domains of size 2 each, whose
    union, the leaf column, has all 3 leaves: the support is min(3, 5) = 3."""
    centres, leaves = list(range(5)), [5, 6, 7]
    edges = {(c, l) for c in centres for l in leaves}
    labels = [1] * 5 + [0] * 3
    wedge = Pattern(3, [(0, 1), (1, 2)], labels=(0, 1, 0))
    maps = algebra.brute_force_matches(8, edges, wedge, labels)
    broken = [m for m in maps if m[0] < m[2]]
    dom = np.zeros((3, 8), bool)
    for m in broken:
        for u in range(3):
            dom[u, m[u]] = True
    assert [int(dom[u].sum()) for u in range(3)] == [2, 5, 2]
    assert algebra.mni_support(wedge, dom) == 3
    assert brute_support(wedge, broken) == 3
    g = oracle.prepare_graph(8, [c for c, l in sorted(edges)], [l for c, l in sorted(edges)],
                             np.array(labels))
    assert oracle.support_direct(g, wedge) == 3


def connected_labeled_subgraphs(n, edge_set, labels, max_edges):
    """{canonical key: pattern} of every connected edge subset of the data
    graph with 1..max_edges edges, as an edge-induced labeled pattern."""
    out = {}
    es = sorted(edge_set)
    for r in range(1, max_edges + 1):
        for F in itertools.combinations(es, r):
            vs = sorted({v for e in F for v in e})
            loc = {v: i for i, v in enumerate(vs)}
            p = Pattern(len(vs), [(loc[a], loc[b]) for a, b in F], [int(labels[v]) for v in vs], False)
            if p.connected():
                out.setdefault(algebra.canonical(p), p)
    return out


@pytest.mark.parametrize("seed,n,prob,n_labels", [(41, 8, 0.45, 2), (42, 9, 0.4, 3), (43, 9, 0.5, 2),
                                                    (46, 10, 0.8, 2)])
def test_fsm_against_brute_force(seed, n, prob, n_labels):
    s, d = gnp_edges(n, prob, seed)
    labels = uniform_ints(seed, 77, n, 0, n_labels).astype(np.int64)
    g = oracle.prepare_graph(n, s, d, labels)
    es = g.edge_set()
    subs = connected_labeled_subgraphs(n, es, labels, 3)
    support = {key: brute_support(p, algebra.brute_force_matches(n, es, p, labels))
               for key, p in subs.items()}
    n_edges = lambda key: len(key[2])
    # all 22 connected labeled 3-edge patterns over 2 labels occur in the
    # seed-46 graph, so a candidate that the level-wise generation misses
    # shows up there as a missing frequent pattern
    for threshold in (1, 2, 3, 4):
        cand, levels = oracle.fsm(g, 3, threshold)
        assert len(levels) == 3
        for j, level in enumerate(levels, start=1):
            want = sorted(key for key, sp in support.items() if n_edges(key) == j and sp >= threshold)
            assert level == want, (threshold, j)
        # every 3-edge candidate's support is the brute-force one (0 if it never occurs)
        for key, sp in cand.items():
            assert sp == support.get(key, 0), key
        # and every frequent 3-edge pattern was a candidate
        assert {key for key, sp in support.items() if n_edges(key) == 3 and sp >= threshold} <= set(cand)
