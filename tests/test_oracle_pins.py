"""Pins for the oracle: values the paper prints, closed forms, brute force,
invariants.  CPU only; the oracle is checked against things other than itself."""
import itertools
import json
import os
from math import comb, factorial

import numpy as np
import pytest

import oracle
from oracle import algebra
from oracle.algebra import Pattern
from pm_inputs import gnp_edges, rmat_edges, splitmix64, zipf_labels, uniform_ints

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# 4-vertex connected graphs in algebra.connected_classes(4) order
STAR, P4, PAW, C4, DIAMOND, K4 = algebra.connected_classes(4)


def pat(mask, k=4, vi=False, labels=None):
    return Pattern.from_mask(k, mask, labels, vi)


def graph_from_pairs(n, pairs_, labels=None):
    s = np.array([a for a, b in pairs_], dtype=np.int32)
    d = np.array([b for a, b in pairs_], dtype=np.int32)
    return oracle.prepare_graph(n, s, d, labels)


# --------------------------------------------------------------- generator
def test_splitmix64_reference_value():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (published test vector)
    assert int(splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


# --------------------------------------------------------------- algebra
def test_graph_class_counts():
    # OEIS A001349 (connected graphs) and A000088 (all graphs) on k vertices
    assert [len(algebra.connected_classes(k)) for k in range(1, 7)] == [1, 1, 2, 6, 21, 112]
    assert [len(algebra.all_classes(k)) for k in range(1, 7)] == [1, 2, 4, 11, 34, 156]


def test_four_vertex_shapes_and_automorphisms():
    shapes = {
        STAR: (3, 6), P4: (3, 2), PAW: (4, 2), C4: (4, 8), DIAMOND: (5, 4), K4: (6, 24)}
    for m, (ne, aut) in shapes.items():
        p = pat(m)
        assert len(p.edges) == ne
        assert len(algebra.automorphisms(p)) == aut
    degs = lambda m: sorted(sum(1 for e in pat(m).edges if v in e) for v in range(4))
    assert degs(STAR) == [1, 1, 1, 3] and degs(P4) == [1, 1, 2, 2]
    assert degs(PAW) == [1, 2, 2, 3] and degs(C4) == [2, 2, 2, 2]


def test_paper_printed_coefficients():
    # Section 3.1: a 4-clique holds three distinct edge-induced 4-cycles, and
    # C4^E = C4^V + diamond^V + 3 K4 ([PR-E2] as described in the text).
    assert algebra.coefficient(pat(C4), pat(K4, vi=True)) == 3
    assert algebra.coefficient(pat(C4), pat(DIAMOND, vi=True)) == 1
    # Section 3.2.1: phi(tailed triangle^E, chordal 4-cycle^V) has four members
    assert algebra.coefficient(pat(PAW), pat(DIAMOND, vi=True)) == 4
    supers = {algebra.canonical(q) for q in algebra.superpatterns(pat(C4))}
    assert supers == {algebra.canonical(pat(m, vi=True)) for m in (C4, DIAMOND, K4)}


def test_k4_coefficient_matrix():
    # rows p, columns q in (K1,3, P4, paw, C4, diamond, K4); brute-force derived
    want = [[1, 0, 1, 0, 2, 4], [0, 1, 2, 4, 6, 12], [0, 0, 1, 0, 4, 12],
            [0, 0, 0, 1, 1, 3], [0, 0, 0, 0, 1, 6], [0, 0, 0, 0, 0, 1]]
    cls = algebra.connected_classes(4)
    got = []
    for a in cls:
        sup = {algebra.canonical(q) for q in algebra.superpatterns(pat(a))}
        got.append([algebra.coefficient(pat(a), pat(b, vi=True))
                    if algebra.canonical(pat(b, vi=True)) in sup else 0 for b in cls])
    assert got == want


def test_coefficient_counts_spanning_copies_by_brute_force():
    # c(p, q) = number of edge subsets of q that are spanning copies of p
    for k in (4, 5):
        for a in algebra.connected_classes(k):
            p = pat(a, k)
            for q in algebra.superpatterns(p):
                copies = 0
                for F in itertools.combinations(sorted(q.edges), len(p.edges)):
                    sub = Pattern(k, F)
                    if len({v for e in F for v in e}) == k and algebra.isomorphic(sub, p):
                        copies += 1
                assert algebra.coefficient(p, q) == copies


def test_paper_worked_example_maps():
    # Section 3.2.1: M(p4) o phi(p2^E, p4) for the 4-clique match {1->a,2->d,3->f,4->e}
    # lists three maps; each is a 4-cycle match and the three cycles are distinct.
    printed = [{1: "a", 2: "d", 3: "f", 4: "e"}, {1: "a", 2: "d", 4: "f", 3: "e"},
               {1: "a", 3: "d", 2: "f", 4: "e"}]
    cycle = [(1, 2), (2, 3), (3, 4), (4, 1)]
    edge_sets = {frozenset(frozenset((m[x], m[y])) for x, y in cycle) for m in printed}
    assert len(edge_sets) == 3
    assert len(edge_sets) == algebra.coefficient(pat(C4), pat(K4, vi=True))


def test_moebius_inverse_identity():
    # E-from-V coefficients C and V-from-E recursion must be mutually inverse:
    # check C @ Chat = I with Chat[p][q] = (-1)^(e(q)-e(p)) c(p, q)
    for k in (4, 5):
        cls = algebra.connected_classes(k)
        idx = {algebra.canonical(pat(m, k, vi=True)): i for i, m in enumerate(cls)}
        C = np.zeros((len(cls), len(cls)), dtype=np.int64)
        for i, m in enumerate(cls):
            for q in algebra.superpatterns(pat(m, k)):
                C[i, idx[algebra.canonical(q)]] = algebra.coefficient(pat(m, k), q)
        e = np.array([bin(m).count("1") for m in cls])
        S = np.where((e[None, :] - e[:, None]) % 2 == 0, 1, -1)
        assert (C @ (S * C) == np.eye(len(cls), dtype=np.int64)).all()


def test_morph_rules_on_symbolic_counts():
    # V-from-E recursion inverts E-from-V on arbitrary (random) vertex-induced counts
    rng = np.random.default_rng(7)
    for k in (4, 5):
        cv = {algebra.canonical(pat(m, k, vi=True)): int(rng.integers(0, 10**6))
              for m in algebra.connected_classes(k)}
        count_V = lambda q: cv[algebra.canonical(q.with_induced(True))]
        ce = {}
        def count_E(q):
            key = algebra.canonical(q)
            if key not in ce:
                ce[key] = algebra.count_E_from_V(q, count_V)
            return ce[key]
        for m in algebra.connected_classes(k):
            p = pat(m, k, vi=True)
            assert algebra.count_V_from_E(p, count_E) == count_V(p)


# --------------------------------------------------------------- counting
@pytest.mark.parametrize("seed,n,prob", [(1, 9, 0.4), (2, 10, 0.55), (3, 11, 0.3), (4, 12, 0.35)])
def test_counts_against_brute_force(seed, n, prob):
    s, d = gnp_edges(n, prob, seed)
    g = oracle.prepare_graph(n, s, d)
    es = g.edge_set()
    for k in (3, 4, 5):
        bv = algebra.brute_force_vertex_induced(n, es, k)
        be = algebra.brute_force_edge_induced(n, es, k)
        for m in algebra.connected_classes(k):
            pv, pe = pat(m, k, vi=True), pat(m, k)
            assert oracle.count(g, pv) == bv.get(algebra.canonical(pv), 0)
            assert oracle.count(g, pe) == be.get(algebra.canonical(pe), 0)
        # every k-subset induces exactly one class (connected or not)
        assert sum(bv.values()) == comb(n, k)


def test_matches_against_brute_force_maps():
    s, d = gnp_edges(8, 0.5, 9)
    g = oracle.prepare_graph(8, s, d)
    es = g.edge_set()
    for m in algebra.connected_classes(4):
        for vi in (False, True):
            p = pat(m, vi=vi)
            assert oracle.match_count(g, p) == len(algebra.brute_force_matches(8, es, p))


def test_labeled_counts_against_brute_force():
    n = 10
    s, d = gnp_edges(n, 0.5, 5)
    labels = np.array([0, 1, 0, 2, 1, 0, 0, 1, 2, 0])
    g = oracle.prepare_graph(n, s, d, labels)
    es = g.edge_set()
    for k in (3, 4):
        bv = algebra.brute_force_vertex_induced(n, es, k, labels)
        be = algebra.brute_force_edge_induced(n, es, k, labels)
        for key, c in list(bv.items())[:25]:
            p = algebra.from_canonical(key)
            if p.connected():
                assert oracle.count(g, p) == c
        for key, c in list(be.items())[:25]:
            assert oracle.count(g, algebra.from_canonical(key)) == c


def test_closed_forms_clique():
    n = 9
    g = graph_from_pairs(n, list(itertools.combinations(range(n), 2)))
    for k in (3, 4, 5):
        for m in algebra.connected_classes(k):
            p = pat(m, k)
            aut = len(algebra.automorphisms(p))
            expect_v = comb(n, k) if p.is_clique else 0
            assert oracle.count(g, p.with_induced(True)) == expect_v
            assert oracle.count(g, p) == comb(n, k) * factorial(k) // aut


def test_closed_forms_cycle_star_biclique():
    n = 11
    cyc = graph_from_pairs(n, [(i, (i + 1) % n) for i in range(n)])
    star = graph_from_pairs(n, [(0, i) for i in range(1, n)])
    a, b = 4, 5
    bic = graph_from_pairs(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    path = lambda k: Pattern(k, [(i, i + 1) for i in range(k - 1)])
    starp = lambda k: Pattern(k, [(0, i) for i in range(1, k)])
    for k in (3, 4, 5, 6):
        assert oracle.count(cyc, path(k).with_induced(True)) == n
        assert oracle.count(cyc, path(k)) == n
        assert oracle.count(star, starp(k).with_induced(True)) == comb(n - 1, k - 1)
        assert oracle.count(star, starp(k)) == comb(n - 1, k - 1)
    c4 = Pattern(4, [(0, 1), (1, 2), (2, 3), (3, 0)], vertex_induced=True)
    assert oracle.count(bic, c4) == comb(a, 2) * comb(b, 2)
    ring = Pattern(n, [(i, (i + 1) % n) for i in range(n)], vertex_induced=True) if n <= 8 else None
    c6 = graph_from_pairs(6, [(i, (i + 1) % 6) for i in range(6)])
    assert oracle.count(c6, Pattern(6, [(i, (i + 1) % 6) for i in range(6)], vertex_induced=True)) == 1


def test_morphed_equals_direct_and_root_additivity():
    s, d = rmat_edges(8, 8, seed=11)
    g = oracle.prepare_graph(256, s, d)
    for k in (3, 4):
        direct = oracle.motif_counts_direct(g, k)
        assert oracle.motif_counts_morphed(g, k) == direct
        # occurrences partition by their highest-ranked vertex
        parts = np.array_split(np.arange(g.n), 5)
        summed = np.sum([oracle.motif_counts_direct(g, k, roots=r) for r in parts], axis=0)
        assert list(summed) == direct


def test_relabel_invariance():
    s, d = rmat_edges(7, 8, seed=12)
    g = oracle.prepare_graph(128, s, d)
    perm = np.argsort(uniform_ints(3, 5, 128, 0, 1 << 30))
    g2 = oracle.prepare_graph(128, perm[s], perm[d])
    assert oracle.motif_counts_direct(g, 4) == oracle.motif_counts_direct(g2, 4)


# --------------------------------------------------------------- MNI
def test_domains_against_brute_force_maps():
    n = 9
    s, d = gnp_edges(n, 0.5, 21)
    labels = np.array([0, 1, 0, 1, 0, 1, 1, 0, 0])
    g = oracle.prepare_graph(n, s, d, labels)
    es = g.edge_set()
    for p in oracle.labeled_edge_patterns(2, [0, 1]) + oracle.labeled_edge_patterns(3, [0, 1])[:12]:
        ms = algebra.brute_force_matches(n, es, p, labels)
        dom = oracle.domains_direct(g, p)
        for u in range(p.k):
            assert set(np.nonzero(dom[u])[0]) == {m[u] for m in ms}


def test_mni_morphed_equals_direct_and_antimonotone():
    s, d = rmat_edges(8, 8, seed=13)
    labels = zipf_labels(256, 3, seed=14)
    g = oracle.prepare_graph(256, s, d, labels)
    for p in oracle.labeled_edge_patterns(3, [0, 1, 2])[:20]:
        dd = oracle.domains_direct(g, p)
        dm = oracle.domains_morphed(g, p)
        assert (dd == dm).all()
        sp = algebra.mni_support(p, dd)
        for sub in oracle.one_edge_smaller(p):
            assert sp <= oracle.support_direct(g, sub)
        assert sp <= min(int((labels == l).sum()) for l in p.labels)


def test_golden_rmat_s12_motifs():
    """Stored 4-motif counts of the scale-12 R-MAT graph (written by
    tests/golden/make_golden.py, which calls only the oracle); re-derive the
    cheap ones here: the vertex-induced star count from degrees is not
    closed-form, but the edge-induced star count is sum C(d, 3)."""
    path = os.path.join(GOLDEN, "rmat_s12_e8_seed1_motifs.json")
    gold = json.load(open(path))
    s, d = rmat_edges(12, 8, seed=1)
    g = oracle.prepare_graph(4096, s, d)
    deg = g.degree.astype(object)
    assert sum(int(x) * (int(x) - 1) * (int(x) - 2) // 6 for x in deg) == gold["edge_induced"]["4"][0]
    assert g.m == gold["m"]
