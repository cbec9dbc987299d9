"""GPU parity: the CUDA path through the C ABI against the oracle, bit-exact.

Counts and supports are integers, so every comparison is exact equality.
Sizes span many 32-edge task chunks with ragged tails; the full-size scale-20
graph is checked on sampled roots, whose counts the oracle computes exactly
(occurrences partition by their highest-ranked vertex)."""
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
from oracle import algebra
import paper_2012_04553_b300 as pm
from pm_inputs import rmat_edges, cached_rmat, gnp_edges, zipf_labels, uniform_ints

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def motif_queries(k, vi=True):
    return [pm.make_pattern(k, m, pm.VERTEX_INDUCED if vi else pm.EDGE_INDUCED)
            for m in algebra.connected_classes(k)]


def load(n, s, d, labels=None):
    return pm.Graph(n, s, d, labels)


def test_rmat_s12_4motifs_golden():
    gold = json.load(open(os.path.join(GOLDEN, "rmat_s12_e8_seed1_motifs.json")))
    s, d = rmat_edges(12, 8, seed=1)
    g = load(4096, s, d)
    assert g.info()["m"] == gold["m"]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        for k in (3, 4):
            assert pm.Plan(g, motif_queries(k), mode=mode).count() == gold["vertex_induced"][str(k)]
            assert pm.Plan(g, motif_queries(k, vi=False), mode=mode).count() == \
                gold["edge_induced"][str(k)]


def test_threaded_graph_build_against_oracle():
    """262144 raw edges (self-loops, duplicates and 15 vertices of degree
    >= 1024 among them): enough that the host builder splits the edge list
    over threads with per-thread row counts and cursors and builds the hub
    bitmaps in parallel. The simple-graph edge count, the dropped loops and
    duplicates, the maximum degree, the (degree, id) order and the
    3-vertex counts equal the oracle's."""
    n = 1 << 14
    s, d = rmat_edges(14, 16, seed=131)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    info = g.info()
    loops = int((np.asarray(s) == np.asarray(d)).sum())
    assert (info["m"], info["self_loops"], info["max_degree"]) == (og.m, loops, int(np.max(og.degree)))
    assert info["duplicates"] == len(s) - loops - og.m
    assert np.array_equal(g.vertex_order(), og.rank)
    want = [oracle.count(og, algebra.Pattern.from_mask(3, m)) for m in algebra.connected_classes(3)]
    assert pm.Plan(g, motif_queries(3, vi=False), mode=pm.MORPH_NONE).count() == want


@pytest.mark.parametrize("scale,ef,seed,kmax", [(7, 6, 100, 5), (8, 8, 101, 4), (9, 6, 102, 4),
                                                (10, 4, 103, 4)])
def test_motifs_small_rmat_against_oracle(scale, ef, seed, kmax):
    n = 1 << scale
    s, d = rmat_edges(scale, ef, seed=seed)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    for k in range(3, kmax + 1):
        want_v = oracle.motif_counts_direct(og, k)
        want_e = [oracle.count(og, algebra.Pattern.from_mask(k, m)) for m in algebra.connected_classes(k)]
        for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE, pm.MORPH_COST):
            for family in (pm.PLANS_AUTO, pm.PLANS_ROOTED, pm.PLANS_FREE):
                pv = pm.Plan(g, motif_queries(k), mode=mode)
                pv.select(family)
                assert pv.count() == want_v, (k, mode, family)
                pe = pm.Plan(g, motif_queries(k, False), mode=mode)
                pe.select(family)
                assert pe.count() == want_e, (k, mode, family)


def test_hub_bitmaps_against_oracle(monkeypatch):
    """Membership tests through hub adjacency bitmaps (every vertex of degree
    >= 16 gets one here) give the oracle's counts, rooted and free plans."""
    monkeypatch.setenv("PM_HUB_MIN_DEGREE", "16")
    n = 512
    s, d = rmat_edges(9, 8, seed=118)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    for k in (3, 4):
        want_v = oracle.motif_counts_direct(og, k)
        for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
            for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
                plan = pm.Plan(g, motif_queries(k), mode=mode)
                plan.select(family)
                assert plan.count() == want_v, (k, mode, family)


def two_hub_graph():
    """R-MAT scale 11 (ef 4, seed 119) plus a dense 16-vertex block and two
    adjacent hubs joined to the 1,100 common vertices 900..1999: the hubs'
    task has more common lower neighbours than the clique kernel's shared
    buffers hold, so its sets spill to global memory, and the 4-cycles
    through the hubs fill many wedge-kernel windows."""
    n = 2048
    s, d = rmat_edges(11, 4, seed=119)
    a, b = 2046, 2047
    extra_s, extra_d = [a], [b]
    for v in range(900, 2000):
        extra_s += [a, b]
        extra_d += [v, v]
    dense = uniform_ints(120, 1, 16 * 16, 0, 2)
    for i in range(16):
        for j in range(i + 1, 16):
            if dense[i * 16 + j]:
                extra_s.append(500 + i)
                extra_d.append(500 + j)
    s = np.concatenate([s, np.array(extra_s, dtype=s.dtype)])
    d = np.concatenate([d, np.array(extra_d, dtype=d.dtype)])
    return n, s, d


@pytest.mark.parametrize("balanced", ["0", "1"])
def test_clique_kernel_against_oracle(monkeypatch, balanced):
    """4- and 5-cliques through the clique kernel (rooted family; plain and
    balanced scheduling) and the set-operation kernel (free family), whole
    graph and a root subset, with the spill path exercised by two hubs of
    degree > 1,024."""
    monkeypatch.setenv("PM_CLIQUE_BALANCED", balanced)
    n, s, d = two_hub_graph()
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    assert g.info()["max_degree"] > 1024
    qs = [pm.make_pattern(4, 63), pm.make_pattern(5, 1023), pm.make_pattern(5, 1023, pm.VERTEX_INDUCED)]
    k4 = oracle.count(og, algebra.Pattern.from_mask(4, 63))
    k5 = oracle.count(og, algebra.Pattern.from_mask(5, 1023))
    want = [k4, k5, k5]                      # a clique's vertex- and edge-induced counts coincide
    assert k4 > 0 and k5 > 0
    for family in (pm.PLANS_ROOTED, pm.PLANS_FREE, pm.PLANS_AUTO):
        plan = pm.Plan(g, qs, mode=pm.MORPH_NONE)
        plan.select(family)
        assert plan.count() == want, family
    plan = pm.Plan(g, qs, mode=pm.MORPH_NONE)
    assert [r["kind"] for r in plan.export_plans(pm.PLANS_ROOTED)] == [2, 2]
    plan.select(pm.PLANS_ROOTED)
    counts, alg = plan.count_instrumented()
    assert counts == want and alg > 0
    roots = np.concatenate([np.arange(0, n, 7), [2046, 2047]]).astype(np.int32)
    r4, r5 = (oracle.count(og, algebra.Pattern.from_mask(k, m), roots=roots) for k, m in ((4, 63), (5, 1023)))
    assert plan.count_roots(roots) == [r4, r5, r5]


@pytest.mark.parametrize("heavy", ["0", "64", "100000"])
def test_wedge_heavy_and_light_roots(monkeypatch, heavy):
    """Edge-induced 4-cycles through the wedge kernels with every root light
    (dense global counters), the top 64 roots heavy (shared-memory windows),
    and every root heavy; whole graph twice (scratch left clean) and a root
    subset."""
    monkeypatch.setenv("PM_WEDGE_HEAVY", heavy)
    n, s, d = two_hub_graph()
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    c4 = algebra.Pattern.from_mask(4, 30)
    want = oracle.count(og, c4)
    plan = pm.Plan(g, [pm.make_pattern(4, 30)], mode=pm.MORPH_NONE)
    plan.select(pm.PLANS_ROOTED)
    assert plan.export_plans(pm.PLANS_ROOTED)[0]["kind"] == 1
    assert plan.count() == [want]
    assert plan.count() == [want]
    roots = np.concatenate([np.arange(1, n, 5), [2046, 2047]]).astype(np.int32)
    assert plan.count_roots(roots) == [oracle.count(og, c4, roots=roots)]


def test_six_vertex_patterns_against_oracle():
    s, d = rmat_edges(7, 5, seed=104)
    og = oracle.prepare_graph(128, s, d)
    g = load(128, s, d)
    masks = algebra.connected_classes(6)[::7]
    for vi in (False, True):
        qs = [pm.make_pattern(6, m, int(vi)) for m in masks]
        want = [oracle.count(og, algebra.Pattern.from_mask(6, m, None, vi)) for m in masks]
        for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
            for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
                plan = pm.Plan(g, qs, mode=mode)
                plan.select(family)
                assert plan.count() == want, (vi, family, mode)


def test_labeled_counts_against_oracle():
    n = 512
    s, d = rmat_edges(9, 8, seed=105)
    labels = zipf_labels(n, 3, seed=106)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    qs = oracle.labeled_edge_patterns(3, [0, 1, 2])[::3]
    cq = [pm.make_pattern(p.k, p.mask, pm.EDGE_INDUCED, p.labels) for p in qs]
    want = [oracle.count(og, p) for p in qs]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
            plan = pm.Plan(g, cq, mode=mode)
            plan.select(family)
            assert plan.count() == want
    vq = [pm.make_pattern(p.k, p.mask, pm.VERTEX_INDUCED, p.labels) for p in qs]
    want_v = [oracle.count(og, p.with_induced(True)) for p in qs]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        assert pm.Plan(g, vq, mode=mode).count() == want_v


def test_closed_form_graphs():
    # clique K_12, star S_40 and cycle C_50: closed forms of Section 2 counting
    cases = []
    n = 12
    a, b = np.triu_indices(n, 1)
    cases.append(("clique", n, a, b))
    cases.append(("star", 41, np.zeros(40, dtype=np.int32), np.arange(1, 41)))
    cases.append(("cycle", 50, np.arange(50), (np.arange(50) + 1) % 50))
    for name, n, s, d in cases:
        g = load(n, s, d)
        for k in (3, 4, 5):
            got_v = pm.Plan(g, motif_queries(k), mode=pm.MORPH_NAIVE).count()
            got_e = pm.Plan(g, motif_queries(k, False), mode=pm.MORPH_NONE).count()
            classes = algebra.connected_classes(k)
            for i, m in enumerate(classes):
                p = algebra.Pattern.from_mask(k, m)
                aut = len(algebra.automorphisms(p))
                degs = [sum(1 for e in p.edges if v in e) for v in range(k)]
                star = len(p.edges) == k - 1 and max(degs) == k - 1
                if name == "clique":
                    assert got_v[i] == (comb(n, k) if p.is_clique else 0)
                    assert got_e[i] == comb(n, k) * int(np.prod(range(1, k + 1))) // aut
                if name == "star":
                    assert got_v[i] == (comb(n - 1, k - 1) if star else 0)
                if name == "cycle":
                    is_path = len(p.edges) == k - 1 and max(degs) == 2
                    assert got_v[i] == (n if is_path else 0)


def test_edge_cases():
    # one vertex, no edges; only self-loops and duplicates; a single edge
    g = load(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert pm.Plan(g, motif_queries(4)).count() == [0] * 6
    g = load(5, np.array([0, 1, 2, 1, 1]), np.array([0, 2, 1, 2, 1]))
    info = g.info()
    assert (info["m"], info["self_loops"], info["duplicates"]) == (1, 2, 2)
    assert pm.Plan(g, [pm.make_pattern(2, 1)]).count() == [1]
    assert pm.Plan(g, motif_queries(3)).count() == [0, 0]
    with pytest.raises(pm.PMError):
        pm.Plan(g, [pm.make_pattern(3, 0b011, 0, [0, 1, 0])])   # labels on unlabeled graph
    with pytest.raises(pm.PMError):
        pm.Graph(4, np.array([0, 5]), np.array([1, 2]))         # id out of range


def test_root_subsets_partition_and_match_oracle():
    n = 2048
    s, d = rmat_edges(11, 8, seed=107)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    plan = pm.Plan(g, motif_queries(4), mode=pm.MORPH_NAIVE)
    total = plan.count()
    parts = np.array_split(np.arange(n, dtype=np.int32), 3)
    got = [plan.count_roots(p) for p in parts]
    assert [sum(x) for x in zip(*got)] == total
    roots = uniform_ints(9, 1, 64, 0, n).astype(np.int32)
    roots = np.unique(roots)
    assert plan.count_roots(roots) == oracle.motif_counts_direct(og, 4, roots=roots)
    assert plan.count_roots(np.zeros(0, np.int32)) == [0] * 6


def test_snake_shards_sum_to_whole_count():
    # the shards a multi-process run would count, summed here in one process
    from paper_2012_04553_b300 import shard
    n = 2048
    s, d = rmat_edges(11, 8, seed=108)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    plan = pm.Plan(g, motif_queries(4), mode=pm.MORPH_NAIVE)
    want = oracle.motif_counts_direct(og, 4)
    for world in (2, 3):
        matched = [plan.count_roots(shard.root_shard(g.vertex_order(), r, world), with_matched=True)[1]
                   for r in range(world)]
        total = [sum(x) % (1 << 128) for x in zip(*matched)]
        assert plan.morph(total) == want
    assert shard.count_sharded(plan, g, 0, 1) == want


def sampled_roots(deg, seed, count, max_degree):
    """Uniformly drawn vertices whose degree is at most max_degree (the oracle
    enumerates every automorphic copy, about degree^(k-1) maps per root)."""
    cand = np.nonzero(deg <= max_degree)[0]
    pick = uniform_ints(seed, 3, count, 0, len(cand))
    return np.unique(cand[pick]).astype(np.int32)


@pytest.fixture(scope="module")
def scale20():
    """The bench's graph: R-MAT scale 20, edge factor 16, seed 2 (oracle and library)."""
    s, d = cached_rmat(20, 16, seed=2)
    n = 1 << 20
    return oracle.prepare_graph(n, s, d), load(n, s, d)


def test_full_size_scale20_sampled_roots(scale20):
    """The scale-20 graph checked exactly on sampled roots through the rooted
    plans (uniform over vertices of degree <= 160 for 4-motifs, <= 40 for
    5-motifs), morphed and direct; 3-motifs also on a band of 32 hub roots
    (ranks 1,000-1,031 from the top, degree ~3,800, where the oracle's cost per
    root is about degree^2)."""
    og, g = scale20
    n = og.n
    roots = sampled_roots(og.degree, 2, 64, 160)
    want = oracle.motif_counts_direct(og, 4, roots=roots)
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        assert pm.Plan(g, motif_queries(4), mode=mode).count_roots(roots) == want
    roots5 = sampled_roots(og.degree, 3, 32, 40)
    want5 = oracle.motif_counts_direct(og, 5, roots=roots5)
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        assert pm.Plan(g, motif_queries(5), mode=mode).count_roots(roots5) == want5
    by_rank = np.argsort(og.rank)                # by_rank[r] = vertex of rank r
    band = by_rank[n - 1032:n - 1000]
    roots3 = np.unique(np.concatenate([band, sampled_roots(og.degree, 4, 32, 1 << 30)])).astype(np.int32)
    want3 = oracle.motif_counts_direct(og, 3, roots=roots3)
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        assert pm.Plan(g, motif_queries(3), mode=mode).count_roots(roots3) == want3


def test_full_size_scale20_closed_forms(scale20):
    """Whole-graph counts on the scale-20 graph through count(), in the
    bench's configuration (autotuned plan families, per-pattern launches)
    and with the free family forced: the edge-induced stars K1,2, K1,3, K1,4
    equal sum_v C(d_v, k-1) (computed from the oracle's degrees); the bench's
    4-motif plan reports the edge-induced K1,3 among its matched counts."""
    og, g = scale20
    deg = [int(x) for x in og.degree]
    stars = [pm.make_pattern(k, (1 << (k - 1)) - 1) for k in (3, 4, 5)]   # edges (0,1)..(0,k-1)
    want = [sum(comb(x, k - 1) for x in deg) for k in (3, 4, 5)]
    for family in (pm.PLANS_AUTO, pm.PLANS_FREE):
        plan = pm.Plan(g, stars, mode=pm.MORPH_NONE)
        plan.select(family)
        assert plan.count() == want, family
    bench = pm.Plan(g, motif_queries(4), mode=pm.MORPH_NAIVE)
    counts, matched = bench.count(with_matched=True)
    idx = [i for i, q in enumerate(bench.matched_patterns())
           if q[0] == 4 and bin(q[1]).count("1") == 3 and q[2] == pm.EDGE_INDUCED and
           max(bin(q[1] & m).count("1") for m in (0b000111, 0b011001, 0b101010, 0b110100)) == 3]
    assert len(idx) == 1 and matched[idx[0]] == want[1]
    assert all(c > 0 for c in counts)


def test_counts_beyond_2_64_on_stars():
    """Four disjoint stars with 2^17 leaves: the edge-induced 6-vertex star
    occurs 4 * C(2^17, 5) ~ 1.3e24 times (beyond 2^64: the 128-bit carries of
    the counter and of the warp sums), built from per-task binomials
    C(c, 4) whose falling product exceeds 2^64 (the long division); the
    5-vertex star gives 4 * C(2^17, 4).  Vertex-induced stars morphed from
    edge-induced superpatterns give the same counts (no edges among leaves)."""
    L = 1 << 17
    n = 4 * (L + 1)
    centres = np.repeat(np.arange(4) * (L + 1), L)
    leaves = centres + np.tile(np.arange(1, L + 1), 4)
    g = load(n, centres.astype(np.int32), leaves.astype(np.int32))
    want = [4 * comb(L, 4), 4 * comb(L, 5)]
    assert want[1] > 1 << 64
    ei = [pm.make_pattern(5, 0b1111), pm.make_pattern(6, 0b11111)]
    for family in (pm.PLANS_AUTO, pm.PLANS_ROOTED, pm.PLANS_FREE):
        plan = pm.Plan(g, ei, mode=pm.MORPH_NONE)
        plan.select(family)
        assert plan.count() == want, family
    vi = [pm.make_pattern(5, 0b1111, pm.VERTEX_INDUCED), pm.make_pattern(6, 0b11111, pm.VERTEX_INDUCED)]
    assert pm.Plan(g, vi, mode=pm.MORPH_NAIVE).count() == want


def test_mni_support_against_oracle():
    n = 512
    s, d = rmat_edges(9, 8, seed=108)
    labels = zipf_labels(n, 3, seed=109)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    qs = oracle.labeled_edge_patterns(3, [0, 1, 2])[::2] + oracle.labeled_edge_patterns(2, [0, 1, 2])
    cq = [pm.make_pattern(p.k, p.mask, pm.EDGE_INDUCED, p.labels) for p in qs]
    want = [oracle.support_direct(og, p) for p in qs]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE, pm.MORPH_COST):
        for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
            plan = pm.Plan(g, cq, op=pm.OP_SUPPORT, mode=mode)
            plan.select(family)
            sup, freq = plan.support(threshold=20)
            assert sup == want, (mode, family)
            assert freq == [w >= 20 for w in want]


def test_mni_domains_returned_in_caller_ids():
    """pm_support's domains_dev output: every query column as a bitset over
    the caller's vertex ids equals the union, over the column's orbit, of the
    oracle's per-vertex domains (all matches), morphed and direct."""
    n = 512
    s, d = rmat_edges(9, 8, seed=120)
    labels = zipf_labels(n, 3, seed=121)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    qs = oracle.labeled_edge_patterns(3, [0, 1, 2])[1::3] + oracle.labeled_edge_patterns(1, [0, 1])
    cq = [pm.make_pattern(p.k, p.mask, pm.EDGE_INDUCED, p.labels) for p in qs]
    want = []
    for p in qs:
        dom = oracle.domains_direct(og, p)
        want.append([np.logical_or.reduce([dom[u] for u in orb]) for orb in algebra.orbits(p)])
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        plan = pm.Plan(g, cq, op=pm.OP_SUPPORT, mode=mode)
        cols = plan.query_columns()
        sup, _, doms = plan.support(threshold=1, domains=True)
        for i, p in enumerate(qs):
            # library columns are orbits numbered by their smallest vertex, as algebra.orbits
            assert cols[i] == [next(c for c, orb in enumerate(algebra.orbits(p)) if u in orb)
                               for u in range(p.k)]
            words = doms[i].cpu().numpy().view(np.uint32)
            bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(len(words), -1)
            got = bits[:, :n].astype(bool)
            for c in range(len(want[i])):
                assert (got[c] == want[i][c]).all(), (mode, i, c)
            assert sup[i] == min(int(w.sum()) for w in want[i])


def test_sharded_mni_support_on_one_gpu():
    """Sharded MNI support (three root shards, their columns ORed by
    pm_domains_or) equals pm_support's supports and columns, morphed and
    direct; each shard's columns are the oracle's over its roots."""
    from paper_2012_04553_b300 import shard
    import torch
    n = 512
    s, d = rmat_edges(9, 8, seed=122)
    labels = zipf_labels(n, 3, seed=123)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    qs = oracle.labeled_edge_patterns(3, [0, 1, 2])[::4]
    cq = [pm.make_pattern(p.k, p.mask, pm.EDGE_INDUCED, p.labels) for p in qs]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        plan = pm.Plan(g, cq, op=pm.OP_SUPPORT, mode=mode)
        sup, freq, doms = plan.support(threshold=10, domains=True)
        parts = torch.stack([plan.support_roots(shard.root_shard(g.vertex_order(), r, 3)) for r in range(3)])
        cols = pm.domains_or(parts)
        assert torch.equal(cols, torch.cat(doms))
        assert plan.support_from_domains(cols, threshold=10) == (sup, freq)
        # shard 0's columns against the oracle's columns over its roots
        r0 = shard.root_shard(g.vertex_order(), 0, 3)
        at = 0
        words = parts[0].cpu().numpy().view(np.uint32)
        for p in qs:
            _, dom = oracle.match_count(og, p, roots=r0, domains=True)
            for orb in algebra.orbits(p):
                want = np.logical_or.reduce([dom[u] for u in orb])
                bits = ((words[at][:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n]
                assert (bits.astype(bool) == want).all()
                at += 1


def test_fsm_against_oracle():
    """Level-wise 3-edge FSM with MNI support (Section 2): the candidates of
    every level, their supports and the frequent sets, morphed and direct."""
    n = 512
    s, d = rmat_edges(9, 8, seed=112)
    labels = zipf_labels(n, 3, seed=113)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    threshold = 40
    want_last, want_levels = oracle.fsm(og, 3, threshold)
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE, pm.MORPH_COST):
        pats, sup, freq = pm.fsm(g, 3, threshold, mode=mode)
        got = {}
        for (k, mask, lab), sp, fr in zip(pats, sup, freq):
            key = algebra.canonical(algebra.Pattern.from_mask(k, mask, lab, False))
            got[key] = (sp, fr)
        edges = lambda key: len(key[2])
        assert {key: v[0] for key, v in got.items() if edges(key) == 3} == want_last
        for j, level in enumerate(want_levels, start=1):
            assert sorted(key for key, v in got.items() if edges(key) == j and v[1]) == level
        assert all(v[1] == (v[0] >= threshold) for v in got.values())


def test_batched_random_patterns_captured_graph():
    """A batch of random connected 3-6 vertex patterns (half vertex-induced,
    half edge-induced) counted in one plan, replayed from a captured CUDA
    graph, against the oracle."""
    from pm_inputs import random_patterns
    s, d = rmat_edges(7, 6, seed=114)
    og = oracle.prepare_graph(128, s, d)
    g = load(128, s, d)
    pats = random_patterns(48, seed=115)
    qs = [pm.make_pattern(k, m, ind) for k, m, ind in pats]
    want = [oracle.count(og, algebra.Pattern.from_mask(k, m, None, bool(ind))) for k, m, ind in pats]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        for launch in (pm.LAUNCH_PER_PATTERN, pm.LAUNCH_SINGLE):
            plan = pm.Plan(g, qs, mode=mode)
            plan.set_launch(launch)
            direct = plan.count()
            assert direct == want
            plan.capture()
            assert plan.count() == want
            assert plan.count() == want


def test_cost_mode_mixed_sets_and_labels():
    """Cost-based selection may mix direct and morphed patterns per query;
    whatever it picks, the counts are the oracle's (labeled, 4 and 5 vertices)."""
    n = 512
    s, d = rmat_edges(9, 8, seed=116)
    labels = zipf_labels(n, 2, seed=117)
    og = oracle.prepare_graph(n, s, d, labels)
    g = load(n, s, d, labels)
    qs = oracle.labeled_edge_patterns(3, [0, 1])[::2]
    for vi in (False, True):
        cq = [pm.make_pattern(p.k, p.mask, int(vi), p.labels) for p in qs]
        want = [oracle.count(og, p.with_induced(vi)) for p in qs]
        assert pm.Plan(g, cq, mode=pm.MORPH_COST).count() == want
    with pytest.raises(pm.PMError):
        pm.Plan(None, [pm.make_pattern(3, 0b011)], mode=pm.MORPH_COST)


def test_count_each_fails_only_queries_of_expired_patterns():
    """A deadline per matched pattern: the vertex-induced 5-star (leaf-wise
    differences on hubs, seconds of work here) runs out of its 0.5 s while the
    triangle and wedge queries of the same plan complete exactly."""
    s, d = rmat_edges(14, 16, seed=119)
    g = load(1 << 14, s, d)
    light = [pm.make_pattern(3, 0b111), pm.make_pattern(3, 0b011)]     # triangle, wedge
    heavy = [pm.make_pattern(5, 0b1111, pm.VERTEX_INDUCED)]              # 5-vertex star
    want = pm.Plan(g, light, mode=pm.MORPH_NONE).count()
    plan = pm.Plan(g, light + heavy, mode=pm.MORPH_NONE)
    plan.select(pm.PLANS_ROOTED)
    counts, status = plan.count_each(timeout_per_pattern_s=0.5, timeout_total_s=30.0)
    assert status == [pm.PM_OK, pm.PM_OK, pm.PM_ETIMEOUT]
    assert counts == want + [0]
    light_only = pm.Plan(g, light, mode=pm.MORPH_NONE)
    assert light_only.count_each(timeout_per_pattern_s=0.0) == (want, [pm.PM_OK, pm.PM_OK])


def test_autotune_choices_are_cached_per_graph():
    s, d = rmat_edges(11, 8, seed=111)
    g = load(2048, s, d)
    a = pm.Plan(g, motif_queries(4), mode=pm.MORPH_NAIVE)
    fam = a.autotune()
    assert len(fam) == a.n_matched and set(fam) <= {pm.PLANS_ROOTED, pm.PLANS_FREE, pm.PLANS_DECOMP}
    b = pm.Plan(g, motif_queries(4), mode=pm.MORPH_NAIVE)
    assert b.autotune() == fam
    assert a.count() == b.count()


def test_deadline_returns_timeout_and_context_survives():
    s, d = rmat_edges(14, 16, seed=110)
    g = load(1 << 14, s, d)
    heavy = pm.Plan(g, motif_queries(5), mode=pm.MORPH_NONE)
    with pytest.raises(pm.PMTimeout):
        heavy.count(timeout_s=1e-4)
    small = pm.Plan(g, motif_queries(3), mode=pm.MORPH_NAIVE)
    a = small.count()
    assert small.count(timeout_s=60.0) == a


def _occurrences(n, es, p, labels=None):
    """Distinct occurrences (edge sets) of p by brute force over injective maps."""
    out = set()
    for m in algebra.brute_force_matches(n, es, p, labels):
        out.add(frozenset(frozenset((m[a], m[b])) for a, b in p.edges) |
                frozenset([frozenset(m)]))
    return out


def test_enumerate_through_theorem_3_1():
    """pm_enumerate lists every occurrence exactly once: edge-induced queries
    from their vertex-induced superpatterns' matches composed with phi
    (Theorem 3.1), vertex-induced and clique queries directly; the listed
    edge sets equal brute force, with no repeats."""
    n = 20
    s, d = gnp_edges(n, 0.35, 124)
    og = oracle.prepare_graph(n, s, d)
    es = og.edge_set()
    g = load(n, s, d)
    qs = [algebra.Pattern.from_mask(4, m) for m in algebra.connected_classes(4)] + \
         [algebra.Pattern.from_mask(3, 0b011, vertex_induced=True),
          algebra.Pattern.from_mask(5, algebra.connected_classes(5)[7])]
    cq = [pm.make_pattern(p.k, p.mask, int(p.vertex_induced)) for p in qs]
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        # a vertex-induced query can be listed only as itself (no morphing)
        use = [i for i, p in enumerate(qs) if mode == pm.MORPH_NONE or not p.vertex_induced]
        plan = pm.Plan(g, [cq[i] for i in use], mode=mode)
        listed = [(use[q], t) for q, t in plan.enumerate(cap=16)]     # grows the buffer once
        for i in use:
            p = qs[i]
            got = [t for q, t in listed if q == i]
            occ = []
            for t in got:
                assert len(t) == p.k and len(set(t)) == p.k
                assert all((min(t[a], t[b]), max(t[a], t[b])) in es for a, b in p.edges)
                if p.vertex_induced:
                    assert all((min(t[a], t[b]), max(t[a], t[b])) not in es for a, b in p.anti_edges)
                occ.append(frozenset(frozenset((t[a], t[b])) for a, b in p.edges) | frozenset([frozenset(t)]))
            assert len(occ) == len(set(occ)), (mode, i)
            assert set(occ) == _occurrences(n, es, p), (mode, i)
    vi = pm.Plan(g, [pm.make_pattern(4, algebra.connected_classes(4)[0], pm.VERTEX_INDUCED)],
                 mode=pm.MORPH_NAIVE)
    with pytest.raises(pm.PMError) as e:
        vi.enumerate()
    assert e.value.status == pm.PM_EUNSUPPORTED


def test_batch_128_patterns_single_launch_with_deadlines():
    """128 random connected 3-6 vertex patterns (half vertex-, half
    edge-induced) on R-MAT scale 10 in one persistent launch, replayed from a
    captured CUDA graph with per-pattern deadlines: every status is OK, the
    3- and 4-vertex counts equal the oracle's, and every count equals the
    same plan run pattern by pattern."""
    from pm_inputs import random_patterns
    n = 1024
    s, d = rmat_edges(10, 4, seed=125)
    og = oracle.prepare_graph(n, s, d)
    g = load(n, s, d)
    pats = random_patterns(128, seed=126)
    qs = [pm.make_pattern(k, m, ind) for k, m, ind in pats]
    ref = pm.Plan(g, qs, mode=pm.MORPH_NAIVE)
    want = ref.count()
    small = [i for i, (k, _, _) in enumerate(pats) if k <= 4]
    for i in small:
        k, m, ind = pats[i]
        assert want[i] == oracle.count(og, algebra.Pattern.from_mask(k, m, None, bool(ind))), i
    plan = pm.Plan(g, qs, mode=pm.MORPH_NAIVE)
    plan.set_launch(pm.LAUNCH_SINGLE)
    plan.capture_each(timeout_per_pattern_s=120.0, timeout_total_s=600.0)
    for _ in range(2):
        counts, status = plan.count_each()
        assert status == [pm.PM_OK] * len(qs)
        assert counts == want


def test_single_launch_per_pattern_deadlines():
    """In the shared launch mode (one persistent launch per pattern size)
    every pattern's deadline runs from its launch's start: the
    vertex-induced 5-star (seconds of work here) is cut and reported, the
    triangle and wedge complete exactly, captured or not."""
    s, d = rmat_edges(14, 16, seed=119)
    g = load(1 << 14, s, d)
    light = [pm.make_pattern(3, 0b111), pm.make_pattern(3, 0b011)]
    heavy = [pm.make_pattern(5, 0b1111, pm.VERTEX_INDUCED)]
    want = pm.Plan(g, light, mode=pm.MORPH_NONE).count()
    plan = pm.Plan(g, light + heavy, mode=pm.MORPH_NONE)
    plan.select(pm.PLANS_FREE)
    plan.set_launch(pm.LAUNCH_SINGLE)
    counts, status = plan.count_each(timeout_per_pattern_s=0.5, timeout_total_s=30.0)
    assert status == [pm.PM_OK, pm.PM_OK, pm.PM_ETIMEOUT] and counts == want + [0]
    plan.capture_each(timeout_per_pattern_s=0.5, timeout_total_s=30.0)
    counts, status = plan.count_each()
    assert status == [pm.PM_OK, pm.PM_OK, pm.PM_ETIMEOUT] and counts == want + [0]


def test_cost_mode_never_slower_than_naive_or_direct():
    """Cost-based morph selection (Section 4.1 optimizer, Table 3) on a fixed
    graph: the set it picks for the 4-motif queries counts no slower than the
    naive morphed set or the direct set (median of 3 timed counts after
    warm-up; 50% tolerance plus 5 ms for timing noise), with equal counts."""
    import time as _t
    import torch
    s, d = rmat_edges(14, 16, seed=127)
    g = load(1 << 14, s, d)
    qs = motif_queries(4)
    times, counts = {}, {}
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE, pm.MORPH_COST):
        plan = pm.Plan(g, qs, mode=mode)
        counts[mode] = plan.count()                  # tuning and warm-up
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = _t.perf_counter()
            assert plan.count() == counts[mode]
            torch.cuda.synchronize()
            ts.append(_t.perf_counter() - t0)
        times[mode] = sorted(ts)[1]
    assert counts[pm.MORPH_COST] == counts[pm.MORPH_NAIVE] == counts[pm.MORPH_NONE]
    best = min(times[pm.MORPH_NONE], times[pm.MORPH_NAIVE])
    assert times[pm.MORPH_COST] <= 1.5 * best + 0.005, times


def test_injected_allocation_failure_is_a_status(monkeypatch):
    """PM_FAULT=alloc: every device allocation fails on the host side; loading
    and counting report PM_ENOMEM and the library stays usable afterwards."""
    s, d = rmat_edges(7, 6, seed=128)
    g = load(128, s, d)
    monkeypatch.setenv("PM_FAULT", "alloc")
    with pytest.raises(pm.PMError) as e:
        pm.Graph(128, s, d)
    assert e.value.status == pm.PM_ENOMEM
    plan = pm.Plan(g, motif_queries(3), mode=pm.MORPH_NAIVE)
    with pytest.raises(pm.PMError) as e:
        plan.count()
    assert e.value.status == pm.PM_ENOMEM
    monkeypatch.delenv("PM_FAULT")
    og = oracle.prepare_graph(128, s, d)
    assert pm.Plan(g, motif_queries(3), mode=pm.MORPH_NAIVE).count() == oracle.motif_counts_direct(og, 3)
