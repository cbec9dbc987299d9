"""GPU parity of the decomposition kernels (edge-induced counts of 4- and
5-vertex patterns from per-vertex, per-edge and per-2-path sums) against the
oracle, bit-exact, and against the set-operation plans on larger graphs.

The morphed 5-motif counts (Theorem 3.1 / Corollary 3.1 over edge-induced
counts, 15 of the 21 from the decomposition) are checked against the
oracle's direct vertex-induced counts."""
import numpy as np
import pytest

import oracle
from oracle import algebra
import paper_2012_04553_b300 as pm
from pm_inputs import rmat_edges, gnp_edges, uniform_ints, cached_rmat

pytestmark = pytest.mark.gpu

# canonical masks (lexicographic pair order) of the decomposed patterns
DECOMP4 = [7, 13, 15, 31, 63]                      # star, P4, tailed triangle, diamond, 4-clique
DECOMP5 = [15, 29, 58, 31, 59, 62, 185, 220, 63, 187, 207, 221, 127, 223, 191, 255, 1023,
           126, 254, 495, 511]   # K2,3, K2,3 plus an edge, 4-wheel, K5 minus an edge (neighbourhood graphs)
WHEEL5 = [126, 254, 495, 511]


def ei(k, m):
    return pm.make_pattern(k, m, pm.EDGE_INDUCED)


def decomp_queries():
    return [ei(4, m) for m in DECOMP4] + [ei(5, m) for m in DECOMP5]


def oracle_counts(og):
    return [oracle.count(og, algebra.Pattern.from_mask(4, m)) for m in DECOMP4] + \
           [oracle.count(og, algebra.Pattern.from_mask(5, m)) for m in DECOMP5]


def hub_graph():
    """R-MAT scale 7 plus two adjacent hubs sharing 60 neighbours and a dense
    12-vertex block: hub-heavy 2-path counters, large per-edge triangle
    counts, 4- and 5-cliques."""
    n = 128
    s, d = rmat_edges(7, 6, seed=301)
    extra_s, extra_d = [126], [127]
    for v in range(20, 80):
        extra_s += [126, 127]
        extra_d += [v, v]
    dense = uniform_ints(302, 1, 144, 0, 3)
    for i in range(12):
        for j in range(i + 1, 12):
            if dense[i * 12 + j]:
                extra_s.append(90 + i)
                extra_d.append(90 + j)
    return n, np.concatenate([s, np.array(extra_s, s.dtype)]), np.concatenate([d, np.array(extra_d, d.dtype)])


def graphs():
    out = []
    s, d = rmat_edges(8, 8, seed=303)
    out.append(("rmat8", 256, s, d))
    s, d = gnp_edges(40, 0.25, 304)
    out.append(("gnp40", 40, s, d))
    out.append(("hubs",) + hub_graph())
    return out


@pytest.mark.parametrize("name,n,s,d", graphs(), ids=lambda x: x if isinstance(x, str) else "")
def test_decomposition_against_oracle(name, n, s, d):
    og = oracle.prepare_graph(n, s, d)
    g = pm.Graph(n, s, d)
    want = oracle_counts(og)
    plan = pm.Plan(g, decomp_queries(), mode=pm.MORPH_NONE)
    fam = plan.autotune()
    assert set(fam) == {pm.PLANS_DECOMP}
    assert plan.count() == want
    assert plan.count() == want                      # scratch (2-path counters) left clean
    plan.capture()                                   # the whole count as one CUDA graph
    assert plan.count() == want
    one = [pm.Plan(g, [q], mode=pm.MORPH_NONE).count()[0] for q in decomp_queries()]
    assert one == want                               # each pattern alone (its own passes only)


@pytest.mark.parametrize("n", [24, 200, 800])
def test_decomposition_closed_forms_on_cliques(n):
    """On the complete graph K_n every connected k-vertex pattern occurs
    C(n, k) k! / |Aut(p)| times edge-induced.  n = 24 keeps every
    out-neighbourhood within one warp, n = 200 puts them in shared memory,
    n = 800 (out-degrees up to 799) in the per-block global area."""
    from math import comb, factorial
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s = np.array([a for a, _ in pairs], np.int32)
    d = np.array([b for _, b in pairs], np.int32)
    g = pm.Graph(n, s, d)
    want = []
    for k, masks in ((4, DECOMP4), (5, DECOMP5)):
        for m in masks:
            aut = len(algebra.automorphisms(algebra.Pattern.from_mask(k, m)))
            want.append(comb(n, k) * factorial(k) // aut)
    plan = pm.Plan(g, decomp_queries(), mode=pm.MORPH_NONE)
    assert plan.count() == want


def test_decomposition_equals_set_operations_scale11():
    """On R-MAT scale 11 (ef 8) the decomposition and the free-family set
    operations (two independent GPU algorithms) agree on every pattern."""
    s, d = rmat_edges(11, 8, seed=305)
    g = pm.Graph(2048, s, d)
    auto = pm.Plan(g, decomp_queries(), mode=pm.MORPH_NONE).count()
    free = pm.Plan(g, decomp_queries(), mode=pm.MORPH_NONE)
    free.select(pm.PLANS_FREE)
    assert free.count() == auto


@pytest.mark.parametrize("scale,ef,seed", [(7, 6, 306), (8, 6, 307)])
def test_five_motifs_morphed_with_decomposition(scale, ef, seed):
    """Vertex-induced 5-motifs via naive morphing (all 21 edge-induced counts
    from the decomposition) against the oracle's direct vertex-induced
    counts."""
    n = 1 << scale
    s, d = rmat_edges(scale, ef, seed=seed)
    og = oracle.prepare_graph(n, s, d)
    g = pm.Graph(n, s, d)
    qs = [pm.make_pattern(5, m, pm.VERTEX_INDUCED) for m in algebra.connected_classes(5)]
    plan = pm.Plan(g, qs, mode=pm.MORPH_NAIVE)
    assert set(plan.autotune()) == {pm.PLANS_DECOMP}
    assert plan.count() == oracle.motif_counts_direct(og, 5)


def test_decomposition_deadline_flags_its_patterns():
    """A per-pattern deadline too short for the decomposition passes marks
    every decomposed pattern as expired (and no other query), the 2-path
    scratch is left clean, and the context stays usable."""
    s, d = rmat_edges(16, 16, seed=308)
    g = pm.Graph(1 << 16, s, d)
    tri = pm.make_pattern(3, 0b111)
    qs = [tri, ei(5, 220), ei(5, 221)]
    want_tri = pm.Plan(g, [tri], mode=pm.MORPH_NONE).count()[0]
    plan = pm.Plan(g, qs, mode=pm.MORPH_NONE)
    counts, status = plan.count_each(timeout_per_pattern_s=1e-6, timeout_total_s=60.0)
    assert status[1:] == [pm.PM_ETIMEOUT, pm.PM_ETIMEOUT] and counts[1:] == [0, 0]
    full = pm.Plan(g, qs, mode=pm.MORPH_NONE).count()
    counts, status = plan.count_each(timeout_per_pattern_s=0.0)
    assert status == [pm.PM_OK] * 3 and counts == full and full[0] == want_tri


def test_decomposition_on_scale20_matches_free_plans():
    """On the bench's scale-20 graph, the decomposed patterns whose free
    set-operation plans finish in seconds (the 4-vertex star, path, tailed
    triangle, diamond and 4-clique; the 5-vertex star, fork, cricket and
    book) get the same counts both ways."""
    s, d = cached_rmat(20, 16, seed=2)
    g = pm.Graph(1 << 20, s, d)
    qs = [ei(4, m) for m in DECOMP4] + [ei(5, m) for m in (15, 29, 31, 127)]   # set operations finish
    auto = pm.Plan(g, qs, mode=pm.MORPH_NONE)
    got = auto.count()
    free = pm.Plan(g, qs, mode=pm.MORPH_NONE)
    free.select(pm.PLANS_FREE)
    assert free.count(timeout_s=120.0) == got


def test_decomposition_with_hub_bitmaps_everywhere(monkeypatch):
    """Adjacency bitmaps for every vertex of degree >= 3: the common-neighbour
    lists and mirror positions then come from the popcount rank index."""
    monkeypatch.setenv("PM_HUB_MIN_DEGREE", "3")
    n, s, d = hub_graph()
    og = oracle.prepare_graph(n, s, d)
    g = pm.Graph(n, s, d)
    qs = [ei(5, m) for m in WHEEL5] + [ei(4, 31), ei(5, 1023)]
    want = [oracle.count(og, algebra.Pattern.from_mask(5, m)) for m in WHEEL5] + \
           [oracle.count(og, algebra.Pattern.from_mask(4, 31)), oracle.count(og, algebra.Pattern.from_mask(5, 1023))]
    assert pm.Plan(g, qs, mode=pm.MORPH_NONE).count() == want


def big_hub_graph(n, p, seed):
    """A vertex adjacent to all n-1 others over a random graph on the rest
    (G(n-1, p), or about p*n*n/2 uniform pairs above 4096 vertices) with a
    dense 40-vertex block: one row far above 2048 positions (block tasks of
    the 4-wheel pass), many rims through the hub."""
    if n <= 4096:
        s, d = gnp_edges(n - 1, p, seed)
    else:
        m = int(p * n * n / 2)
        s, d = uniform_ints(seed, 3, m, 0, n - 1), uniform_ints(seed, 4, m, 0, n - 1)
    dense = uniform_ints(seed + 1, 1, 40 * 40, 0, 2)
    bs = [10 + i for i in range(40) for j in range(i + 1, 40) if dense[i * 40 + j]]
    bd = [10 + j for i in range(40) for j in range(i + 1, 40) if dense[i * 40 + j]]
    S = np.concatenate([s.astype(np.int32) + 1, np.array(bs, np.int32), np.zeros(n - 1, np.int32)])
    D = np.concatenate([d.astype(np.int32) + 1, np.array(bd, np.int32), np.arange(1, n, dtype=np.int32)])
    return S, D


def wheel_vs_plans(g, masks, families=(pm.PLANS_FREE, pm.PLANS_ROOTED)):
    qs = [ei(5, m) for m in masks]
    dec = pm.Plan(g, qs, mode=pm.MORPH_NONE)
    dec.select(pm.PLANS_DECOMP)
    got = dec.count()
    for fam in families:
        other = pm.Plan(g, qs, mode=pm.MORPH_NONE)
        other.select(fam)
        assert other.count(timeout_s=300.0) == got, fam
    return got


@pytest.mark.parametrize("which", ["rmat14", "hub2600"])
def test_wheel_block_tasks_match_set_operations(which):
    """Rows of more than 2048 positions (shared-memory block tasks of the
    4-wheel pass, hub roots of the K2,3 pass) against the free and rooted
    set-operation plans."""
    if which == "rmat14":
        s, d = rmat_edges(14, 16, seed=309)
        n = 1 << 14
    else:
        n = 2600
        s, d = big_hub_graph(n, 0.004, 310)
    g = pm.Graph(n, s, d)
    assert g.info()["max_degree"] > 2048
    got = wheel_vs_plans(g, WHEEL5)
    assert all(c > 0 for c in got)


def test_wheel_global_counters_above_65536_positions():
    """A row of 70000 positions: 4-wheel tasks beyond 65536 positions use the
    per-block global counters, and the K2,3 pass its 32/64-bit counters (a
    degree above 65535 rules out the 16/32-bit ones)."""
    n = 70001
    s, d = big_hub_graph(n, 5.0 / n, 311)
    g = pm.Graph(n, s, d)
    assert g.info()["max_degree"] == n - 1
    got = wheel_vs_plans(g, [495, 126, 254], families=(pm.PLANS_FREE,))
    assert all(c > 0 for c in got)


def test_bounds_checked_build_agrees_with_the_oracle():
    """The PM_DEBUG library (every data-derived index checked before its
    access, a failed check reported as an error) counts the hub graph's
    decomposed patterns, the neighbourhood-graph ones included, exactly as
    the oracle, in a child process that loads it."""
    import json
    import os
    import subprocess
    import sys
    n, s, d = hub_graph()
    og = oracle.prepare_graph(n, s, d)
    masks5 = [220, 221] + WHEEL5
    want = [oracle.count(og, algebra.Pattern.from_mask(5, m)) for m in masks5]
    code = (
        "import json, numpy as np, paper_2012_04553_b300 as pm\n"
        "from tests.test_gpu_decomp import hub_graph\n"
        "assert pm.LIB_PATH.endswith('libpm_b300_debug.so')\n"
        "n, s, d = hub_graph()\n"
        "g = pm.Graph(n, s, d)\n"
        f"qs = [pm.make_pattern(5, m, pm.EDGE_INDUCED) for m in {masks5!r}]\n"
        "print(json.dumps([str(c) for c in pm.Plan(g, qs, mode=pm.MORPH_NONE).count()]))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PM_DEBUG="1", PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    got = [int(x) for x in json.loads(out.stdout.strip().splitlines()[-1])]
    assert got == want
