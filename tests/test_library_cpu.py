"""CPU tests of the library (no GPU): the C ABI loads and exports every
declared symbol, compiled plans count correctly (checked with a plain-Python
interpreter of the plan semantics against the oracle), and the host morph
transform recovers oracle results."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from oracle import algebra
import paper_2012_04553_b300 as pm
from pm_inputs import rmat_edges, gnp_edges, zipf_labels
from tests.plan_interp import degree_ordered, run_plans

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    return sorted(set(re.findall(r"^(?:pm_status|void|const char \*)\s*(pm_\w+)\s*\(", text, re.M)))


def test_abi_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(pm.lib(), name), name
    assert sorted(pm.ABI_SYMBOLS) == names


def test_errors_are_statuses_not_aborts():
    disconnected = pm.make_pattern(4, 0b100001)  # edges (0,1) and (2,3)
    with pytest.raises(pm.PMError) as e:
        pm.Plan(None, [disconnected])
    assert e.value.status == pm.PM_EINVAL
    with pytest.raises(pm.PMError):
        pm.Plan(None, [pm.make_pattern(1, 0)])
    with pytest.raises(pm.PMError):
        pm.Plan(None, [pm.make_pattern(3, 1 << 5)])
    p = pm.Plan(None, [pm.make_pattern(3, 0b111)])
    with pytest.raises(pm.PMError) as e:
        p.count()
    assert e.value.status == pm.PM_EINVAL
    assert pm.lib().pm_strerror(pm.PM_ETIMEOUT) == b"deadline expired"


def pats(k, vi):
    return [pm.make_pattern(k, m, pm.VERTEX_INDUCED if vi else pm.EDGE_INDUCED)
            for m in algebra.connected_classes(k)]


def oracle_pattern(k, mask, induced, labels=None):
    return algebra.Pattern.from_mask(k, mask, labels, induced == pm.VERTEX_INDUCED)


@pytest.fixture(scope="module")
def small_graph():
    s, d = rmat_edges(6, 6, seed=31)
    return oracle.prepare_graph(64, s, d)


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("vi", [False, True])
@pytest.mark.parametrize("family", [pm.PLANS_ROOTED, pm.PLANS_FREE])
def test_plans_count_matched_patterns(small_graph, k, vi, family):
    g = small_graph
    adj, labels = degree_ordered(g)
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        plan = pm.Plan(None, pats(k, vi), mode=mode)
        got = run_plans(plan.export_plans(family), plan.n_matched, adj, labels)
        for (kk, mask, ind, lab), c in zip(plan.matched_patterns(), got):
            assert c == oracle.count(g, oracle_pattern(kk, mask, ind)), (kk, mask, ind, mode)


def test_free_plans_shapes():
    # diamond: chord rooted, the two degree-2 vertices a binomial tail of 2;
    # paw: rooted at the degree-3 vertex with a closed single-vertex tail
    diamond = pm.Plan(None, [pm.make_pattern(4, 31)], mode=pm.MORPH_NONE).export_plans(pm.PLANS_FREE)[0]
    assert (diamond["tail"], diamond["task_space"]) == (2, 1)
    paw = pm.Plan(None, [pm.make_pattern(4, 15)], mode=pm.MORPH_NONE).export_plans(pm.PLANS_FREE)[0]
    assert (paw["tail"], paw["closed"], paw["task_space"]) == (1, 1, 2)


def test_morph_transform_recovers_requested(small_graph):
    g = small_graph
    adj, labels = degree_ordered(g)
    for k in (4, 5):
        for vi in (False, True):
            plan = pm.Plan(None, pats(k, vi), mode=pm.MORPH_NAIVE)
            matched = run_plans(plan.export_plans(), plan.n_matched, adj, labels)
            want = [oracle.count(g, algebra.Pattern.from_mask(k, m, None, vi))
                    for m in algebra.connected_classes(k)]
            assert plan.morph(matched) == want


def test_plans_root_partition(small_graph):
    g = small_graph
    adj, labels = degree_ordered(g)
    plan = pm.Plan(None, pats(4, True), mode=pm.MORPH_NAIVE)
    tbl = plan.export_plans()
    roots_caller = np.arange(0, g.n, 3)
    roots_internal = [int(g.rank[v]) for v in roots_caller]
    part = plan.morph(run_plans(tbl, plan.n_matched, adj, labels, roots=roots_internal))
    want = oracle.motif_counts_direct(g, 4, roots=roots_caller)
    assert part == want


def test_labeled_plans(small_graph):
    s, d = gnp_edges(14, 0.45, seed=8)
    labels = np.array([0, 1, 2, 0, 1, 0, 0, 2, 1, 0, 1, 0, 2, 0])
    g = oracle.prepare_graph(14, s, d, labels)
    adj, lab = degree_ordered(g)
    queries = oracle.labeled_edge_patterns(3, [0, 1])
    for mode in (pm.MORPH_NONE, pm.MORPH_NAIVE):
        for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
            cq = [pm.make_pattern(p.k, p.mask, pm.EDGE_INDUCED, p.labels) for p in queries]
            plan = pm.Plan(None, cq, mode=mode)
            matched = run_plans(plan.export_plans(family), plan.n_matched, adj, lab)
            assert plan.morph(matched) == [oracle.count(g, p) for p in queries]


def test_six_vertex_plans_on_tiny_graph():
    s, d = gnp_edges(11, 0.5, seed=41)
    g = oracle.prepare_graph(11, s, d)
    adj, labels = degree_ordered(g)
    masks = algebra.connected_classes(6)[::9]
    for vi in (False, True):
        for family in (pm.PLANS_ROOTED, pm.PLANS_FREE):
            plan = pm.Plan(None, [pm.make_pattern(6, m, int(vi)) for m in masks], mode=pm.MORPH_NONE)
            got = plan.morph(run_plans(plan.export_plans(family), plan.n_matched, adj, labels))
            assert got == [oracle.count(g, algebra.Pattern.from_mask(6, m, None, vi)) for m in masks]


def test_morph_coefficients_match_oracle_algebra():
    # the library's transform applied to symbolic vertex-induced counts gives the
    # edge-induced counts of the oracle's Theorem 3.1 implementation
    rng = np.random.default_rng(3)
    for k in (4, 5):
        plan = pm.Plan(None, pats(k, False), mode=pm.MORPH_NAIVE)
        matched = plan.matched_patterns()
        vals = {}
        for (kk, mask, ind, lab) in matched:
            vals[algebra.canonical(oracle_pattern(kk, mask, pm.VERTEX_INDUCED))] = int(rng.integers(0, 10**9))
        cv = lambda q: vals[algebra.canonical(q.with_induced(True))]
        got = plan.morph([vals[algebra.canonical(oracle_pattern(kk, mask, pm.VERTEX_INDUCED))]
                          for (kk, mask, ind, lab) in matched])
        want = [algebra.count_E_from_V(algebra.Pattern.from_mask(k, m), cv)
                for m in algebra.connected_classes(k)]
        assert got == want


def test_morph_is_modulo_2_128():
    plan = pm.Plan(None, pats(4, True), mode=pm.MORPH_NAIVE)
    big = [(1 << 127) + 12345] * plan.n_matched
    out = plan.morph(big)
    assert all(0 <= x < (1 << 128) for x in out)


def test_special_plan_kinds():
    # counting: the 4-cycle's rooted plan runs the wedge kernel, the 4- and
    # 5-clique's the clique kernel; MNI support keeps set-operation plans
    qs = [pm.make_pattern(4, 30), pm.make_pattern(4, 63), pm.make_pattern(5, 1023),
          pm.make_pattern(6, (1 << 15) - 1), pm.make_pattern(4, 31)]
    plan = pm.Plan(None, qs, mode=pm.MORPH_NONE)
    matched = plan.matched_patterns()
    kinds = {}
    for r in plan.export_plans(pm.PLANS_ROOTED):
        k, m = matched[int(r["counter"])][:2]
        kinds.setdefault((k, m), set()).add(int(r["kind"]))
    kinds = {key: v.pop() if len(v) == 1 else v for key, v in kinds.items()}
    assert kinds == {(4, 30): 1, (4, 63): 2, (5, 1023): 2, (6, (1 << 15) - 1): 0, (4, 31): 0}
    assert all(int(r["kind"]) == 0 for r in plan.export_plans(pm.PLANS_FREE))
    sup = pm.Plan(None, qs[:3], op=pm.OP_SUPPORT, mode=pm.MORPH_NONE)
    assert all(int(r["kind"]) == 0 for r in sup.export_plans(pm.PLANS_ROOTED))


def _permuted(k, mask, labels, perm):
    """The pattern with vertex v renamed perm[v] (mask over pairs a < b)."""
    pairs = [(a, b) for a in range(k) for b in range(a + 1, k)]
    index = {p: i for i, p in enumerate(pairs)}
    out = 0
    for i, (a, b) in enumerate(pairs):
        if mask >> i & 1:
            x, y = sorted((perm[a], perm[b]))
            out |= 1 << index[(x, y)]
    lab = [-1] * k
    for v in range(k):
        lab[perm[v]] = labels[v]
    return out, lab


def test_canonical_labelling_is_a_class_function():
    # the library's canonical form (least labels/mask over the relabelings
    # ordered by a vertex invariant) must name isomorphism classes exactly:
    # all connected graphs on k <= 6 vertices give 2 / 6 / 21 / 112 classes
    # (OEIS A001349), and random labeled patterns keep their class under
    # random relabelings and split into exactly the oracle's classes
    for k, want in ((3, 2), (4, 6), (5, 21), (6, 112)):
        qs = [pm.make_pattern(k, m) for m in range(1 << (k * (k - 1) // 2))
              if algebra.Pattern.from_mask(k, m).connected()]
        assert pm.Plan(None, qs, mode=pm.MORPH_NONE).n_matched == want
    rng = np.random.default_rng(17)
    from pm_inputs import random_patterns
    pool = random_patterns(300, kmin=3, kmax=7, seed=18)
    lib_q, keys = [], set()
    for k, m, ind in pool:
        labels = [int(x) for x in rng.integers(-1, 2, size=k)]
        perm = [int(x) for x in rng.permutation(k)]
        m2, l2 = _permuted(k, m, labels, perm)
        a = pm.make_pattern(k, m, ind, labels)
        b = pm.make_pattern(k, m2, ind, l2)
        assert pm.Plan(None, [a, b], mode=pm.MORPH_NONE).n_matched == 1
        lib_q.append(a)
        op = algebra.Pattern.from_mask(k, m, labels, bool(ind))
        # a clique's vertex- and edge-induced forms are one pattern
        keys.add(algebra.canonical(op.with_induced(False) if op.is_clique else op))
    assert pm.Plan(None, lib_q, mode=pm.MORPH_NONE).n_matched == len(keys)


def test_host_fault_injection(monkeypatch):
    """PM_FAULT makes graph loading and planning fail with their statuses and
    an explanatory error text, before any device work."""
    monkeypatch.setenv("PM_FAULT", "plan")
    with pytest.raises(pm.PMError) as e:
        pm.Plan(None, [pm.make_pattern(3, 0b111)])
    assert e.value.status == pm.PM_EUNSUPPORTED and "fault injected" in str(e.value)
    monkeypatch.setenv("PM_FAULT", "load")
    with pytest.raises(pm.PMError) as e:
        pm.Graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    assert e.value.status == pm.PM_EINVAL and "fault injected" in str(e.value)
    monkeypatch.delenv("PM_FAULT")
    assert pm.Plan(None, [pm.make_pattern(3, 0b111)]).n_matched == 1


def test_debug_build_exports_the_same_symbols():
    """The PM_DEBUG (bounds-checked) library builds for sm_103a and exports
    the same C ABI as the release library."""
    import runpy
    import subprocess
    here = os.path.dirname(os.path.abspath(pm.__file__))
    mod = runpy.run_path(os.path.join(here, "build.py"))
    rel, dbg = mod["build"](), mod["build"](debug=True)

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
        return {line.split()[-1] for line in out.splitlines() if line.split()[-1].startswith("pm_")}
    assert exported(dbg) == exported(rel)
    assert set(pm.ABI_SYMBOLS) <= exported(dbg)
