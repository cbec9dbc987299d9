"""CPU oracle for pattern morphing: plain, slow, independent of the CUDA path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import, call, link or run anything in this
package.  It shares no code with the library: graph preparation, the pattern
algebra (oracle/algebra.py) and the matcher (oracle/match.c) are written here
from the paper's definitions.

What it computes (counts are distinct subgraphs = matches / |Aut(p)|):
* count(p) for a vertex- or edge-induced, optionally labeled pattern
  (Section 2 match definition), optionally restricted to occurrences whose
  highest-ranked vertex is in a root set, rank ordering vertices by
  (degree, vertex id);
* k-motif counts directly and through morphing (Theorem 3.1, Corollary 3.1);
* MNI domains and supports (Section 2, FSM) directly and through morphing
  (Theorem 3.2);
* level-wise frequent subgraph mining with MNI support.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

from . import algebra
from .algebra import Pattern

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_match.so")
_lib = None


def build(force=False):
    """Compile match.c (gcc, OpenMP) into oracle/_match.so."""
    src = os.path.join(_HERE, "match.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _SO, src])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.orc_count.restype = ctypes.c_int
        lib.orc_count.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_set_budget.restype = None
        lib.orc_set_budget.argtypes = [ctypes.c_double]
        _lib = lib
    return _lib


def max_threads():
    return _load().orc_max_threads()


class OracleTimeout(RuntimeError):
    """The wall-clock budget set with set_budget() ran out during a count."""


def set_budget(seconds):
    """Wall-clock budget (from now) for the following counts; 0 = none.  A
    count still running when it passes raises OracleTimeout."""
    _load().orc_set_budget(float(seconds))


class Graph:
    """Undirected simple graph as CSR with sorted rows (vertex ids as given)."""

    def __init__(self, n, rowptr, col, labels=None):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
        deg = np.diff(self.rowptr)
        # rank: position in the order by (degree, vertex id), ascending
        order = np.lexsort((np.arange(self.n), deg))
        self.rank = np.empty(self.n, dtype=np.int64)
        self.rank[order] = np.arange(self.n)
        self.degree = deg

    @property
    def m(self):
        return len(self.col) // 2

    def edge_set(self):
        s = set()
        for v in range(self.n):
            for x in self.col[self.rowptr[v]:self.rowptr[v + 1]]:
                if v < x:
                    s.add((v, int(x)))
        return s


def prepare_graph(n, src, dst, labels=None):
    """Drop self-loops, make undirected, drop duplicates, sort each row."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    a = np.concatenate([src[keep], dst[keep]])
    b = np.concatenate([dst[keep], src[keep]])
    key = np.unique(a * n + b)
    rows, cols = key // n, key % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Graph(n, rowptr, cols.astype(np.int32), labels)


def _relation_arrays(p):
    rel = np.array(p.relation(), dtype=np.int8).reshape(-1)
    plab = np.array(p.labels, dtype=np.int32)
    return rel, plab


def match_count(g, p, roots=None, threads=0, domains=False):
    """Number of matches (injective maps) of p; with roots, only those whose
    highest-ranked image vertex is in roots.  Optionally also per-vertex domains
    (k x n boolean array: dom[u, x] = some match sends u to x)."""
    lib = _load()
    rel, plab = _relation_arrays(p)
    out = np.zeros(2, dtype=np.uint64)
    r = None if roots is None else np.ascontiguousarray(roots, dtype=np.int32)
    dom = np.zeros((p.k, g.n), dtype=np.uint8) if domains else None
    if p.labels is not None and any(x >= 0 for x in p.labels) and g.labels is None:
        raise ValueError("labeled pattern on an unlabeled graph")
    rc = lib.orc_count(
        g.n, g.rowptr.ctypes.data, g.col.ctypes.data,
        None if g.labels is None else g.labels.ctypes.data, g.rank.ctypes.data,
        p.k, rel.ctypes.data, plab.ctypes.data,
        0 if r is None else len(r), None if r is None else r.ctypes.data,
        int(threads), out.ctypes.data, None if dom is None else dom.ctypes.data)
    if rc == -2:
        raise OracleTimeout("oracle budget expired")
    if rc != 0:
        raise ValueError(f"orc_count rejected pattern {p}")
    total = int(out[0]) | (int(out[1]) << 64)
    return (total, dom.astype(bool)) if domains else total


def count(g, p, roots=None, threads=0):
    """Distinct occurrences of p = matches / |Aut(p)| (exact Python int)."""
    total = match_count(g, p, roots, threads)
    aut = len(algebra.automorphisms(p))
    assert total % aut == 0, (p, total, aut)
    return total // aut


# ---------------------------------------------------------------------------
# Motif counting (Section 2, Motif Counting): all connected k-vertex
# vertex-induced unlabeled patterns, in algebra.connected_classes(k) order.

def motif_patterns(k):
    return [Pattern.from_mask(k, m, vertex_induced=True) for m in algebra.connected_classes(k)]


def motif_counts_direct(g, k, roots=None, threads=0):
    return [count(g, p, roots, threads) for p in motif_patterns(k)]


def motif_counts_morphed(g, k, roots=None, threads=0):
    """Count the edge-induced variant of every motif (cliques are both), then
    recover the vertex-induced counts with Corollary 3.1 applied recursively."""
    ei = {}

    def count_E(pe):
        key = algebra.canonical(pe)
        if key not in ei:
            ei[key] = count(g, pe, roots, threads)
        return ei[key]

    memo = {}
    return [algebra.count_V_from_E(p, count_E, memo) for p in motif_patterns(k)]


# ---------------------------------------------------------------------------
# MNI support (Section 2, FSM).

def domains_direct(g, p, threads=0):
    """Per-vertex MNI domains of p from all of its matches (k x n booleans)."""
    _, dom = match_count(g, p, None, threads, domains=True)
    return dom


def support_direct(g, p, threads=0):
    return algebra.mni_support(p, domains_direct(g, p, threads))


def domains_morphed(g, p, threads=0):
    """Domains of p^E from the vertex-induced superpatterns (Theorem 3.2)."""
    cache = {}

    def dv(q):
        key = algebra.canonical(q)
        if key not in cache:
            cache[key] = domains_direct(g, q, threads)
        return cache[key]

    return np.array(algebra.mni_E_from_V(p, dv))


def support_morphed(g, p, threads=0):
    return algebra.mni_support(p, domains_morphed(g, p, threads))


def labeled_edge_patterns(n_edges, labels_allowed):
    """Every connected labeled pattern with n_edges edges over the allowed
    labels, one per isomorphism class (edge-induced)."""
    out = {}
    for k in range(2, n_edges + 2):
        for m in algebra.connected_classes(k):
            if bin(m).count("1") != n_edges:
                continue
            for lab in itertools.product(labels_allowed, repeat=k):
                p = Pattern.from_mask(k, m, lab, False)
                out.setdefault(algebra.canonical(p), p)
    return [out[key] for key in sorted(out)]


def fsm(g, n_edges, threshold, threads=0, morphed=False):
    """Level-wise frequent subgraph mining with MNI support.

    Level 1: every labeled edge.  Level j+1 candidates: connected labeled
    patterns with j+1 edges all of whose connected j-edge subpatterns (remove
    one edge, drop an isolated vertex) are frequent; anti-monotonicity of MNI
    (Section 2) makes this lose no frequent pattern.  Returns
    {canonical key: support} for every candidate of the last level and the
    list of frequent keys at each level."""
    labels_present = sorted(set(int(x) for x in np.unique(g.labels)))
    supp_fn = support_morphed if morphed else support_direct
    frequent_prev = None
    levels = []
    cand_support = {}
    for j in range(1, n_edges + 1):
        cand_support = {}
        for p in labeled_edge_patterns(j, labels_present):
            if frequent_prev is not None:
                if not all(algebra.canonical(s) in frequent_prev for s in one_edge_smaller(p)):
                    continue
            cand_support[algebra.canonical(p)] = supp_fn(g, p, threads)
        frequent_prev = {key for key, s in cand_support.items() if s >= threshold}
        levels.append(sorted(frequent_prev))
    return cand_support, levels


def one_edge_smaller(p):
    """Connected subpatterns of p with one edge fewer (isolated vertex dropped)."""
    out = []
    for e in p.edges:
        rest = [x for x in p.edges if x != e]
        used = sorted({v for x in rest for v in x}) if rest else []
        if len(rest) == 0:
            continue
        ren = {v: i for i, v in enumerate(used)}
        q = Pattern(len(used), [(ren[a], ren[b]) for a, b in rest],
                    [p.labels[v] for v in used], False)
        if q.connected():
            out.append(q)
    return out
