"""Test-only interpreter of the library's compiled matching plans, in plain
Python sets, so plan compilation (orbit roots, symmetry-breaking order
constraints, injectivity, shared tails) is checked on the CPU against the
oracle before any kernel runs.  It executes the plan semantics documented in
paper_2012_04553_b300/csrc/plan.hpp and is never used by the library."""
from math import comb

import numpy as np


def degree_ordered(g):
    """CSR of the oracle graph g renumbered by rank (degree, id) ascending."""
    n = g.n
    adj = [set() for _ in range(n)]
    for v in range(n):
        rv = int(g.rank[v])
        for x in g.col[g.rowptr[v]:g.rowptr[v + 1]]:
            adj[rv].add(int(g.rank[x]))
    labels = None
    if g.labels is not None:
        labels = np.empty(n, dtype=np.int64)
        labels[g.rank] = g.labels
    return adj, labels


def _bits(mask):
    return [j for j in range(8) if (mask >> j) & 1]


def run_plans(plans, n_matched, adj, labels, roots=None):
    counts = [0] * n_matched
    n = len(adj)
    for P in plans:
        k, n_enum, tail = int(P["k"]), int(P["n_enum"]), int(P["tail"])
        lv = P["lv"]

        def candidates(L, m):
            d = lv[L]
            lo = max([m[j] for j in _bits(d["gt"])], default=-1)
            # (levels 1+ of every plan intersect at least one earlier list)
            hi = min([m[j] for j in _bits(d["lt"])], default=n)
            c = set.intersection(*[adj[m[j]] for j in _bits(d["isect"])])
            for j in _bits(d["diff"]):
                c = c - adj[m[j]]
            c = c - {m[j] for j in _bits(d["neq"])}
            out = [x for x in c if lo < x < hi and (d["label"] < 0 or labels[x] == d["label"])]
            return sorted(out)

        pair = int(P["pair"]) if "pair" in P.dtype.names else 0

        def dfs(L, m):
            if L == n_enum and pair:
                A = candidates(L, m)
                B = candidates(L + 1, m + [None])   # level L+1 has no constraint on level L
                return len(A) * len(B) - len(set(A) & set(B))
            if L == n_enum:
                if tail == 0:
                    return 1
                return comb(len(candidates(L, m)), tail)
            total = 0
            for x in candidates(L, m):
                total += dfs(L + 1, m + [x])
            return total

        space = int(P["task_space"])   # 0: v1 < root, 1: v1 > root, 2: any neighbour
        for root in (range(n) if roots is None else roots):
            if lv[0]["label"] >= 0 and labels[root] != lv[0]["label"]:
                continue
            for v1 in sorted(adj[root]):
                if (space == 0 and v1 >= root) or (space == 1 and v1 <= root):
                    continue
                if lv[1]["label"] >= 0 and labels[v1] != lv[1]["label"]:
                    continue
                counts[int(P["counter"])] += dfs(2, [root, v1])
    return counts
