"""Graph preparation (Section 2's data graph as the matching kernels read it)
on the host alone, through pm_prepare_csr, against the oracle's graph: the
library's CSR must be the oracle's simple graph (self-loops and duplicates
dropped, both directions) with vertices renumbered by (degree, id) ascending
and every row sorted, entry for entry.  The expected arrays are the oracle's
CSR permuted here by the oracle's own rank; nothing runs on a GPU.

The cases reach every branch of the builder: one thread and several (edge
lists above 2 * 65536 entries are split over threads), rows sorted by
comparison (fewer than 128 ids) and by radix sort with an even and an odd
number of 8-bit passes, hub rows, and the degenerate inputs."""
import numpy as np
import pytest

import oracle
import paper_2012_04553_b300 as pm
from pm_inputs import gnp_edges, rmat_edges


def expected(n, s, d):
    """(rowptr, col, new_id, lowdeg) from the oracle's graph: row r of the
    result is the sorted ranks of the neighbours of the vertex ranked r."""
    og = oracle.prepare_graph(n, s, d)
    rank = np.asarray(og.rank)
    old_of = np.argsort(rank)
    rows = [np.sort(rank[og.col[og.rowptr[v]:og.rowptr[v + 1]]]) for v in old_of]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    lowdeg = np.array([np.searchsorted(r, i) for i, r in enumerate(rows)], dtype=np.int64)
    return rowptr, col, rank.astype(np.int32), lowdeg


def check(n, s, d):
    got = pm.prepare_csr(n, s, d)
    want = expected(n, s, d)
    for name, g, w in zip(("rowptr", "col", "new_id", "lowdeg"), got, want):
        assert np.array_equal(g, w), name
    return got


def star_with_duplicates(leaves):
    """Vertex 0 joined to every other vertex twice (once per direction) and
    one self-loop: a single row of `leaves` ids after deduplication."""
    a = np.zeros(2 * leaves + 1, np.int64)
    b = np.concatenate([np.arange(1, leaves + 1), np.arange(1, leaves + 1), [0]])
    a[leaves:2 * leaves], b[leaves:2 * leaves] = b[leaves:2 * leaves], 0
    return leaves + 1, a.astype(np.int32), b.astype(np.int32)


def test_rmat_scale16_threaded_against_oracle():
    """1,048,576 raw edges with self-loops, duplicates and rows of
    thousands of ids (radix-sorted, 2 passes for 16-bit ids)."""
    n = 1 << 16
    s, d = rmat_edges(16, 16, seed=141)
    rowptr, col, new_id, lowdeg = check(n, s, d)
    assert np.diff(rowptr).max() > 1000 and (np.asarray(s) == np.asarray(d)).any()


def test_dense_graph_with_many_duplicates():
    """500,000 raw edges on 1,000 vertices: every row is a few hundred ids
    after removing about a third of the entries as duplicates."""
    rng = np.random.default_rng(142)
    s = rng.integers(0, 1000, 500_000).astype(np.int32)
    d = rng.integers(0, 1000, 500_000).astype(np.int32)
    rowptr, _, _, _ = check(1000, s, d)
    assert np.diff(rowptr).min() >= 128


def test_star_one_long_row():
    """One row of 200,000 ids (18-bit ids: three radix passes, the result
    copied back from the scratch row) and 200,000 rows of one id."""
    n, s, d = star_with_duplicates(200_000)
    rowptr, col, new_id, lowdeg = check(n, s, d)
    assert new_id[0] == n - 1 and rowptr[-1] == 2 * (n - 1)


@pytest.mark.parametrize("m_raw", [2 * 65536 - 1, 2 * 65536 + 1, 3 * 65536 + 7])
def test_thread_split_boundaries(m_raw):
    """Edge lists just below and above the two-thread threshold, and one
    that does not divide evenly into the threads' slices."""
    rng = np.random.default_rng(145 + m_raw)
    s = rng.integers(0, 5000, m_raw).astype(np.int32)
    d = rng.integers(0, 5000, m_raw).astype(np.int32)
    check(5000, s, d)


@pytest.mark.parametrize("n,p,seed", [(40, 0.3, 143), (300, 0.05, 144)])
def test_small_random_graphs(n, p, seed):
    s, d = gnp_edges(n, p, seed)
    check(n, s, d)


def test_degenerate_inputs():
    # no edges: the identity order, empty rows
    rowptr, col, new_id, lowdeg = check(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert np.array_equal(new_id, np.arange(5)) and len(col) == 0 and not rowptr.any()
    # only self-loops and one duplicated edge
    s = np.array([2, 2, 0, 1, 0], np.int32)
    d = np.array([2, 2, 1, 0, 1], np.int32)
    rowptr, col, new_id, lowdeg = check(3, s, d)
    assert rowptr[-1] == 2
    # a single vertex
    check(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    # the complete graph K_6 given in both directions
    a, b = np.triu_indices(6, 1)
    s = np.concatenate([a, b]).astype(np.int32)
    d = np.concatenate([b, a]).astype(np.int32)
    rowptr, col, _, _ = check(6, s, d)
    assert np.array_equal(np.diff(rowptr), np.full(6, 5))


def test_invalid_input_is_a_status():
    ok = np.array([0], np.int32), np.array([1], np.int32)
    with pytest.raises(pm.PMError) as e:
        pm.prepare_csr(0, *ok)
    assert e.value.status == pm.PM_EINVAL
    with pytest.raises(pm.PMError) as e:
        pm.prepare_csr(2, np.array([0, 2], np.int32), np.array([1, 1], np.int32))
    assert e.value.status == pm.PM_EINVAL
    with pytest.raises(pm.PMError) as e:
        pm.prepare_csr(2, np.array([-1], np.int32), np.array([1], np.int32))
    assert e.value.status == pm.PM_EINVAL
