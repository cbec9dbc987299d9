"""The allocation-free 4-cycle entry point (pm_count_c4_noalloc) against the
regular one (pm_count) and the oracle, through the C ABI, on two calls in a
row.

The entry point exists for callers that cannot allocate device memory while
counting; it keeps its scratch in an array built into the library, so its
results must match pm_count's exactly and must not depend on what an earlier
call left in that shared array.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from oracle import algebra
import paper_2012_04553_b300 as pm
from pm_inputs import rmat_edges

pytestmark = pytest.mark.gpu

C4_MASK = 0b011110   # edges (0,2), (0,3), (1,2), (1,3): a 4-cycle


def undirected_csr(n, src, dst):
    """Sorted, symmetric, loop-free CSR of a raw edge list (test-side)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    a = np.concatenate([src[keep], dst[keep]])
    b = np.concatenate([dst[keep], src[keep]])
    key = np.unique(a * n + b)
    rows, cols = key // n, key % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32)


def as_int(words):
    lo, hi = (int(x) & ((1 << 64) - 1) for x in words)
    return lo | (hi << 64)


# scale 16 holds 65,536 vertices: the scratch then fits 64 blocks, fewer
# than the SMs, so each block's counters sit far into the shared array
@pytest.mark.parametrize("scale,ef,seed", [(12, 8, 71), (14, 16, 72), (16, 8, 73)])
def test_noalloc_c4_matches_pm_count_on_two_calls(scale, ef, seed):
    import torch
    n = 1 << scale
    s, d = rmat_edges(scale, ef, seed=seed)
    g = pm.Graph(n, s, d)
    want = pm.Plan(g, [pm.make_pattern(4, C4_MASK)], mode=pm.MORPH_NONE).count()[0]
    assert want > 0
    if scale == 12:
        # and against the oracle (plain backtracking), not only the other entry point
        assert want == oracle.count(oracle.prepare_graph(n, s, d), algebra.Pattern.from_mask(4, C4_MASK))
    rowptr, col = undirected_csr(n, s, d)
    rowptr_d = torch.from_numpy(rowptr).cuda()
    col_d = torch.from_numpy(col).cuda()
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for _ in range(2):
        out.fill_(-1)                      # stale output must be overwritten
        pm.count_c4_noalloc(rowptr_d, col_d, n, out)
        torch.cuda.synchronize()
        assert as_int(out.cpu().tolist()) == want


def test_noalloc_rejects_malformed_tensors():
    import torch
    rowptr_d = torch.zeros(5, dtype=torch.int64, device="cuda")
    col_d = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for args in ((rowptr_d.int(), col_d, 4, out), (rowptr_d, col_d.long(), 4, out),
                 (rowptr_d, col_d, 5, out), (rowptr_d, col_d, 4, out[:1]), (rowptr_d.cpu(), col_d, 4, out)):
        with pytest.raises(pm.PMError) as e:
            pm.count_c4_noalloc(*args)
        assert e.value.status == pm.PM_EINVAL


def test_noalloc_rejects_graphs_beyond_its_scratch():
    import torch
    n = (1 << 22) + 1
    rowptr_d = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.count_c4_noalloc(rowptr_d, col_d, n, out)
    assert e.value.status == pm.PM_EINVAL
