"""Root-range sharding of a count over several processes (one GPU each).

Every occurrence of a pattern has exactly one highest-ranked vertex, rank
ordering vertices by (degree, caller id), so the per-root counts of
pm_count_roots over a partition of the vertex set add up to the whole count.
Each process holds a replica of the data graph, counts the matched
(morphed) patterns over its own roots, the partial counts are summed exactly
across processes, and the morph transform (Theorem 3.1 / Corollary 3.1) is
applied once to the sum.  The transform is linear over the integers mod
2^128, so summing matched counts and then morphing equals morphing each
partial and summing.

The only exchange is one sum of n_matched 128-bit integers, carried out as
16-bit limbs in int64 so that it is exact for any realistic world size.

MNI support shards the same way: the columns of a query over all matches
are the union of its columns over each process's roots, so each process
fills its columns (pm_support_roots), the columns are gathered, ORed by
the library (pm_domains_or) and the smallest column of each query is its
support (pm_support_from_domains).  There is no OR reduction in NCCL, hence
an all-gather followed by a local OR.
"""
import numpy as np

LIMB_BITS = 16
LIMBS = 128 // LIMB_BITS


def root_shard(new_id, rank, world):
    """Caller vertex ids whose occurrences process `rank` of `world` counts.

    new_id[v] is the degree-ordered id of caller vertex v (as returned by
    Graph.vertex_order).  Work per root grows with its degree, so vertices are
    dealt out from the highest rank down in a snake order (0,1,..,w-1,w-1,..,0,
    ...), which keeps the hubs spread evenly over the processes.  The shards
    of rank 0..world-1 partition range(len(new_id))."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    new_id = np.asarray(new_id)
    by_rank = np.empty(len(new_id), dtype=np.int64)
    by_rank[new_id] = np.arange(len(new_id))     # caller id at each degree-ordered id
    desc = by_rank[::-1]
    pos = np.arange(len(desc)) % (2 * world)
    owner = np.where(pos < world, pos, 2 * world - 1 - pos)
    return np.sort(desc[owner == rank]).astype(np.int32)


def to_limbs(values):
    """128-bit integers (Python ints, taken mod 2^128) as int64 limbs, least
    significant first: shape (len(values), LIMBS)."""
    out = np.zeros((len(values), LIMBS), dtype=np.int64)
    mask = (1 << LIMB_BITS) - 1
    for i, v in enumerate(values):
        v %= 1 << 128
        for j in range(LIMBS):
            out[i, j] = (v >> (LIMB_BITS * j)) & mask
    return out


def from_limbs(limbs):
    """Inverse of to_limbs after limb-wise sums: carries propagate through
    Python integers, the result is reduced mod 2^128."""
    out = []
    for row in np.asarray(limbs):
        v = 0
        for j in range(LIMBS - 1, -1, -1):
            v = (v << LIMB_BITS) + int(row[j])
        out.append(v % (1 << 128))
    return out


def allreduce_counts(values, group=None):
    """Exact sum mod 2^128 of per-process lists of 128-bit counts over a
    torch.distributed process group (any backend that sums int64)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(to_limbs(values))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return from_limbs(t.numpy())


def count_sharded(plan, graph, rank, world, stream=None, timeout_s=0.0, group=None):
    """Requested counts of `plan` with the roots split over `world` processes:
    this process counts its shard with pm_count_roots, the matched counts
    are summed across processes, and every process morphs the sum."""
    roots = root_shard(graph.vertex_order(), rank, world)
    _, matched = plan.count_roots(roots, stream=stream, timeout_s=timeout_s, with_matched=True)
    total = allreduce_counts(matched, group) if world > 1 else matched
    return plan.morph(total)


def gather_columns(local, group=None):
    """All processes' MNI column bitsets stacked: shape (world,) + local.shape.
    CUDA tensors are gathered with the group's backend on the device; with a
    CPU-only backend (gloo) they are staged through host memory."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    staged = local if dist.get_backend(group) == "nccl" else local.cpu()
    parts = [torch.empty_like(staged) for _ in range(world)]
    dist.all_gather(parts, staged.contiguous(), group=group)
    return torch.stack(parts).to(local.device)


def support_sharded(plan, graph, rank, world, threshold=0, stream=None, timeout_s=0.0, group=None):
    """MNI supports of a PM_OP_SUPPORT plan with the roots split over `world`
    processes: each fills the columns of its shard, the columns are gathered
    and ORed on the device, and each process reads the supports."""
    import paper_2012_04553_b300 as pm
    roots = root_shard(graph.vertex_order(), rank, world)
    local = plan.support_roots(roots, stream=stream, timeout_s=timeout_s)
    cols = pm.domains_or(gather_columns(local, group), stream=stream) if world > 1 else local
    return plan.support_from_domains(cols, threshold, stream=stream)
