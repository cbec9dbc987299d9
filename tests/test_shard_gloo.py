"""Root-range sharding across processes, on CPU: two gloo ranks each count
their share of the roots (with the plan interpreter standing in for the
kernels), the matched counts are summed exactly across ranks, and the
morphed result equals the oracle's whole-graph count (additivity over root
ranges: every occurrence has one highest-ranked vertex)."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import paper_2012_04553_b300 as pm
    from oracle import algebra
    from paper_2012_04553_b300 import shard
    from pm_inputs import rmat_edges
    from tests.plan_interp import degree_ordered, run_plans

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    s, d = rmat_edges(6, 6, seed=31)
    g = oracle.prepare_graph(64, s, d)
    adj, labels = degree_ordered(g)
    queries = [pm.make_pattern(4, m, pm.VERTEX_INDUCED) for m in algebra.connected_classes(4)]
    plan = pm.Plan(None, queries, mode=pm.MORPH_NAIVE)
    mine = shard.root_shard(g.rank, rank, world)
    partial = run_plans(plan.export_plans(pm.PLANS_ROOTED), plan.n_matched, adj, labels,
                        roots=[int(g.rank[v]) for v in mine])
    total = shard.allreduce_counts(partial)
    result = plan.morph(total)
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"counts": [str(c) for c in result],
                       "want": [str(c) for c in oracle.motif_counts_direct(g, 4)]}, f)
    dist.barrier()
    dist.destroy_process_group()


def _columns(g, p, roots=None):
    """MNI columns of p (orbit unions of per-vertex domains), from the oracle,
    over the matches whose highest-ranked vertex is in roots, packed as
    uint32 words (bit v % 32 of word v / 32)."""
    import oracle
    from oracle import algebra
    _, dom = oracle.match_count(g, p, roots=roots, domains=True)
    cols = [np.logical_or.reduce([dom[u] for u in orb]) for orb in algebra.orbits(p)]
    words = (g.n + 31) // 32
    out = np.zeros((len(cols), words), dtype=np.uint32)
    for c, col in enumerate(cols):
        for v in np.nonzero(col)[0]:
            out[c, v >> 5] |= np.uint32(1 << (int(v) & 31))
    return out


def _mni_worker(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2012_04553_b300 import shard
    from pm_inputs import rmat_edges, zipf_labels

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    n = 128
    s, d = rmat_edges(7, 8, seed=33)
    labels = zipf_labels(n, 2, seed=34)
    g = oracle.prepare_graph(n, s, d, labels)
    pats = oracle.labeled_edge_patterns(2, [0, 1]) + oracle.labeled_edge_patterns(3, [0, 1])[::3]
    mine = shard.root_shard(g.rank, rank, world)
    local = np.concatenate([_columns(g, p, roots=mine) for p in pats])
    parts = shard.gather_columns(torch.from_numpy(local.view(np.int32)))
    # the OR the library's pm_domains_or computes on the device, on the host here
    cols = np.bitwise_or.reduce(parts.numpy().view(np.uint32), axis=0)
    got, at = [], 0
    for p in pats:
        nc = len(__import__("oracle").algebra.orbits(p))
        got.append(int(min(sum(bin(int(w)).count("1") for w in cols[at + c]) for c in range(nc))))
        at += nc
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"got": got, "want": [oracle.support_direct(g, p) for p in pats],
                       "whole": bool((cols == np.concatenate([_columns(g, p) for p in pats])).all())}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_mni_support(tmp_path):
    """MNI columns of each rank's roots, gathered over gloo and ORed, equal
    the columns over all matches, and their smallest sizes the supports."""
    import torch.multiprocessing as mp
    out = str(tmp_path / "mni.json")
    mp.spawn(_mni_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = json.load(open(out))
    assert res["whole"] and res["got"] == res["want"]


def test_two_rank_root_sharding(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.json")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = json.load(open(out))
    assert res["counts"] == res["want"]


def test_root_shards_partition_and_balance():
    from paper_2012_04553_b300 import shard
    rng = np.random.default_rng(5)
    new_id = rng.permutation(1000).astype(np.int32)
    for world in (1, 2, 3, 8):
        parts = [shard.root_shard(new_id, r, world) for r in range(world)]
        allv = np.concatenate(parts)
        assert sorted(allv.tolist()) == list(range(1000))
        # the `world` highest-ranked vertices land on distinct ranks
        top = set(np.argsort(new_id)[-world:].tolist())
        owners = [r for r in range(world) for v in parts[r] if v in top]
        assert sorted(owners) == list(range(world))
    with pytest.raises(ValueError):
        shard.root_shard(new_id, 2, 2)


def test_limb_sums_are_exact_mod_2_128():
    from paper_2012_04553_b300 import shard
    vals = [[(1 << 128) - 1, 3, 1 << 127], [1, (1 << 64) - 1, 1 << 127]]
    summed = np.sum([shard.to_limbs(v) for v in vals], axis=0)
    assert shard.from_limbs(summed) == [0, 1 << 64 | 2, 0]
    assert shard.from_limbs(shard.to_limbs([12345678901234567890123])) == [12345678901234567890123]
