"""Serving loop: every request's result is the same served alone and in a
concurrent mix (continuous batching across two graphs), and matches the
oracle; batching deduplicates matched patterns across requests."""
import numpy as np
import pytest

import oracle
from oracle import algebra
import paper_2012_04553_b300 as pm
from pm_inputs import pair_index, rmat_edges, random_patterns, uniform_ints

pytestmark = pytest.mark.gpu


def make_requests(seed, count, kmax):
    pats = random_patterns(count * 4, kmin=3, kmax=kmax, seed=seed)
    sizes = uniform_ints(seed, 2, count, 1, 8)
    reqs, at = [], 0
    for i, sz in enumerate(sizes):
        reqs.append((i % 2, pats[at:at + sz]))
        at += sz
        if at >= len(pats):
            at = 0
    return reqs


def test_results_alone_equal_results_in_mix_and_oracle():
    graphs_raw = [(256, rmat_edges(8, 8, seed=121)), (512, rmat_edges(9, 6, seed=122))]
    graphs = [pm.Graph(n, s, d) for n, (s, d) in graphs_raw]
    ograph = [oracle.prepare_graph(n, s, d) for n, (s, d) in graphs_raw]
    reqs = make_requests(123, 24, 5)
    queries = [[pm.make_pattern(k, m, ind) for k, m, ind in pats] for _, pats in reqs]
    # alone: one request at a time through the server
    alone = []
    srv = pm.Server(graphs, workers_per_graph=2, max_batch_patterns=64)
    for (gi, _), q in zip(reqs, queries):
        rid = srv.submit(gi, q)
        done, counts, lat, st = srv.wait(rid)
        assert done and st == pm.PM_OK
        alone.append(counts)
    srv.close()
    # mix: everything submitted at once, batched and overlapped
    srv = pm.Server(graphs, workers_per_graph=2, max_batch_patterns=64)
    ids = [srv.submit(gi, q) for (gi, _), q in zip(reqs, queries)]
    mixed = []
    for rid in ids:
        done, counts, lat, st = srv.wait(rid)
        assert done and st == pm.PM_OK and lat > 0
        mixed.append(counts)
    stats = srv.stats()
    srv.close()
    assert mixed == alone
    assert stats["requests_done"] == len(reqs)
    assert stats["batches"] < len(reqs)                 # requests were batched
    assert stats["matched_batched"] < stats["matched_alone"]   # shared patterns matched once
    # a few requests against the oracle
    for (gi, pats), counts in list(zip(reqs, alone))[:6]:
        want = [oracle.count(ograph[gi], algebra.Pattern.from_mask(k, m, None, bool(ind)))
                for k, m, ind in pats]
        assert counts == want


def test_server_rejects_bad_requests():
    s, d = rmat_edges(7, 4, seed=124)
    g = pm.Graph(128, s, d)
    srv = pm.Server([g])
    with pytest.raises(pm.PMError):
        srv.submit(0, [pm.make_pattern(4, 0b100001)])   # disconnected
    with pytest.raises(pm.PMError):
        srv.submit(3, [pm.make_pattern(3, 0b111)])      # no such graph
    srv.close()


def test_requests_past_their_deadline_are_shed():
    """With a request deadline shorter than any batch, requests queued behind
    the first batch complete unrun with PM_ETIMEOUT (load shedding), the
    server keeps answering, and a later request with time to spare runs."""
    s, d = rmat_edges(8, 8, seed=124)
    g = pm.Graph(256, s, d)
    q = [pm.make_pattern(4, 0b111111, pm.EDGE_INDUCED)]
    srv = pm.Server([g], workers_per_graph=1, max_batch_patterns=1, request_timeout_s=1e-9)
    ids = [srv.submit(0, q) for _ in range(50)]
    res = [srv.wait(rid, per_query=True) for rid in ids]
    assert all(done for done, _, _, _, _ in res)
    assert all(st == pm.PM_ETIMEOUT and qst == [pm.PM_ETIMEOUT] for _, _, _, st, qst in res)
    st = srv.stats()
    assert st["shed"] >= 1 and st["timeouts"] == 50 and st["requests_done"] == 50
    srv.close()
    srv = pm.Server([g], workers_per_graph=1, max_batch_patterns=1, request_timeout_s=30.0)
    done, counts, lat, status = srv.wait(srv.submit(0, q))
    assert done and status == pm.PM_OK and counts == pm.Plan(g, q, mode=pm.MORPH_NONE).count()
    srv.close()


def test_per_query_status_keeps_finished_queries():
    """A request mixing a pattern that finishes at once (the triangle) with
    one far beyond its deadline (the vertex-induced 6-star matched directly
    on hub rows of several hundred): the request fails, the finished query
    keeps PM_OK and its exact count."""
    s, d = rmat_edges(12, 16, seed=125)
    g = pm.Graph(4096, s, d)
    easy = pm.make_pattern(3, 0b111)
    star6 = sum(1 << pair_index(6, 0, v) for v in range(1, 6))
    hard = pm.make_pattern(6, star6, pm.VERTEX_INDUCED)
    want = pm.Plan(g, [easy], mode=pm.MORPH_NONE).count()[0]
    srv = pm.Server([g], workers_per_graph=1, max_batch_patterns=8, batch_timeout_s=0.2,
                    mode=pm.MORPH_NONE, family=pm.PLANS_FREE)
    done, counts, lat, st, qst = srv.wait(srv.submit(0, [easy, hard]), per_query=True)
    srv.close()
    assert done and st == pm.PM_ETIMEOUT
    assert qst == [pm.PM_OK, pm.PM_ETIMEOUT] and counts[0] == want
