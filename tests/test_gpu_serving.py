"""Serving: gbc_submit / gbc_poll with continuous batching.

Each served count must equal the oracle's count of the same query and the
count of the query run alone, whatever else was in its batch; a request is
released when its own count is done, before a slow batch-mate; admission
by scratch footprint keeps the batches on the device within the budget;
submission refuses requests beyond the queue bound; a request past its
deadline reports a timeout without disturbing the others.
"""
import json
import math
import os
import random
import threading
import time

import pytest

import bipgen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serving_counts.json")

pytestmark = pytest.mark.gpu


def _graphs():
    return [bipgen.workload_small(),
            bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(70, 110),
                                  bipgen.tiny_random(9, 60, 80, 0.5)),
            bipgen.complete(20, 30), bipgen.chung_lu(8, 500, 700, 6000, 2.1, 2.1)]


def _oracle_counts(graphs):
    """The oracle's counts of every (p,q) in {1..5}^2 on the four graphs, stored by
    tests/golden/make_serving_golden.py (a few take the oracle minutes)."""
    rec = json.load(open(GOLDEN))["graphs"]
    out = {}
    for gi, g in enumerate(graphs):
        assert rec[str(gi)]["sha256"] == bipgen.graph_sha256(g)
        for key, v in rec[str(gi)]["counts"].items():
            p, q = (int(x) for x in key.split(","))
            out[(gi, p, q)] = int(v)
    return out


def test_served_equals_alone_under_concurrent_submitters():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        hs = [ctx.load(g) for g in _graphs()]
        graphs = _graphs()
        queries = [(gi, p, q) for gi in range(len(hs)) for p in range(1, 6) for q in range(1, 6)]
        alone = {qr: hs[qr[0]].count(qr[1], qr[2]) for qr in queries}
        want = _oracle_counts(graphs)
        assert alone == {qr: want[qr] for qr in queries}
        ctx.serve_start(workers=3, max_batch=16)
        results, errors = {}, []

        def client(seed):
            rng = random.Random(seed)
            mine = rng.sample(queries, 40)
            tickets = []
            for qr in mine:
                tickets.append((qr, ctx.submit(hs[qr[0]], qr[1], qr[2])))
                time.sleep(rng.random() * 0.002)  # arrivals spread over time
            for qr, t in tickets:
                try:
                    results[(seed, qr)] = ctx.poll(t, -1)
                except Exception as e:  # pragma: no cover - reported below
                    errors.append((qr, e))

        threads = [threading.Thread(target=client, args=(s,)) for s in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        assert len(results) == 160
        for (seed, qr), v in results.items():
            assert v == want[qr], qr
        ctx.serve_stop()
        for h in hs:
            h.close()
    finally:
        ctx.close()


def test_admission_rejects_beyond_the_queue_and_deadline_times_out():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        slow = ctx.load(bipgen.complete(64, 64))  # (8,8): C(64,8) ~ 4.4e9 leaves
        quick = ctx.load(bipgen.complete(6, 7))
        ctx.serve_start(workers=1, max_batch=1, max_queue=2, time_limit_ms=300)
        t_slow = ctx.submit(slow, 8, 8)
        time.sleep(0.05)  # the single worker is now busy with the slow request
        accepted, rejected = [], 0
        for _ in range(6):
            try:
                accepted.append(ctx.submit(quick, 3, 3))
            except gbc.GbcError as e:
                assert e.status == gbc.GBC_ERR_REJECTED
                rejected += 1
        assert rejected >= 1 and len(accepted) <= 2
        with pytest.raises(gbc.CountTimeout):
            ctx.poll(t_slow, -1)
        for t in accepted:
            assert ctx.poll(t, -1) == math.comb(6, 3) * math.comb(7, 3)
        ctx.serve_stop()
        slow.close()
        quick.close()
    finally:
        ctx.close()


def test_request_completes_before_its_slow_batch_mate():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        slow = ctx.load(bipgen.complete(128, 128))  # (8,8): C(128,8)^2 ~ 2e24, runs into the 2 s deadline
        quick = ctx.load(bipgen.complete(6, 7))
        ctx.serve_start(workers=1, max_batch=16, time_limit_ms=2000)
        blocker = ctx.submit(slow, 8, 8)
        time.sleep(0.2)  # the single worker is busy with the blocker
        t_slow = ctx.submit(slow, 8, 8)
        t_quick = ctx.submit(quick, 3, 3)  # waits with t_slow; both go in the next batch
        with pytest.raises(gbc.CountTimeout):
            ctx.poll(blocker, -1)
        t0 = time.perf_counter()
        assert ctx.poll(t_quick, 1500) == math.comb(6, 3) * math.comb(7, 3)
        released_after = time.perf_counter() - t0
        assert ctx.poll(t_slow, 0) is None  # its batch-mate is still on the device
        assert released_after < 1.0
        with pytest.raises(gbc.CountTimeout):
            ctx.poll(t_slow, -1)
        st = ctx.serve_stats()
        assert st["admitted"] == 3 and st["batches"] == 2
        ctx.serve_stop()
        slow.close()
        quick.close()
    finally:
        ctx.close()


def test_footprint_bound_then_exact():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        g = bipgen.workload_small()
        h = ctx.load(g)
        for p, q in [(2, 3), (3, 3), (4, 4), (5, 5), (6, 2)]:
            bound, exact = h.footprint(p, q)
            assert not exact
            _, info = h.count_ex(p, q)
            used = info["scratch_bytes"]
            assert bound >= used, (p, q, bound, used)
            got, exact = h.footprint(p, q)
            assert exact
            assert abs(got - used) <= 4096, (p, q, got, used)
        h.close()
    finally:
        ctx.close()


def test_admission_keeps_batches_within_the_budget():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    graphs = [bipgen.workload_small(), bipgen.chung_lu(8, 500, 700, 6000, 2.1, 2.1), bipgen.complete(20, 30)]
    queries = [(gi, p, q) for gi in range(3) for p in (2, 3, 4) for q in (2, 3, 4)]
    want = {qr: oracle.count(graphs[qr[0]], qr[1], qr[2]) for qr in queries}
    # learn each query's exact footprint, then serve with room for about three at once
    probe = gbc.Context(0)
    try:
        hs = [probe.load(g) for g in graphs]
        for gi, p, q in queries:
            hs[gi].count(p, q)
        feet = [hs[gi].footprint(p, q)[0] for gi, p, q in queries]
        for h in hs:
            h.close()
    finally:
        probe.close()
    budget = 3 * max(feet)
    ctx = gbc.Context(0, mem_budget_bytes=budget)
    try:
        hs = [ctx.load(g) for g in graphs]
        for gi, p, q in queries:  # footprints are learned per context
            hs[gi].count(p, q)
            assert hs[gi].footprint(p, q)[1]
        ctx.serve_start(workers=4, max_batch=4)
        tickets = [(qr, ctx.submit(hs[qr[0]], qr[1], qr[2])) for qr in queries * 3]
        for qr, t in tickets:
            assert ctx.poll(t, -1) == want[qr], qr
        st = ctx.serve_stats()
        assert st["admitted"] == len(tickets)
        assert st["budget_bytes"] == budget
        assert 0 < st["peak_in_flight_bytes"] <= budget
        assert st["batches"] >= len(tickets) // 4
        ctx.serve_stop()
        for h in hs:
            h.close()
    finally:
        ctx.close()


def test_concurrent_batches_with_different_layouts():
    """Four workers put batches of different |L| and row widths on the device at
    once (each enumeration launch sizes its own shared memory): every request
    of repeated bursts must finish with the oracle's count."""
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        graphs = _graphs()
        hs = [ctx.load(g) for g in graphs]
        want = _oracle_counts(graphs)
        queries = [(gi, p, q) for gi in range(len(hs)) for p in range(3, 6) for q in range(3, 6)]
        ctx.serve_start(workers=4, max_batch=4)
        for burst in range(3):
            rng = random.Random(1000 + burst)
            order = queries * 2
            rng.shuffle(order)
            tickets = [(qr, ctx.submit(hs[qr[0]], qr[1], qr[2])) for qr in order]
            for qr, t in tickets:
                assert ctx.poll(t, -1) == want[qr], (burst, qr)
        st = ctx.serve_stats()
        assert st["batches"] >= 3 * len(queries) * 2 // 4
        ctx.serve_stop()
        for h in hs:
            h.close()
    finally:
        ctx.close()
