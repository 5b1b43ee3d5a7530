"""Serving: gbc_submit / gbc_poll with continuous batching.

Each served count must equal the count of the same query run alone, whatever
else was in its batch; admission refuses requests beyond the queue bound; a
request past its deadline reports a timeout without disturbing the others.
"""
import math
import random
import threading
import time

import pytest

import bipgen

pytestmark = pytest.mark.gpu


def _graphs():
    return [bipgen.workload_small(),
            bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(70, 110),
                                  bipgen.tiny_random(9, 60, 80, 0.5)),
            bipgen.complete(20, 30), bipgen.chung_lu(8, 500, 700, 6000, 2.1, 2.1)]


def test_served_equals_alone_under_concurrent_submitters():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        hs = [ctx.load(g) for g in _graphs()]
        queries = [(gi, p, q) for gi in range(len(hs)) for p in range(1, 6) for q in range(1, 6)]
        alone = {qr: hs[qr[0]].count(qr[1], qr[2]) for qr in queries}
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
            assert v == alone[qr], qr
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
