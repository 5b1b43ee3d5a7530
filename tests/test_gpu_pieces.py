"""Counts whose search scratch exceeds the context's budget run in pieces:
contiguous ranges of roots, each within the budget, one after the other
(the closure partitioning of Sec. VI applied to the scratch; roots' search
trees are independent, Sec. III-B).  The pieces' sum must equal the oracle's
count, and so must every per-root value."""
import json
import os

import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


@pytest.mark.parametrize("p,q", [(3, 3), (4, 4), (5, 5), (2, 6), (6, 2)])
def test_over_budget_counts_run_in_pieces(p, q):
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    g = bipgen.workload_small()
    rec = json.load(open(GOLDEN))
    assert rec["sha256"] == bipgen.graph_sha256(g)
    want = int(rec["counts"][f"{p},{q}"])
    roomy = gbc.Context(0)
    try:
        h = roomy.load(g)
        n, info = h.count_ex(p, q)
        assert n == want and info["pieces"] == 1
        full = info["scratch_bytes"]
        h.close()
    finally:
        roomy.close()
    # room for the per-count minimum (|E|-sized position maps) and about a
    # third of the rest: several pieces
    budget = 8 * g.n_edges + 8192 + (full - 8 * g.n_edges) // 3
    tight = gbc.Context(0, mem_budget_bytes=budget)
    try:
        h = tight.load(g)
        n, info = h.count_ex(p, q)
        assert n == want
        if info["set_size"] >= 3:
            assert info["pieces"] > 1, info
            assert info["scratch_bytes"] <= budget
        anchor = info["anchor"]
        tot, per = h.count_per_root(p, q, anchor)
        assert tot == want
        _, want_per, _ = oracle.count(g, p, q, anchor=anchor, per_root=True, stats=True)
        assert per == want_per
        h.close()
    finally:
        tight.close()


def test_a_root_larger_than_the_budget_is_reported():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    g = bipgen.complete(40, 40)
    ctx = gbc.Context(0, mem_budget_bytes=8 * g.n_edges + 8192 + 256)
    try:
        h = ctx.load(g)
        with pytest.raises(gbc.GbcError) as ei:
            h.count(4, 4)
        assert ei.value.status == gbc.GBC_ERR_OOM and "root" in str(ei.value)
        h.close()
    finally:
        ctx.close()


def test_pieces_inside_a_batch():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    g = bipgen.workload_small()
    rec = json.load(open(GOLDEN))
    pairs = [(3, 3), (4, 4), (5, 5), (2, 3)]
    roomy = gbc.Context(0)
    try:
        h = roomy.load(g)
        alone = [h.count_ex(p, q)[1]["scratch_bytes"] for p, q in pairs]
        h.close()
    finally:
        roomy.close()
    # half of what the jobs hold when they all run at once (plus one set of the
    # |E|-sized position maps): the batch must split into waves or pieces
    tight = gbc.Context(0, mem_budget_bytes=sum(alone) // 2 + 8 * g.n_edges)
    try:
        h = tight.load(g)
        got = tight.count_batch([h] * len(pairs), [p for p, _ in pairs], [q for _, q in pairs])
        assert got == [int(rec["counts"][f"{p},{q}"]) for p, q in pairs]
        h.close()
    finally:
        tight.close()
