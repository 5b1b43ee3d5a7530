"""The bit order of a root's C_R bitmaps (most shared position first, or the
other side's id order as after gbc_border_order) and loading a graph with its
ids kept change the search's layout, never its result: counts and search-tree
statistics must equal the oracle's."""
import json
import os

import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


@pytest.mark.parametrize("p,q", [(3, 3), (4, 4), (5, 5), (4, 3)])
def test_position_orders_and_kept_ids_give_the_oracle_count(gpu_ctx, p, q):
    import paper_2403_07858_gb300 as gbc
    g = bipgen.workload_small()
    want = int(json.load(open(GOLDEN))["counts"][f"{p},{q}"])
    new_v, _, _ = gbc.border_order(g.n_u, g.n_v, g.off_u, g.adj_u, iterations=500, max_cand=32)
    import numpy as np
    us = np.repeat(np.arange(g.n_u), np.diff(g.off_u))
    gb = bipgen.from_edges(g.n_u, g.n_v, us, new_v[np.asarray(g.adj_u)])
    for graph, keep in [(g, False), (g, True), (gb, True)]:
        h = gpu_ctx.load(graph, keep_ids=keep)
        for order in ("shared", "id"):
            n, info = h.count_ex(p, q, anchor="U", position_order=order, stats=True)
            assert n == want, (keep, order)
        _, _, st = oracle.count(graph, p, q, anchor="U", per_root=True, stats=True)
        k = info["set_size"]
        assert info["evals"][2:k + 1] == st["evals"][2:k + 1]
        h.close()
