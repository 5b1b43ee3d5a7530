"""Border (Sec. V-B, Alg. 2), host preprocessing: it returns a permutation of the
reordered side, the 1-blocks it reports (32-id blocks of an adjacency row
holding a single neighbour) equal a brute-force recount before (the degree
order it starts from) and after, and greedy exchanges never add 1-blocks.
CPU only: gbc_border_order runs on the host."""
import numpy as np
import pytest

import bipgen


def _one_blocks(off, adj, new_id):
    total = 0
    for r in range(len(off) - 1):
        blocks = {}
        for v in adj[off[r]:off[r + 1]]:
            b = int(new_id[v]) // 32
            blocks[b] = blocks.get(b, 0) + 1
        total += sum(1 for c in blocks.values() if c == 1)
    return total


def _degree_order(n_o, adj):
    deg = np.bincount(np.asarray(adj, dtype=np.int64), minlength=n_o)
    order = sorted(range(n_o), key=lambda v: (-int(deg[v]), v))
    pos = np.empty(n_o, dtype=np.int64)
    pos[order] = np.arange(n_o)
    return pos


@pytest.mark.parametrize("g", [bipgen.chung_lu(7, 300, 400, 3000, 2.1, 2.1),
                               bipgen.chung_lu(9, 500, 1200, 6000, 2.0, 2.4),
                               bipgen.tiny_random(3, 40, 90, 0.05)])
def test_border_is_a_permutation_and_lowers_one_blocks(g):
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    new_id, before, after = gbc.border_order(g.n_u, g.n_v, g.off_u, g.adj_u, iterations=2000, max_cand=64)
    assert sorted(new_id.tolist()) == list(range(g.n_v))
    assert before == _one_blocks(g.off_u, g.adj_u, _degree_order(g.n_v, g.adj_u))
    assert after == _one_blocks(g.off_u, g.adj_u, new_id)
    assert after <= before


def test_border_joins_a_split_pair():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    # 33 columns of degree 2: columns 31 and 32 share two rows, every other
    # column has two rows to itself.  The degree order (all equal, ties by id)
    # leaves 31 in block 0 and 32 in block 1, so each shared row holds two
    # 1-blocks (4), besides the 62 lone rows'.  Exchanging 32 with a column of
    # block 0 that shares no row with it removes those 4 and adds none.
    rows = [[31, 32], [31, 32]] + [[c] for c in range(31) for _ in range(2)]
    us = [r for r, vs in enumerate(rows) for _ in vs]
    vs = [v for vs in rows for v in vs]
    g = bipgen.from_edges(len(rows), 33, np.array(us), np.array(vs))
    new_id, before, after = gbc.border_order(g.n_u, g.n_v, g.off_u, g.adj_u, iterations=100, max_cand=64)
    assert before == 66
    assert after == _one_blocks(g.off_u, g.adj_u, new_id) == 62
    assert new_id[31] // 32 == new_id[32] // 32
