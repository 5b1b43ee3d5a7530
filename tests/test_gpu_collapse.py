"""GPU parity of the enumeration's subtree collapse against the oracle.

A node whose common neighbourhood C_R holds at most q' + 2 positions (q' the
set size on the other side) adds its whole subtree in closed form: the sum,
over the q'-subsets Q of C_R, of C(n_Q, vertices still to add), n_Q the
candidates of C_L adjacent to all of Q.  That is the subtree's leaves counted
from the other side (Def. 1), so counts with and without it must equal the
oracle's exactly.
"""
import math

import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,p,q", [(30, 6, 6, 6), (30, 7, 6, 6), (30, 8, 6, 6), (24, 4, 5, 2),
                                     (26, 5, 8, 3), (20, 17, 16, 16), (40, 10, 8, 8), (60, 9, 4, 7)])
def test_complete_graphs_collapse_at_the_units(gpu_ctx, m, n, p, q):
    """Anchored on U, every level-2 unit of K_{m,n} has |C_R| = n, so n - q =
    0, 1, 2 collapse at the unit (one, n or C(n, 2) subsets Q; K_{40,10} at
    (8,8) needs 45 > 32 subsets and (60, 9, 4, 7) a skip set of 2 with 36, so
    neither collapses); the count is C(m,p) C(n,q)."""
    want = math.comb(m, p) * math.comb(n, q)
    h = gpu_ctx.load(bipgen.complete(m, n))
    on, info = h.count_ex(p, q, anchor="U", stats="exec")
    assert on == want
    assert h.count_ex(p, q, anchor="U")[0] == want
    assert h.count_ex(p, q, anchor="U", collapse=False)[0] == want
    s = n - q
    if p >= 4 and (s == 0 or (s == 1 and n <= 32) or (s == 2 and n * (n - 1) <= 64)):
        assert info["collapsed"] > 0
    elif p >= 4:
        assert info["collapsed"] == 0
    h.close()


@pytest.mark.parametrize("p,q", [(4, 4), (5, 5), (6, 6), (5, 4), (4, 6), (6, 3), (7, 7)])
def test_power_law_graph_collapse_on_and_off(gpu_ctx, p, q):
    """The 20k-edge power-law graph, both anchors: the count with the collapse,
    without it, and the per-root split all equal the oracle's."""
    g = bipgen.workload_small()
    h = gpu_ctx.load(g)
    for anchor in ("U", "V"):
        want, per_want = oracle.count(g, p, q, anchor=anchor, per_root=True)
        got, info = h.count_ex(p, q, anchor=anchor, stats="exec")
        assert got == want, (p, q, anchor)
        assert h.count_ex(p, q, anchor=anchor, collapse=False)[0] == want, (p, q, anchor)
        tot, per = h.count_per_root(p, q, anchor)
        assert tot == want and per == per_want, (p, q, anchor)
        k = p if anchor == "U" else q
        if k >= 4 and want > 0:
            assert info["collapsed"] > 0 and info["words_exec"] > 0, (p, q, anchor)
    h.close()


def test_collapse_in_a_batch_with_mixed_sizes(gpu_ctx):
    """One enumeration launch over jobs with different q' (so different subset
    sizes and binomial rows) on the medium graph of all candidate tiers."""
    g = bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(30, 7),
                              bipgen.tiny_random(9, 60, 80, 0.5))
    h = gpu_ctx.load(g)
    pq = [(4, 4), (5, 5), (6, 6), (4, 6), (6, 4), (5, 7)]
    got = gpu_ctx.count_batch([h] * len(pq), [p for p, _ in pq], [q for _, q in pq])
    for (p, q), v in zip(pq, got):
        assert v == oracle.count(g, p, q), (p, q)
    h.close()
