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


def _collapses(m, kq, slack):
    """The library's rule: |C_R| = m exceeds kq by s <= slack, and the skip
    sets fit (s <= 1 with m <= 32; else s <= 4, m <= 16, C(m, s) <= 256)."""
    s = m - kq
    if s > slack:
        return False
    return m <= 32 if s <= 1 else (s <= 4 and m <= 16 and math.comb(m, s) <= 256)


@pytest.mark.parametrize("m,n,p,q", [(30, 6, 6, 6), (30, 7, 6, 6), (30, 8, 6, 6), (24, 4, 5, 2),
                                     (26, 5, 8, 3), (20, 17, 16, 16), (40, 10, 8, 8), (30, 9, 6, 6),
                                     (30, 10, 5, 6), (20, 18, 16, 16), (30, 12, 4, 8)])
def test_complete_graphs_collapse_at_the_units(gpu_ctx, m, n, p, q):
    """Anchored on U, every level-2 unit of K_{m,n} has |C_R| = n, so with a
    slack s >= n - q the unit collapses: C(n, n - q) subsets Q, each with every
    higher candidate; the count is C(m,p) C(n,q) with and without it, at every
    slack (K_{20,18} at (16,16) needs a skip set of 2 from 18 positions, beyond
    the 16 the skip-set table covers, so it is always entered)."""
    want = math.comb(m, p) * math.comb(n, q)
    h = gpu_ctx.load(bipgen.complete(m, n))
    assert h.count_ex(p, q, anchor="U")[0] == want
    assert h.count_ex(p, q, anchor="U", collapse=False)[0] == want
    for slack in (1, 2, 3, 4):
        got, info = h.count_ex(p, q, anchor="U", stats="exec", collapse=slack)
        assert got == want, slack
        if p >= 4:
            assert (info["collapsed"] > 0) == _collapses(n, q, slack), slack
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
        for slack in (1, 3, 4):
            assert h.count_ex(p, q, anchor=anchor, collapse=slack)[0] == want, (p, q, anchor, slack)
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
