"""Listing mode: the bicliques themselves (Alg. 1 outputs them, Sec. IV).

Each record is (L, C_R): an anchor-side set L and its whole common
neighbourhood C_R on the other side; every biclique is (L, a q-subset of C_R)
of exactly one record.  On small graphs the records, expanded into (L, R)
pairs, must equal the brute-force set of Def. 1 exactly; on the 20k-edge
graph every record must hold an exact common neighbourhood, no L may repeat,
and the records must add up to the oracle's count.  A buffer far smaller
than the output exercises the back-pressure (many calls, nothing dropped)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import bipgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


def _nbrs(off, adj):
    return [frozenset(int(x) for x in adj[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def _brute_pairs(g, p, q):
    """Def. 1 literally: every (L, R) with |L| = p, |R| = q and L x R in E."""
    nu = _nbrs(g.off_u, g.adj_u)
    out = set()
    for L in itertools.combinations(range(g.n_u), p):
        common = frozenset(range(g.n_v))
        for u in L:
            common &= nu[u]
        for R in itertools.combinations(sorted(common), q):
            out.add((L, R))
    return out


def _pairs_of(records, p, q, anchor):
    """(L on U, R on V) pairs of the records (anchor V records hold L on V)."""
    out = set()
    for L, C in records:
        if anchor == "U":
            for R in itertools.combinations(sorted(C), q):
                out.add((tuple(sorted(L)), R))
        else:
            for Lu in itertools.combinations(sorted(C), p):
                out.add((Lu, tuple(sorted(L))))
    return out


@pytest.fixture(scope="module")
def torch_and_gbc():
    torch = pytest.importorskip("torch")
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    return torch, gbc


def _graphs():
    fig1 = json.load(open(os.path.join(os.path.dirname(GOLDEN), "fig1.json")))
    gs = [bipgen.from_edges(fig1["n_u"], fig1["n_v"], np.array([e[0] for e in fig1["edges"]]),
                            np.array([e[1] for e in fig1["edges"]]))]
    gs += [bipgen.tiny_random(s, 8, 9, d) for s, d in [(41, 0.4), (42, 0.6), (43, 0.8)]]
    gs += [bipgen.complete(6, 7), bipgen.disjoint_union(bipgen.complete(4, 5), bipgen.tiny_random(44, 6, 6, 0.5))]
    return gs


@pytest.mark.parametrize("anchor", ["U", "V"])
def test_listed_bicliques_equal_brute_force(torch_and_gbc, anchor):
    torch, gbc = torch_and_gbc
    ctx = gbc.Context(0)
    try:
        buf = torch.zeros(4096, dtype=torch.int32, device="cuda")
        for g in _graphs():
            h = ctx.load(g)
            for p in range(1, 5):
                for q in range(1, 5):
                    want = _brute_pairs(g, p, q)
                    recs = list(h.list_records(p, q, buf, anchor=anchor))
                    k = p if anchor == "U" else q
                    assert all(len(L) == k and len(set(L)) == k for L, _ in recs)
                    assert len({frozenset(L) for L, _ in recs}) == len(recs)  # each L once
                    got = _pairs_of(recs, p, q, anchor)
                    assert got == want, (p, q, anchor)
            h.close()
    finally:
        ctx.close()


@pytest.mark.parametrize("p,q", [(2, 3), (3, 3), (4, 4)])
def test_listing_on_the_20k_edge_graph(torch_and_gbc, p, q):
    torch, gbc = torch_and_gbc
    g = bipgen.workload_small()
    rec = json.load(open(GOLDEN))
    assert rec["sha256"] == bipgen.graph_sha256(g)
    want = int(rec["counts"][f"{p},{q}"])
    nu = _nbrs(g.off_u, g.adj_u)
    ctx = gbc.Context(0)
    try:
        h = ctx.load(g)
        total, seen, calls = 0, set(), []
        # a buffer of max(4096 words, the largest root's records): many calls
        for L, C in h.list_records(p, q, min_words=4096, calls=calls):
            assert len(L) == p and len(C) >= q
            common = frozenset.intersection(*(nu[u] for u in L))
            assert frozenset(C) == common
            key = frozenset(L)
            assert key not in seen
            seen.add(key)
            total += math.comb(len(C), q)
        assert total == want
        assert len(calls) > 1 and sum(r for _, r in calls) == len(seen)
        h.close()
    finally:
        ctx.close()


def test_a_root_larger_than_the_buffer_is_reported(torch_and_gbc):
    torch, gbc = torch_and_gbc
    ctx = gbc.Context(0)
    try:
        h = ctx.load(bipgen.complete(10, 10))
        buf = torch.zeros(16, dtype=torch.int32, device="cuda")
        with pytest.raises(gbc.GbcError) as ei:
            list(h.list_records(3, 3, buf))
        assert ei.value.status == gbc.GBC_ERR_OOM and "words" in str(ei.value)
        h.close()
    finally:
        ctx.close()
