"""GPU parity: the CUDA library (through its C ABI) against the oracle.

Counts are integers, so the bar is bit-exact equality.  The search-tree
statistics (children evaluated per level, bitmap words read) must match the
oracle's instrumented traversal exactly as well: both walk the same tree.
"""
import json
import math
import os

import numpy as np
import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gpu_count(ctx, g, p, q, anchor="auto"):
    h = ctx.load(g)
    try:
        if anchor == "auto":
            return h.count(p, q)
        return h.count_ex(p, q, anchor=anchor)[0]
    finally:
        h.close()


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_all_pq(gpu_ctx, seed):
    g = bipgen.tiny_random(seed, 7 + seed % 4, 8 + seed % 5, 0.2 + 0.05 * seed)
    h = gpu_ctx.load(g)
    for p in range(1, 6):
        for q in range(1, 6):
            want = oracle.count(g, p, q)
            assert h.count(p, q) == want, (p, q)
            assert h.count_ex(p, q, anchor="U")[0] == want, (p, q, "U")
            assert h.count_ex(p, q, anchor="V")[0] == want, (p, q, "V")
    h.close()


@pytest.mark.parametrize("m,n,p,q", [(7, 9, 3, 4), (20, 20, 8, 8), (40, 40, 8, 8), (40, 40, 4, 8),
                                     (12, 200, 6, 16), (64, 64, 5, 5), (33, 65, 6, 7)])
def test_complete_bipartite(gpu_ctx, m, n, p, q):
    g = bipgen.complete(m, n)
    want = math.comb(m, p) * math.comb(n, q)
    h = gpu_ctx.load(g)
    assert h.count(p, q) == want
    # anchored on a side, the search enumerates that side's sets: C(m, p) or C(n, q) leaves
    if math.comb(m, p) <= 10 ** 8:
        assert h.count_ex(p, q, anchor="U", time_limit_ms=60_000)[0] == want
    if math.comb(n, q) <= 10 ** 8:
        assert h.count_ex(p, q, anchor="V", time_limit_ms=60_000)[0] == want
    h.close()


def test_time_limit_stops_a_runaway_count(gpu_ctx):
    """Anchoring K_{12,200} on V for (6,16) would enumerate C(200,16) ~ 2e23 sets;
    the device deadline ends it with a timeout and the context stays usable."""
    import paper_2403_07858_gb300 as gbc
    g = bipgen.complete(12, 200)
    h = gpu_ctx.load(g)
    with pytest.raises(gbc.CountTimeout):
        h.count_ex(6, 16, anchor="V", time_limit_ms=300)
    assert h.count(6, 16) == math.comb(12, 6) * math.comb(200, 16)
    h.close()


def test_overflow_reported(gpu_ctx):
    import paper_2403_07858_gb300 as gbc
    g = bipgen.complete(16, 1000)
    h = gpu_ctx.load(g)
    with pytest.raises(gbc.CountOverflow):
        h.count_ex(8, 16, anchor="U")
    assert h.count(1, 16) == 16 * math.comb(1000, 16)
    h.close()


def test_small_workload_golden(gpu_ctx):
    fx = json.load(open(os.path.join(GOLDEN, "workloads.json")))
    g = bipgen.workload_small()
    assert bipgen.graph_sha256(g) == fx["sha256"]  # same graph on this host as where the values were made
    h = gpu_ctx.load(g)
    for key, val in fx["counts"].items():
        p, q = map(int, key.split(","))
        assert h.count(p, q) == int(val), key
        assert h.count_ex(p, q, anchor="U")[0] == int(val), key
        assert h.count_ex(p, q, anchor="V")[0] == int(val), key
    h.close()


@pytest.mark.parametrize("p,q,anchor", [(2, 2, "U"), (3, 3, "U"), (3, 3, "V"), (4, 4, "U"), (4, 3, "V"),
                                        (5, 5, "U"), (4, 2, "U"), (2, 4, "V")])
def test_tree_statistics_match_oracle(gpu_ctx, p, q, anchor):
    g = bipgen.workload_small()
    h = gpu_ctx.load(g)
    got, info = h.count_ex(p, q, anchor=anchor, stats=True)
    want, st = oracle.count(g, p, q, anchor=anchor, stats=True)
    assert got == want
    assert info["roots"] == st["roots_expanded"]
    assert info["evals"] == st["evals"]
    assert info["passed"] == st["passed"]
    assert info["words_r"] == st["words_r"]
    assert info["words_l"] == st["words_l"]
    k = p if anchor == "U" else q  # size of the set enumerated on the anchor side
    # enum_words counts the words the enumeration kernel actually loads (C_R read
    # up to its span, two words at a time); it runs only when k >= 4 and then
    # has work exactly when the tree has nodes below the root's children
    below = st["words_r"] + st["words_l"] - st["words_lvl2"]
    if k >= 4 and sum(st["evals"][4:]) > 0:
        assert info["enum_words"] > 0 and below > 0
    elif k < 4:
        assert info["enum_words"] == 0
    # the model words of the nodes the enumeration kernel evaluates (|L| >= 3)
    # are the oracle's words below the roots' children
    assert info["words_enum"] == (below if k >= 4 else 0)
    assert info["launches"] > 0
    if k >= 2:
        assert info["scratch_bytes"] > 0
    h.close()


@pytest.mark.parametrize("p,q", [(1, 3), (2, 2), (3, 3), (4, 4), (5, 3)])
def test_per_root_small_workload(gpu_ctx, p, q):
    g = bipgen.workload_small()
    h = gpu_ctx.load(g)
    for anchor in ("U", "V"):
        tot, per = h.count_per_root(p, q, anchor)
        otot, oper = oracle.count(g, p, q, anchor=anchor, per_root=True)
        assert tot == otot
        assert per == oper
    h.close()


def _all_tiers_graph():
    # power-law part (small and medium roots), a dense random block (medium),
    # and K_{70,110}, whose low-ranked roots see ~7.6k oriented wedges (largest tier)
    return bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(70, 110),
                                 bipgen.tiny_random(9, 60, 80, 0.5))


def test_medium_graph_all_tiers(gpu_ctx):
    """Roots in all three candidate tiers; counts and tree statistics."""
    g = _all_tiers_graph()
    h = gpu_ctx.load(g)
    for p, q, anchors in [(2, 2, "UV"), (3, 3, "UV"), (4, 4, "UV"), (3, 5, "U"), (5, 4, "UV")]:
        for anchor in anchors:
            want, st = oracle.count(g, p, q, anchor=anchor, stats=True)
            got, info = h.count_ex(p, q, anchor=anchor, stats=True)
            assert got == want, (p, q, anchor)
            assert info["evals"] == st["evals"] and info["words_r"] == st["words_r"], (p, q, anchor)
    h.close()


def test_edge_cases(gpu_ctx):
    empty = bipgen.from_edges(4, 5, [], [])
    h = gpu_ctx.load(empty)
    for p, q in [(1, 1), (2, 2), (3, 1)]:
        assert h.count(p, q) == 0
    h.close()
    nothing = bipgen.from_edges(0, 0, [], [])
    h = gpu_ctx.load(nothing)
    assert h.count(1, 1) == 0 and h.count(2, 2) == 0
    h.close()
    g = bipgen.complete(3, 4)
    h = gpu_ctx.load(g)
    assert h.count(4, 1) == 0 and h.count(1, 5) == 0 and h.count(3, 4) == 1 and h.count(16, 16) == 0
    import paper_2403_07858_gb300 as gbc
    with pytest.raises(gbc.GbcError):
        h.count(0, 1)
    with pytest.raises(gbc.GbcError):
        h.count(1, 17)
    h.close()
    # isolated vertices and a star
    star = bipgen.from_edges(10, 50, [0] * 50, list(range(50)))
    h = gpu_ctx.load(star)
    assert h.count(1, 3) == math.comb(50, 3) and h.count(2, 1) == 0 and h.count(1, 16) == math.comb(50, 16)
    h.close()


def _csr(g):
    return [g.off_u.copy(), g.adj_u.copy(), g.off_v.copy(), g.adj_v.copy()]


def test_invalid_graphs_rejected(gpu_ctx):
    import paper_2403_07858_gb300 as gbc
    g = bipgen.tiny_random(5, 8, 9, 0.5)
    bad = _csr(g)
    bad[1][[0, 1]] = bad[1][[1, 0]]  # unsorted row (row 0 has >= 2 entries at this density)
    with pytest.raises(gbc.InvalidGraph):
        gpu_ctx.load_graph(g.n_u, g.n_v, *bad)
    bad = _csr(g)
    bad[1][0] = g.n_v + 3  # out of range
    with pytest.raises(gbc.InvalidGraph):
        gpu_ctx.load_graph(g.n_u, g.n_v, *bad)
    bad = _csr(g)
    bad[0][1] = bad[0][2] + 1  # offsets not monotone
    with pytest.raises(gbc.InvalidGraph):
        gpu_ctx.load_graph(g.n_u, g.n_v, *bad)
    h2 = bipgen.add_edges(g, [0], [int(np.setdiff1d(np.arange(g.n_v), g.adj_u[g.off_u[0]:g.off_u[1]])[0])])
    mixed = [h2.off_u, h2.adj_u, g.off_v, g.adj_v]  # U side has one more edge
    with pytest.raises(gbc.InvalidGraph):
        gpu_ctx.load_graph(g.n_u, g.n_v, *mixed)
    # same edge count, not transposes: move one V-row entry to another vertex
    off_v, adj_v = g.off_v.copy(), g.adj_v.copy()
    v = int(np.argmax(np.diff(off_v)))
    row = adj_v[off_v[v]:off_v[v + 1]]
    missing = np.setdiff1d(np.arange(g.n_u), row)
    if missing.size:
        adj_v[off_v[v]] = missing[0]
        adj_v[off_v[v]:off_v[v + 1]].sort()
        with pytest.raises(gbc.InvalidGraph):
            gpu_ctx.load_graph(g.n_u, g.n_v, g.off_u, g.adj_u, off_v, adj_v)
    # the context still works afterwards
    h = gpu_ctx.load(g)
    assert h.count(2, 2) == oracle.count(g, 2, 2)
    h.close()


def test_device_arrays_load(gpu_ctx):
    torch = pytest.importorskip("torch")
    g = bipgen.workload_small()
    arrs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (g.off_u, g.adj_u, g.off_v, g.adj_v)]
    h = gpu_ctx.load_graph(g.n_u, g.n_v, *arrs)
    assert h.count(3, 3) == oracle.count(g, 3, 3)
    # the library renumbers vertices internally; per-root results come back
    # in the caller's ids, the same from device or host arrays
    hh = gpu_ctx.load(g)
    for anchor in ("U", "V"):
        tot_d, per_d = h.count_per_root(3, 3, anchor)
        tot_h, per_h = hh.count_per_root(3, 3, anchor)
        assert tot_d == tot_h and list(per_d) == list(per_h)
    hh.close()
    h.close()


def test_relabel_and_swap_invariance_gpu(gpu_ctx):
    g = bipgen.workload_small()
    ref = _gpu_count(gpu_ctx, g, 4, 3)
    assert _gpu_count(gpu_ctx, bipgen.permute(g, 5), 4, 3) == ref
    assert _gpu_count(gpu_ctx, bipgen.swap_sides(g), 3, 4) == ref


def test_disjoint_union_additive_gpu(gpu_ctx):
    a = bipgen.workload_small()
    b = bipgen.complete(30, 30)
    c = bipgen.chung_lu(8, 500, 700, 6000, 2.1, 2.1)
    u = bipgen.disjoint_union(a, b, c)
    for p, q in [(3, 3), (4, 4)]:
        assert _gpu_count(gpu_ctx, u, p, q) == sum(_gpu_count(gpu_ctx, x, p, q) for x in (a, b, c))


def test_batch_equals_single_counts(gpu_ctx):
    """gbc_count_batch: one pipeline and one enumeration launch for many jobs on
    several graphs; every job equals its own gbc_count, errors stay per job."""
    import paper_2403_07858_gb300 as gbc
    graphs = [bipgen.workload_small(), _all_tiers_graph(), bipgen.complete(20, 30),
              bipgen.tiny_random(4, 9, 11, 0.5), bipgen.from_edges(3, 3, [], []), bipgen.complete(16, 1000)]
    hs = [gpu_ctx.load(g) for g in graphs]
    jobs = []
    for gi in range(4):
        for p, q in [(1, 2), (2, 2), (3, 3), (4, 4), (2, 5), (5, 2), (4, 6), (6, 3)]:
            jobs.append((gi, p, q))
    jobs += [(4, 2, 2), (5, 8, 16), (0, 0, 3), (1, 5, 5)]
    res = gpu_ctx.count_batch([hs[gi] for gi, _, _ in jobs], [p for _, p, _ in jobs], [q for _, _, q in jobs])
    for (gi, p, q), r in zip(jobs, res):
        if p == 0:
            assert isinstance(r, gbc.GbcError) and r.status == gbc.GBC_ERR_ARG
        elif gi == 5:
            assert isinstance(r, gbc.GbcError) and r.status == gbc.GBC_ERR_OVERFLOW
        else:
            assert r == hs[gi].count(p, q), (gi, p, q)
            if gi in (0, 3) or (gi == 1 and p + q <= 7):
                assert r == oracle.count(graphs[gi], p, q), (gi, p, q)
    # a second batch in a row gives the same numbers
    res2 = gpu_ctx.count_batch([hs[gi] for gi, _, _ in jobs], [p for _, p, _ in jobs], [q for _, _, q in jobs])
    assert [x if isinstance(x, int) else x.status for x in res] == [x if isinstance(x, int) else x.status for x in res2]
    for h in hs:
        h.close()


def test_autotune_keeps_counts_and_records_a_side(gpu_ctx):
    g = bipgen.workload_small()
    h = gpu_ctx.load(g)
    pqs = [(2, 2), (3, 3), (4, 4), (2, 5), (5, 5)]
    before = [h.count(p, q) for p, q in pqs]
    gpu_ctx.autotune([h] * len(pqs), [p for p, _ in pqs], [q for _, q in pqs], time_limit_ms=20_000)
    for (p, q), b in zip(pqs, before):
        assert h.tuned_anchor(p, q) in ("U", "V")
        assert h.count(p, q) == b
    assert h.tuned_anchor(1, 3) is None
    res = gpu_ctx.count_batch([h] * len(pqs), [p for p, _ in pqs], [q for _, q in pqs])
    assert res == before
    h.close()


def test_root_ranges_add_up_to_the_count(gpu_ctx):
    """Disjoint root ranges (the multi-GPU split) sum to the whole count, and
    each range equals the oracle's count over the same roots."""
    from paper_2403_07858_gb300.shard import root_ranges
    g = bipgen.workload_small()
    h = gpu_ctx.load(g)
    for p, q, anchor in [(3, 3, "U"), (4, 4, "V"), (1, 3, "U"), (2, 2, "V")]:
        n_a = g.n_u if anchor == "U" else g.n_v
        deg = np.diff(g.off_u if anchor == "U" else g.off_v).astype(float)
        parts = [h.count_ex(p, q, anchor=anchor, roots=r)[0] for r in root_ranges(deg ** 2, 3)]
        assert sum(parts) == h.count(p, q)
        r = root_ranges(deg ** 2, 3)[1]
        assert parts[1] == oracle.count(g, p, q, anchor=anchor, roots=r)
        assert h.count_ex(p, q, anchor=anchor, roots=(0, n_a))[0] == h.count(p, q)
    h.close()


@pytest.mark.parametrize("m,n,p,q,anchor", [(18, 18, 16, 2, "U"), (18, 18, 2, 16, "V"), (17, 17, 16, 16, "U"),
                                            (17, 20, 16, 3, "U"), (20, 17, 3, 16, "V")])
def test_deepest_search_trees(gpu_ctx, m, n, p, q, anchor):
    """|L| = 16 on the anchor side: the enumeration runs at its largest depth
    (13 levels below the level-2 units); complete graphs fix the count."""
    h = gpu_ctx.load(bipgen.complete(m, n))
    assert h.count_ex(p, q, anchor=anchor)[0] == math.comb(m, p) * math.comb(n, q)
    h.close()
