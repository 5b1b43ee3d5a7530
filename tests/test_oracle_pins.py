"""Pins of the oracle against facts fixed by the paper and by mathematics.

Each test compares the oracle (Sec. III-A Basic model with the Def. 2 priority)
with something that is not the oracle: brute force over all subsets (Def. 1),
closed forms, the butterfly identity, symmetries, invariances and the values the
paper prints for its worked examples.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import bipgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _edges_graph(n_u, n_v, edges):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return bipgen.from_edges(n_u, n_v, e[:, 0], e[:, 1])


def test_fig1_example_two_32_bicliques():
    fx = json.load(open(os.path.join(GOLDEN, "fig1.json")))
    g = _edges_graph(fx["n_u"], fx["n_v"], fx["edges"])
    assert oracle.count(g, fx["p"], fx["q"]) == fx["count"]
    assert oracle.count(g, fx["p"], fx["q"], anchor="V") == fx["count"]
    assert oracle.brute_force(g, fx["p"], fx["q"]) == fx["count"]
    # the stated overlaps hold in the reconstruction
    nb = {u: set(g.adj_u[g.off_u[u]:g.off_u[u + 1]].tolist()) for u in range(g.n_u)}
    assert nb[2] & nb[3] == {1, 2} and nb[2] & nb[4] == {0, 2, 4} and nb[3] & nb[4] == {2, 3}
    assert nb[1] & nb[2] == {0, 1, 2}


def test_htb_worked_example_word_and_bit_convention():
    """Id x lives in word x // 32 at bit x % 32, LSB first: the convention of the
    C_R / C_L bitmap rows.  The paper's printed words pin it."""
    fx = json.load(open(os.path.join(GOLDEN, "htb_example.json")))

    def pack(ids):
        words = {}
        for x in ids:
            words[x // 32] = words.get(x // 32, 0) | (1 << (x % 32))
        return words

    w = pack(fx["n2q_u"])
    assert [[x // 32, x % 32] for x in fx["n2q_u"]] == fx["pairs"]
    assert sorted(w) == fx["idx"] and [w[i] for i in sorted(w)] == fx["val"]
    c = pack(fx["cl_prev"])
    assert sorted(c) == fx["cl_prev_idx"] and c[0] == fx["cl_prev_word0"]
    a = w[0] & c[0]
    assert a == fx["and_word0"] and [b for b in range(32) if a >> b & 1] == fx["and_members"]


@pytest.mark.parametrize("seed", range(16))
def test_brute_force_small_random(seed):
    """Def. 1 literally (all L and R subsets) on random graphs of <= 8+9 vertices."""
    n_u, n_v = 6 + seed % 3, 7 + seed % 3
    g = bipgen.tiny_random(seed, n_u, n_v, 0.25 + 0.04 * seed)
    for p in range(1, 5):
        for q in range(1, 5):
            want = oracle.brute_force(g, p, q)
            assert oracle.count(g, p, q) == want, (p, q)
            assert oracle.count(g, p, q, anchor="V") == want, (p, q)


@pytest.mark.parametrize("seed", range(6))
def test_definition_12x12(seed):
    """Sum over p-subsets of C(|common|, q) on 12+12 graphs, every 1 <= p, q <= 6."""
    g = bipgen.tiny_random(100 + seed, 12, 12, 0.15 + 0.12 * seed)
    for p in range(1, 7):
        for q in range(1, 7):
            want = oracle.by_definition(g, p, q)
            assert oracle.count(g, p, q) == want, (p, q)
            assert oracle.count(g, p, q, anchor="V") == want, (p, q)


@pytest.mark.parametrize("m,n,p,q", [(7, 9, 3, 4), (20, 20, 8, 8), (40, 40, 4, 8), (40, 24, 4, 8),
                                     (12, 200, 6, 16), (1, 5, 1, 5), (5, 1, 5, 1), (3, 3, 4, 1)])
def test_complete_bipartite_closed_form(m, n, p, q):
    g = bipgen.complete(m, n)
    want = math.comb(m, p) * math.comb(n, q)
    assert oracle.count(g, p, q) == want
    if math.comb(n, q) <= 200_000:  # the V-anchored search enumerates the q-subsets
        assert oracle.count(g, p, q, anchor="V") == want


def test_u128_range_exercised():
    g = bipgen.complete(12, 200)
    v = oracle.count(g, 6, 16)
    assert v > 2 ** 64 and v == math.comb(12, 6) * math.comb(200, 16)


def test_overflow_detected():
    g = bipgen.complete(16, 1000)
    exact = math.comb(16, 8) * math.comb(1000, 16)
    assert exact >= 2 ** 128
    with pytest.raises(oracle.OracleOverflow):
        oracle.count(g, 8, 16)
    below = math.comb(16, 1) * math.comb(1000, 16)
    assert below < 2 ** 128
    assert oracle.count(g, 1, 16) == below


def test_binomial_table_matches_math_comb():
    for n in list(range(0, 60)) + [100, 1000, 1442, 5000]:
        for k in range(0, 17):
            c = math.comb(n, k)
            got = oracle.binomial(n, k)
            assert got == (c if c < 2 ** 128 else None), (n, k)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_closed_forms_single_side(seed):
    """(1,1) = |E|; (p,1) = sum_v C(deg v, p); (1,q) = sum_u C(deg u, q)."""
    g = bipgen.chung_lu(seed, 200, 300, 1500, 2.1, 2.1)
    du = np.diff(g.off_u)
    dv = np.diff(g.off_v)
    assert oracle.count(g, 1, 1) == g.n_edges
    for p in (2, 3, 4):
        assert oracle.count(g, p, 1) == sum(math.comb(int(d), p) for d in dv)
        assert oracle.count(g, p, 1, anchor="V") == sum(math.comb(int(d), p) for d in dv)
    for q in (2, 3, 4):
        assert oracle.count(g, 1, q) == sum(math.comb(int(d), q) for d in du)


def _butterflies(g):
    """(2,2) from wedges: sum over pairs u < u' of C(|N(u) & N(u')|, 2)."""
    a = np.zeros((g.n_u, g.n_v), dtype=np.float64)  # counts < 2^53: exact in float64
    us, vs = g.edges()
    a[us, vs] = 1.0
    c = np.rint(a @ a.T).astype(np.int64)
    iu = np.triu_indices(g.n_u, 1)
    x = c[iu]
    return int((x * (x - 1) // 2).sum())


@pytest.mark.parametrize("seed", [4, 5])
def test_butterfly_identity(seed):
    g = bipgen.chung_lu(seed, 300, 200, 2500, 2.0, 2.3)
    assert oracle.count(g, 2, 2) == _butterflies(g)


def test_butterfly_identity_small_workload():
    g = bipgen.workload_small()
    assert oracle.count(g, 2, 2) == _butterflies(g)


@pytest.mark.parametrize("p,q", [(2, 3), (3, 2), (3, 3), (4, 2)])
def test_symmetry_swap_sides(p, q):
    g = bipgen.chung_lu(11, 250, 350, 2500, 2.1, 2.1)
    assert oracle.count(g, p, q) == oracle.count(bipgen.swap_sides(g), q, p)


@pytest.mark.parametrize("p,q", [(2, 2), (3, 3), (4, 3)])
def test_relabel_invariance(p, q):
    g = bipgen.chung_lu(12, 250, 300, 2500, 2.1, 2.1)
    assert oracle.count(g, p, q) == oracle.count(bipgen.permute(g, 99), p, q)


@pytest.mark.parametrize("p,q", [(2, 2), (3, 3), (3, 4)])
def test_disjoint_union_additive(p, q):
    g1 = bipgen.chung_lu(13, 150, 200, 1500, 2.1, 2.1)
    g2 = bipgen.complete(9, 11)
    g3 = bipgen.tiny_random(3, 10, 12, 0.5)
    u = bipgen.disjoint_union(g1, g2, g3)
    assert oracle.count(u, p, q) == sum(oracle.count(x, p, q) for x in (g1, g2, g3))


def test_monotone_under_edge_addition():
    g = bipgen.chung_lu(14, 120, 150, 900, 2.1, 2.1)
    rng = np.random.default_rng(0)
    us = rng.integers(0, g.n_u, 200)
    vs = rng.integers(0, g.n_v, 200)
    h = bipgen.add_edges(g, us, vs)
    for p, q in [(2, 2), (3, 2), (2, 3), (3, 3)]:
        assert oracle.count(h, p, q) >= oracle.count(g, p, q)


def test_per_root_split_matches_lowest_ranked_member():
    """Per-root counts: bicliques whose lowest-ranked L member (key (deg, id)) is the root."""
    g = bipgen.tiny_random(21, 9, 10, 0.5)
    deg = np.diff(g.off_u)
    masks = []
    for u in range(g.n_u):
        m = 0
        for v in g.adj_u[g.off_u[u]:g.off_u[u + 1]]:
            m |= 1 << int(v)
        masks.append(m)
    import itertools
    for p, q in [(2, 2), (3, 2), (3, 3)]:
        want = [0] * g.n_u
        for L in itertools.combinations(range(g.n_u), p):
            m = (1 << g.n_v) - 1
            for u in L:
                m &= masks[u]
            root = min(L, key=lambda u: (int(deg[u]), u))
            want[root] += math.comb(bin(m).count("1"), q)
        tot, per = oracle.count(g, p, q, per_root=True)
        assert per == want and tot == sum(want)


def test_pair_level_count_identity():
    """For p = 2 the level-2 nodes are the pairs {u, w} sharing >= q neighbours."""
    g = bipgen.chung_lu(15, 300, 300, 3000, 2.1, 2.1)
    a = np.zeros((g.n_u, g.n_v), dtype=np.int64)
    us, vs = g.edges()
    a[us, vs] = 1
    c = (a @ a.T)[np.triu_indices(g.n_u, 1)]
    for q in (1, 2, 3):
        _, st = oracle.count(g, 2, q, stats=True)
        assert st["evals"][2] == int((c >= q).sum())


def test_edge_cases():
    empty = bipgen.from_edges(4, 5, [], [])
    assert oracle.count(empty, 1, 1) == 0 and oracle.count(empty, 2, 2) == 0
    g = bipgen.complete(3, 4)
    assert oracle.count(g, 4, 1) == 0  # p > |U|
    assert oracle.count(g, 1, 5) == 0  # q > |V|
    assert oracle.count(g, 3, 4) == 1
    with pytest.raises(ValueError):
        oracle.count(g, 0, 1)
    with pytest.raises(ValueError):
        oracle.count(g, 1, 17)


def test_golden_workload_values_and_generator_determinism():
    fx = json.load(open(os.path.join(GOLDEN, "workloads.json")))
    g = bipgen.workload_small()
    assert bipgen.graph_sha256(g) == fx["sha256"]
    assert bipgen.graph_sha256(bipgen.chung_lu(7, 300, 400, 3000, 2.1, 2.1)) == fx["small_sha256"]
    for key in ("2,2", "3,3", "1,3"):
        p, q = map(int, key.split(","))
        assert oracle.count(g, p, q) == int(fx["counts"][key])


@pytest.mark.parametrize("m,n,p,q", [(9, 7, 3, 2), (12, 5, 4, 3), (10, 40, 5, 6), (8, 33, 4, 1), (14, 3, 6, 3)])
def test_tree_statistics_closed_form_on_complete_graphs(m, n, p, q):
    """The search-tree statistics (Alg. 1's nodes and the words a bitmap
    implementation reads) in closed form on K_{m,n}.  All degrees are equal, so
    the rank order is the id order; every pair shares n >= q neighbours, so
    every evaluated child passes.  A node with |L| = s whose largest member is
    i has C_L = the m - 1 - i later vertices and is entered when that is at
    least p - s; the C(i, s - 1) nodes with largest member i each evaluate all
    of their C_L.  C_R rows have ceil(n/32) words; C_L rows one word (m <= 33)."""
    _, st = oracle.count(bipgen.complete(m, n), p, q, stats=True)
    evals = [0] * len(st["evals"])
    for s in range(1, p):
        evals[s + 1] = sum(math.comb(i, s - 1) * (m - 1 - i) for i in range(m) if m - 1 - i >= p - s)
    assert st["evals"] == evals
    assert st["passed"] == evals
    assert st["roots_expanded"] == max(0, m - p + 1)
    wr = (n + 31) // 32
    assert st["words_r"] == wr * sum(evals)
    assert st["words_l"] == sum(evals[2:p])  # passed children that are not leaves, one word each
    assert st["words_lvl2"] == wr * evals[2] + (evals[2] if p > 2 else 0)


@pytest.mark.parametrize("p,q", [(3, 2), (4, 3)])
def test_tree_statistics_additive_over_disjoint_unions(p, q):
    """Search trees never cross components (2-hop neighbours stay inside one),
    and the rank order inside each component is kept, so every statistic of a
    disjoint union is the sum of its parts'."""
    g1 = bipgen.chung_lu(41, 200, 150, 1500, 2.1, 2.1)
    g2 = bipgen.tiny_random(42, 20, 25, 0.4)
    g3 = bipgen.complete(9, 11)
    parts = [oracle.count(g, p, q, stats=True)[1] for g in (g1, g2, g3)]
    _, whole = oracle.count(bipgen.disjoint_union(g1, g2, g3), p, q, stats=True)
    for key in ("roots_expanded", "words_r", "words_l", "words_lvl2"):
        assert whole[key] == sum(st[key] for st in parts), key
    for key in ("evals", "passed"):
        assert whole[key] == [sum(x) for x in zip(*(st[key] for st in parts))], key
