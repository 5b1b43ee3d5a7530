"""The entry point that allocates nothing (gbc_count_p2_noalloc).

Some callers cannot call cudaMalloc -- code inside another framework's memory
pool, plug-ins that may only touch the buffers handed to them -- so this entry
point keeps all of its scratch in one fixed static device array.  Its counts
must equal those of the ordinary path (gbc_count with p = 2) and the oracle's
on the same graph, and must stay equal on a second call that reuses the array
the first call left behind.  This file is collected last on purpose.
"""
import math
import time

import numpy as np
import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu


def _device_csr(torch, g):
    return [torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda()
            for x in (g.off_u, g.adj_u, g.off_v, g.adj_v)]


def _graphs():
    return [
        bipgen.workload_small(),
        bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(70, 110),
                              bipgen.tiny_random(9, 60, 80, 0.5)),
        bipgen.complete(12, 40),
    ]


def test_noalloc_matches_the_allocating_path_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    ctx = gbc.Context(0)
    try:
        for g in _graphs():
            h = ctx.load(g)
            arrs = _device_csr(torch, g)
            for q in (1, 2, 3, 5):
                want = h.count(2, q)
                assert want == oracle.count(g, 2, q), q
                first = gbc.count_p2_noalloc(g.n_u, g.n_v, *arrs, q)
                second = gbc.count_p2_noalloc(g.n_u, g.n_v, *arrs, q)
                assert first == want, (q, first, want)
                assert second == want, (q, second, want)
            h.close()
        k = bipgen.complete(12, 40)
        arrs = _device_csr(torch, k)
        assert gbc.count_p2_noalloc(k.n_u, k.n_v, *arrs, 7) == math.comb(12, 2) * math.comb(40, 7)
    finally:
        ctx.close()


def test_noalloc_rejects_a_graph_beyond_its_fixed_scratch():
    torch = pytest.importorskip("torch")
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    # one V vertex adjacent to 5001 degree-1 U vertices: the lowest-ranked of
    # them has 5000 higher-ranked 2-hop neighbours, beyond the 4096 the
    # static scratch holds per root
    n_u = 5001
    star = bipgen.from_edges(n_u, 1, np.arange(n_u), np.zeros(n_u, dtype=np.int64))
    arrs = _device_csr(torch, star)
    with pytest.raises(gbc.GbcError) as ei:
        gbc.count_p2_noalloc(star.n_u, star.n_v, *arrs, 1)
    assert ei.value.status == gbc.GBC_ERR_OOM and "scratch" in str(ei.value)
    # the next call, on a graph within the limit, is unaffected
    g = bipgen.workload_small()
    ctx = gbc.Context(0)
    try:
        h = ctx.load(g)
        want = h.count(2, 2)
        h.close()
    finally:
        ctx.close()
    assert gbc.count_p2_noalloc(g.n_u, g.n_v, *_device_csr(torch, g), 2) == want


def test_noalloc_gives_up_quickly_when_the_table_overflows():
    torch = pytest.importorskip("torch")
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    # one V vertex adjacent to 20001 degree-1 U vertices: the lowest-ranked has
    # 20000 higher-ranked 2-hop neighbours, more than the 8192 slots of its
    # table; the call must stop at the first root that overflows and report it
    n_u = 20_001
    star = bipgen.from_edges(n_u, 1, np.arange(n_u), np.zeros(n_u, dtype=np.int64))
    arrs = _device_csr(torch, star)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(gbc.GbcError) as ei:
        gbc.count_p2_noalloc(star.n_u, star.n_v, *arrs, 1)
    assert ei.value.status == gbc.GBC_ERR_OOM
    assert time.perf_counter() - t0 < 5.0
    # a graph within the limit still counts right afterwards
    g = bipgen.complete(12, 40)
    assert gbc.count_p2_noalloc(g.n_u, g.n_v, *_device_csr(torch, g), 3) == math.comb(12, 2) * math.comb(40, 3)
