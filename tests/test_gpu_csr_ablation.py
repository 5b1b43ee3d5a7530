"""The sorted-list (CSR) ablation of the enumeration (the set representation
Sec. III-B describes, intersections by binary search): it walks the same
search trees as the bitmap kernels, so its counts must equal the oracle's and
its per-level search statistics must equal the bitmap path's and the
oracle's instrumented traversal."""
import json
import math
import os

import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


@pytest.mark.parametrize("p,q", [(3, 3), (4, 4), (5, 5), (3, 4), (4, 3)])
@pytest.mark.parametrize("anchor", ["U", "V"])
def test_csr_counts_and_trees_equal_the_bitmap_path(gpu_ctx, p, q, anchor):
    g = bipgen.workload_small()
    rec = json.load(open(GOLDEN))
    want = int(rec["counts"][f"{p},{q}"])
    h = gpu_ctx.load(g)
    n_b, info_b = h.count_ex(p, q, anchor=anchor, stats=True)
    n_c, info_c = h.count_ex(p, q, anchor=anchor, stats=True, kernel="csr")
    assert n_b == n_c == want
    k = info_b["set_size"]
    assert info_c["set_size"] == k
    for lvl in range(2, k + 1):
        assert info_c["evals"][lvl] == info_b["evals"][lvl], lvl
        assert info_c["passed"][lvl] == info_b["passed"][lvl], lvl
    _, _, st = oracle.count(g, p, q, anchor=anchor, per_root=True, stats=True)
    assert info_c["evals"][2:k + 1] == st["evals"][2:k + 1]
    assert info_c["passed"][2:k + 1] == st["passed"][2:k + 1]
    tot, per = h.count_per_root(p, q, anchor)
    assert tot == want
    h.close()


@pytest.mark.parametrize("m,n,p,q", [(12, 15, 4, 5), (20, 9, 6, 3), (16, 16, 8, 8)])
def test_csr_on_complete_graphs(gpu_ctx, m, n, p, q):
    h = gpu_ctx.load(bipgen.complete(m, n))
    assert h.count_ex(p, q, kernel="csr")[0] == math.comb(m, p) * math.comb(n, q)
    h.close()


def test_csr_stops_at_its_deadline(gpu_ctx):
    import time
    import paper_2403_07858_gb300 as gbc
    h = gpu_ctx.load(bipgen.complete(128, 128))  # (8,8): C(128,8)^2 ~ 2e24 bicliques, far beyond the limit
    t0 = time.perf_counter()
    with pytest.raises(gbc.CountTimeout):
        h.count_ex(8, 8, kernel="csr", time_limit_ms=300)
    assert time.perf_counter() - t0 < 10.0
    h.close()
