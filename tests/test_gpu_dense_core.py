"""The dense-core workload: an Erdos-Renyi bipartite graph (50k x 50k, 5M
edges) with 20 planted K_{40,40}; (4,4), (6,6), (8,8) and (4,8) counts, whose
planted part reaches 20 * C(40,8)^2 ~ 1.2e17 at (8,8) (beyond 2^53).  The
oracle cannot walk every tree here, so the GPU is checked by agreement of the
two anchors (different search trees), per-root counts on sampled roots --
including planted-block members -- and the planted lower bound."""
import math

import numpy as np
import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu


def _rank_order(deg, members):
    return sorted(members, key=lambda x: (int(deg[x]), int(x)))


@pytest.fixture(scope="module")
def dense():
    g = bipgen.workload_dense_core()
    blocks = bipgen.planted_blocks(3, 50_000, 50_000, 20, 40)
    return g, blocks


@pytest.mark.parametrize("p,q", [(4, 4), (6, 6), (8, 8), (4, 8)])
def test_dense_core_counts(gpu_ctx, dense, p, q):
    g, blocks = dense
    h = gpu_ctx.load(g)
    n_u = h.count_ex(p, q, anchor="U", time_limit_ms=120_000)[0]
    if p == q:
        assert h.count_ex(p, q, anchor="V", time_limit_ms=120_000)[0] == n_u
    assert h.count(p, q) == n_u
    if p == q:
        # every planted block alone holds C(40,p) * C(40,q) bicliques; distinct
        # blocks' bicliques are distinct, and ER edges can only add more
        assert n_u >= len(blocks) * math.comb(40, p) * math.comb(40, q)
    tot, per = h.count_per_root(p, q, "U")
    assert tot == n_u
    deg = np.diff(g.off_u)
    rng = np.random.default_rng(p * 10 + q)
    sample = set(int(x) for x in rng.choice(g.n_u, 40, replace=False))
    for lu, _ in blocks[:6]:
        order = _rank_order(deg, lu)
        # high-ranked members root small trees; low-ranked ones the largest
        sample.update(int(x) for x in (order[-4:] if p + q >= 12 else order))
    for r in sorted(sample):
        assert per[r] == oracle.count(g, p, q, roots=(r, r + 1)), r
    h.close()
