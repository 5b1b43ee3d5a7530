"""The dense-core workload: an Erdos-Renyi bipartite graph (50k x 50k, 5M
edges) with 20 planted K_{40,40}; (4,4), (6,6), (8,8) and (4,8) counts, whose
planted part reaches 20 * C(40,8)^2 ~ 1.2e17 at (8,8) (beyond 2^53).

The oracle counted all four to completion (tests/golden/oracle_full_counts.py):
the GPU's whole count, its whole per-root vector (SHA-256) and the oracle's 50
heaviest roots must match; the two anchors must agree and the count must
clear the planted lower bound."""
import hashlib
import json
import math
import os

import pytest

import bipgen

pytestmark = pytest.mark.gpu

FULL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_counts.json")


def _sha(values):
    h = hashlib.sha256()
    for v in values:
        h.update(f"{int(v)}\n".encode())
    return h.hexdigest()


@pytest.fixture(scope="module")
def dense():
    g = bipgen.workload_dense_core()
    blocks = bipgen.planted_blocks(3, 50_000, 50_000, 20, 40)
    rec = json.load(open(FULL))["dense_core"]
    assert rec["sha256"] == bipgen.graph_sha256(g)
    return g, blocks, rec["counts"]


@pytest.mark.parametrize("p,q", [(4, 4), (6, 6), (8, 8), (4, 8)])
def test_dense_core_counts(gpu_ctx, dense, p, q):
    g, blocks, stored = dense
    res = stored[f"{p},{q}"]
    h = gpu_ctx.load(g)
    n_u = h.count_ex(p, q, anchor="U", time_limit_ms=120_000)[0]
    assert n_u == int(res["count"])
    if p == q:
        assert h.count_ex(p, q, anchor="V", time_limit_ms=120_000)[0] == n_u
        # every planted block alone holds C(40,p) * C(40,q) bicliques; distinct
        # blocks' bicliques are distinct, and ER edges can only add more
        assert n_u >= len(blocks) * math.comb(40, p) * math.comb(40, q)
    assert h.count(p, q) == n_u
    tot, per = h.count_per_root(p, q, "U")
    assert tot == n_u
    for hr in res["heaviest_roots"]:
        assert per[hr["root"]] == int(hr["value"]), hr["root"]
    assert _sha(per) == res["per_root_sha256"]
    h.close()
