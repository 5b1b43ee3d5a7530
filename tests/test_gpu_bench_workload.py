"""Parity at full size on the benchmark's workload: the 2M-edge power-law graph
(Chung-Lu seed 2, 200k x 100k, exponents 2.0 / 2.3) with the p = q = 2..6
counts the benchmark times, each through the anchor the library picks.

The oracle cannot walk every tree here (10^12 leaves at p = q = 5), so the GPU
is checked by sampled per-root counts against the oracle, one root at a time,
and, for p = q >= 4, by agreement of the two anchors, whose search trees share
nothing.  Roots are sampled uniformly from those of at most 64 neighbours (most
of them; the oracle walks each in well under a second), plus three of 65 to 128
neighbours, whose trees are deep at p = q = 5 and 6 (a second or two of oracle
time each), plus, for p = q <= 4, the largest roots of at most 64 neighbours."""
import numpy as np
import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def powerlaw():
    return bipgen.workload_powerlaw_2m()


@pytest.mark.parametrize("k,n_sample", [(2, 24), (3, 24), (4, 16), (5, 12), (6, 8)])
def test_sampled_roots_match_the_oracle(gpu_ctx, powerlaw, k, n_sample):
    g = powerlaw
    h = gpu_ctx.load(g)
    total, info = h.count_ex(k, k)
    anchor = info["anchor"]
    tot, per = h.count_per_root(k, k, anchor)
    assert tot == total
    deg = np.diff(g.off_u if anchor == "U" else g.off_v)
    light = np.flatnonzero(deg <= 64)
    rng = np.random.default_rng(100 + k)
    sample = [int(x) for x in rng.choice(light, n_sample, replace=False)]
    mid = np.flatnonzero((deg > 64) & (deg <= 128))
    sample += [int(x) for x in rng.choice(mid, 3, replace=False)]
    if k <= 4:
        sample += [int(x) for x in light[np.argsort(deg[light])[-3:]]]
    for r in sample:
        assert per[r] == oracle.count(g, k, k, anchor=anchor, roots=(r, r + 1)), (k, anchor, r)
    h.close()


@pytest.mark.parametrize("k", [4, 5, 6])
def test_anchors_agree(gpu_ctx, powerlaw, k):
    h = gpu_ctx.load(powerlaw)
    n_u = h.count_ex(k, k, anchor="U", time_limit_ms=60_000)[0]
    n_v = h.count_ex(k, k, anchor="V", time_limit_ms=60_000)[0]
    assert n_u == n_v
    h.close()
