"""Parity on the 256-graph batch workload (seeds 100..355, |E| = 10^U[3,6],
(p,q) uniform in {2..6}^2): every job of at most 20k edges (112 of the 256)
runs in one gbc_count_batch pipeline, whole, against the oracle's full count;
the batch's larger jobs are covered by the benchmark's batched-equals-plain
check and by the full-size tests."""
import pytest

import bipgen
import oracle

pytestmark = pytest.mark.gpu


def _small_seeds(limit=20_000):
    seeds = []
    for seed in range(100, 356):
        r = bipgen.uniform(bipgen.stream_state(seed, "JOB"), 0, 5)
        if int(round(10.0 ** (3.0 + 3.0 * float(r[0])))) <= limit:
            seeds.append(seed)
    return seeds


def test_small_batch_jobs_match_the_oracle(gpu_ctx):
    jobs = [bipgen.batch_job(s) for s in _small_seeds()]
    assert len(jobs) >= 100
    hs = [gpu_ctx.load(g) for g, _, _ in jobs]
    res = gpu_ctx.count_batch(hs, [p for _, p, _ in jobs], [q for _, _, q in jobs])
    for (g, p, q), r in zip(jobs, res):
        assert r == oracle.count(g, p, q), (p, q, g.n_u, g.n_v, g.n_edges)
    for h in hs:
        h.close()
