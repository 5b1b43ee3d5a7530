"""Write tests/golden/serving_counts.json from the oracle (run by hand; never by the tests).

The served-count test submits every (p, q) in {1..5}^2 on four small graphs;
some of those counts take the oracle minutes ((5,1) walks every 5-set), so
they are computed once here.  Every value comes from ``oracle`` on graphs
drawn by ``bipgen`` and is keyed by the graph's SHA-256; nothing is taken from
the CUDA library.

    python tests/golden/make_serving_golden.py
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bipgen  # noqa: E402


def serving_graphs():
    """The graphs of the served-count test (tests/test_gpu_serving.py)."""
    return [bipgen.workload_small(),
            bipgen.disjoint_union(bipgen.chung_lu(31, 3000, 2000, 24000, 2.0, 2.0), bipgen.complete(70, 110),
                                  bipgen.tiny_random(9, 60, 80, 0.5)),
            bipgen.complete(20, 30), bipgen.chung_lu(8, 500, 700, 6000, 2.1, 2.1)]


def _one(args):
    import oracle
    gi, p, q = args
    return gi, p, q, oracle.count(serving_graphs()[gi], p, q)


def main():
    gs = serving_graphs()
    jobs = [(gi, p, q) for gi in range(len(gs)) for p in range(1, 6) for q in range(1, 6)]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_one, jobs)
    out = {"about": "oracle counts (Sec. III-A Basic model, Def. 2 priority) of every (p,q) in {1..5}^2 on the "
                    "four graphs of the served-count test, keyed by graph SHA-256",
           "graphs": {}}
    for gi, g in enumerate(gs):
        out["graphs"][str(gi)] = {"sha256": bipgen.graph_sha256(g),
                                  "counts": {f"{p},{q}": str(v) for gj, p, q, v in res if gj == gi}}
    with open(os.path.join(HERE, "serving_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
