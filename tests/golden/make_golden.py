"""Write tests/golden/workloads.json from the oracle (run by hand; never by the tests).

Every expected value here comes from ``oracle`` on graphs drawn by ``bipgen``;
nothing is taken from the CUDA library.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bipgen  # noqa: E402
import oracle  # noqa: E402


def main():
    g = bipgen.workload_small()
    out = {
        "about": "Chung-Lu seed 1, |U|=2000, |V|=3000, |E|=20000, exponent 2.1 on both sides; "
                 "counts from the oracle (Sec. III-A Basic model with the Def. 2 priority)",
        "sha256": bipgen.graph_sha256(g),
        "counts": {},
    }
    for p, q in [(1, 1), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3), (3, 4), (4, 3), (4, 4), (5, 5), (2, 6), (6, 2)]:
        out["counts"][f"{p},{q}"] = str(oracle.count(g, p, q))
    small = bipgen.chung_lu(7, 300, 400, 3000, 2.1, 2.1)
    out["small_sha256"] = bipgen.graph_sha256(small)
    with open(os.path.join(HERE, "workloads.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
