"""The whole-count script's host logic (tests/golden/oracle_full_counts.py), on
CPU: a run that stops at its budget and resumes from its checkpoint gives the
same per-root values and total as one uninterrupted run, and a stopped run's
partial record holds exactly the roots it finished, with their exact values."""
import importlib
import json
import os
import sys

import pytest

import bipgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _script():
    # importable by name, so the script's spawned oracle processes find its functions
    golden = os.path.join(HERE, "golden")
    if golden not in sys.path:
        sys.path.insert(0, golden)
    return importlib.import_module("oracle_full_counts")


def test_resumed_run_equals_one_run(tmp_path):
    sc = _script()
    g = bipgen.workload_small()
    p, q, anchor = 3, 3, "U"
    ck = str(tmp_path / "ck.jsonl")
    # a budget of 0 s stops the first segment after its first chunk
    first = sc.run_count(g, "workload_small", p, q, anchor, 2, 0.0, None, checkpoint=ck)
    assert "unavailable" in first
    done = sum(len(json.loads(line)["roots"]) for line in open(ck))
    assert 0 < done < g.n_u
    part = sc.partial_record(g, p, q, anchor, ck, 0.0)
    assert part["roots_done"] == len(part["per_root_done"]) == done
    for r, v in part["per_root_done"].items():
        assert int(v) == oracle.count(g, p, q, anchor=anchor, roots=(int(r), int(r) + 1))
    # the second segment finishes the rest
    whole = sc.run_count(g, "workload_small", p, q, anchor, 2, 1e9, None, checkpoint=ck)
    want, per = oracle.count(g, p, q, anchor=anchor, per_root=True)
    assert int(whole["count"]) == want
    assert whole["per_root_sha256"] == sc.per_root_sha256(per)


def test_partial_record_lists_no_unfinished_root(tmp_path):
    sc = _script()
    g = bipgen.workload_small()
    ck = tmp_path / "ck.jsonl"
    # a checkpoint with one finished chunk, a chunk of another count, and a cut-off line
    ck.write_text(json.dumps({"k": "4,4,V", "seg": "a", "el": 3.0, "roots": [5, 9], "vals": ["7", "0"],
                              "secs": [0.5, 0.25]}) + "\n"
                  + json.dumps({"k": "3,3,V", "seg": "a", "el": 4.0, "roots": [1], "vals": ["2"], "secs": [1.0]})
                  + "\n" + '{"k": "4,4,V", "seg"')
    rec = sc.partial_record(g, 4, 4, "V", str(ck), 100.0)
    assert rec["per_root_done"] == {"5": "7", "9": "0"}
    assert rec["roots_done"] == 2 and rec["roots_total"] == g.n_v
    assert rec["oracle_wall_s"] == pytest.approx(3.0)  # the largest elapsed time of its segment
