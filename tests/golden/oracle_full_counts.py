"""Whole counts of the large workloads by the oracle alone (run by hand; never by the tests).

Writes tests/golden/full_counts.json.  Every stored value comes from ``oracle``
(Sec. III-A Basic model, Def. 2 priority, Alg. 1 pruning) on graphs drawn by
``bipgen``; nothing is taken from the CUDA library.

The roots of one count are independent search trees (Sec. III-B), so the script
deals them out to one oracle process per host core, sums the exact per-root
values (Python ints, no width limit) and records per root:
  * the value (the bicliques whose lowest-ranked anchor vertex is the root);
  * the oracle's wall time for that root alone.
Stored per count: the total; the anchor; a SHA-256 of the full per-root vector
in the caller's ids; the 50 roots that took the oracle longest, with their
values; the oracle's core-seconds and wall time and the core count; and a
fixed sample of roots drawn with probability proportional to their oracle
time, with those times, which the benchmark's CPU baseline re-times on the
GPU host to scale this machine's full-count time to that host.

A count whose wall time passes --budget-s is recorded as "oracle unavailable
at this size (budget X s)" instead.  With --checkpoint, every finished chunk of
roots is appended to a JSON-lines file, and a later run resumes from it (its
wall time adds up the segments).

    python tests/golden/oracle_full_counts.py --workload powerlaw2m [--cores N]
    python tests/golden/oracle_full_counts.py --workload dense_core
    python tests/golden/oracle_full_counts.py --workload powerlaw2m --only 6:6 --checkpoint ck.jsonl
    python tests/golden/oracle_full_counts.py --workload powerlaw2m --only 6:6 --checkpoint ck.jsonl \
        --store-partial --budget-s 21600
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bipgen  # noqa: E402

OUT = os.path.join(HERE, "full_counts.json")
MAX_SAMPLE = 400  # roots in a stored sample at most

# (p, q, anchor): the anchors are the ones the benchmark's counts take, so the
# per-root vectors compare with the library's per-root output directly
WORKLOADS = {
    "powerlaw2m": {
        "about": "Chung-Lu seed 2, |U|=200000, |V|=100000, |E|=2000000, exponents 2.0 (U) / 2.3 (V)",
        "make": "workload_powerlaw_2m",
        "counts": [(2, 2, "U"), (3, 3, "U"), (4, 4, "U"), (5, 5, "V"), (6, 6, "V")],
    },
    "dense_core": {
        "about": "Erdos-Renyi seed 3, 50000 x 50000, 5000000 edges, plus 20 planted K_{40,40}",
        "make": "workload_dense_core",
        "counts": [(4, 4, "U"), (6, 6, "U"), (8, 8, "U"), (4, 8, "U")],
    },
}

_G = None


def _init(make):
    global _G
    import oracle
    oracle.build()
    _G = getattr(bipgen, make)()


def _run_chunk(args):
    """Per-root values and times of a list of roots (one oracle call per root)."""
    import oracle
    p, q, anchor, roots = args
    vals, secs = [], []
    for r in roots:
        t0 = time.perf_counter()
        v = oracle.count(_G, p, q, anchor=anchor, roots=(r, r + 1))
        secs.append(time.perf_counter() - t0)
        vals.append(v)
    return roots, vals, secs


def per_root_sha256(values) -> str:
    """SHA-256 of the per-root values in root order, as decimal lines."""
    h = hashlib.sha256()
    for v in values:
        h.update(f"{int(v)}\n".encode())
    return h.hexdigest()


def pps_sample(secs: np.ndarray, target_s: float, seed: int, cap_s: float) -> list[int]:
    """Roots of at most cap_s seconds drawn with probability proportional to
    their time: systematic sampling along the cumulative time of a seeded random
    order of those roots, one pick every (their total / n) seconds, n chosen so
    the picks add to about target_s."""
    rng = np.random.default_rng(seed)
    eligible = np.flatnonzero(secs <= cap_s)
    order = eligible[rng.permutation(len(eligible))]
    secs = secs[order]
    order_pos = np.arange(len(order))
    total = float(secs.sum())
    # the expected time of n PPS picks is n * sum(t^2)/sum(t); solve for ~target_s
    mean_pick = float((secs ** 2).sum() / max(total, 1e-12))
    n = int(min(len(secs), MAX_SAMPLE, max(8, round(target_s / max(mean_pick, 1e-9)))))
    step = total / n
    cum = np.cumsum(secs[order_pos])
    picks = np.searchsorted(cum, step * (np.arange(n) + rng.random()), side="right")
    picks = np.minimum(picks, len(secs) - 1)
    return sorted({int(order[i]) for i in picks})


def _read_checkpoint(path, key):
    """Finished chunks of one count from an append-only checkpoint (JSON lines),
    and the wall time of every earlier segment of the run (its largest elapsed)."""
    chunks, seg_wall = [], {}
    if path and os.path.exists(path):
        with open(path) as f:
            for line in f:
                try:
                    rec = json.loads(line)
                except ValueError:  # a line cut off when a segment ended
                    continue
                if rec.get("k") != key:
                    continue
                chunks.append(rec)
                seg_wall[rec["seg"]] = max(seg_wall.get(rec["seg"], 0.0), rec["el"])
    return chunks, sum(seg_wall.values())


def run_count(g, make, p, q, anchor, cores, budget_s, log, checkpoint=None):
    n_a = g.n_u if anchor == "U" else g.n_v
    deg = np.diff(g.off_u if anchor == "U" else g.off_v)
    # heaviest (by degree) roots first, alone; the light tail in chunks
    order = np.argsort(-deg, kind="stable")
    chunks, i = [], 0
    while i < n_a:
        size = 1 if i < 4000 else (16 if i < 40000 else 512)
        chunks.append((p, q, anchor, [int(x) for x in order[i:i + size]]))
        i += size
    vals = [0] * n_a
    secs = np.zeros(n_a)
    key = f"{p},{q},{anchor}"
    earlier, earlier_wall = _read_checkpoint(checkpoint, key)
    finished = np.zeros(n_a, dtype=bool)
    for rec in earlier:
        for r, x, t in zip(rec["roots"], rec["vals"], rec["secs"]):
            vals[r] = int(x)
            secs[r] = t
            finished[r] = True
    todo = [c for c in chunks if not all(finished[r] for r in c[3])]
    done = int(finished.sum())
    if earlier and log:
        log(f"  ({p},{q}) anchor {anchor}: resuming with {done}/{n_a} roots from {checkpoint}, "
            f"{earlier_wall:.0f} s of earlier wall time")
    seg = f"{os.getpid()}-{time.time():.0f}"
    ckf = open(checkpoint, "a") if checkpoint else None
    t0 = time.perf_counter()
    over = False
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_init, initargs=(make,)) as pool:
        for roots, v, s in pool.imap_unordered(_run_chunk, todo):
            for r, x, t in zip(roots, v, s):
                vals[r] = x
                secs[r] = t
            done += len(roots)
            el = time.perf_counter() - t0
            if ckf:
                ckf.write(json.dumps({"k": key, "seg": seg, "el": round(el, 2), "roots": roots,
                                      "vals": [str(x) for x in v], "secs": [round(t, 5) for t in s]}) + "\n")
                ckf.flush()
            if earlier_wall + el > budget_s:
                over = True
                pool.terminate()
                break
            if log and done % 20000 < len(roots):
                log(f"  ({p},{q}) anchor {anchor}: {done}/{n_a} roots, {earlier_wall + el:.0f} s")
    if ckf:
        ckf.close()
    wall = earlier_wall + time.perf_counter() - t0
    if over:
        return {"p": p, "q": q, "anchor": anchor,
                "unavailable": f"oracle unavailable at this size (budget {budget_s:.0f} s on {cores} cores)"}
    total = sum(vals)
    heavy = np.argsort(-secs, kind="stable")[:50]
    cap = 1.0
    sample = pps_sample(secs, target_s=12.0, seed=1000 * p + q, cap_s=cap)
    return {
        "p": p, "q": q, "anchor": anchor, "count": str(total),
        "per_root_sha256": per_root_sha256(vals),
        "heaviest_roots": [{"root": int(r), "value": str(vals[int(r)]), "oracle_s": round(float(secs[r]), 4)}
                           for r in heavy],
        "oracle_core_s": round(float(secs.sum()), 2), "oracle_wall_s": round(wall, 2), "cores": cores,
        "max_root_s": round(float(secs.max()), 3),
        "pps_sample": {"roots": sample, "oracle_s": [round(float(secs[r]), 5) for r in sample],
                       "cap_s": cap, "core_s_at_most_cap": round(float(secs[secs <= cap].sum()), 2),
                       "how": "systematic sample, among the roots that took at most cap_s, with probability "
                              "proportional to the oracle time of each root on this machine (seeded order); "
                              "the sum of all roots' times is oracle_core_s"},
    }


def partial_record(g, p, q, anchor, checkpoint, budget_s):
    """The record of a count the oracle did not finish: every root of the
    checkpoint (roots taken in descending degree, the heaviest first) with its
    exact value and time, and the wall time spent."""
    chunks, wall = _read_checkpoint(checkpoint, f"{p},{q},{anchor}")
    done = {}
    for rec in chunks:
        for r, x, t in zip(rec["roots"], rec["vals"], rec["secs"]):
            done[int(r)] = (str(int(x)), round(float(t), 3))
    n_a = g.n_u if anchor == "U" else g.n_v
    cores = max(1, round(sum(t for _, t in done.values()) / max(wall, 1e-9)))
    return {"p": p, "q": q, "anchor": anchor,
            "unavailable": f"oracle unavailable at this size (budget {budget_s:.0f} s wall on about {cores} cores): "
                           f"{len(done)} of {n_a} roots finished",
            "roots_done": len(done), "roots_total": n_a,
            "order": "roots in descending degree (ties by id), the heaviest first",
            "per_root_done": {str(r): v for r, (v, _) in sorted(done.items())},
            "per_root_oracle_s": {str(r): t for r, (_, t) in sorted(done.items())},
            "oracle_core_s": round(sum(t for _, t in done.values()), 1), "oracle_wall_s": round(wall, 1)}


def trim_samples(rec: dict, seed: int = 7) -> None:
    """Cut every stored sample to at most MAX_SAMPLE roots by a seeded uniform
    subsample (a uniform subsample of a probability-proportional-to-time sample
    is still one)."""
    rng = np.random.default_rng(seed)
    for entry in rec.values():
        for res in entry.get("counts", {}).values():
            smp = res.get("pps_sample")
            if not smp or len(smp["roots"]) <= MAX_SAMPLE:
                continue
            keep = sorted(rng.choice(len(smp["roots"]), MAX_SAMPLE, replace=False).tolist())
            smp["roots"] = [smp["roots"][i] for i in keep]
            smp["oracle_s"] = [smp["oracle_s"][i] for i in keep]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trim-samples", action="store_true", help="only cut the stored samples to MAX_SAMPLE roots")
    ap.add_argument("--workload", choices=sorted(WORKLOADS))
    ap.add_argument("--cores", type=int, default=len(os.sched_getaffinity(0)))
    ap.add_argument("--budget-s", type=float, default=4 * 3600.0, help="wall-time budget per count")
    ap.add_argument("--only", default="", help="comma-separated p,q pairs as p:q (default all)")
    ap.add_argument("--checkpoint", default="",
                    help="append every finished chunk to this JSON-lines file and resume from it")
    ap.add_argument("--store-partial", action="store_true",
                    help="with --checkpoint and one --only pair: store the roots the checkpoint finished "
                         "(exact per-root values) as that count's record, marked unavailable at this size")
    args = ap.parse_args()
    if args.trim_samples:
        rec = json.load(open(OUT))
        trim_samples(rec)
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
            f.write("\n")
        return
    if not args.workload:
        ap.error("--workload is required")
    w = WORKLOADS[args.workload]
    g = getattr(bipgen, w["make"])()
    rec = json.load(open(OUT)) if os.path.exists(OUT) else {}
    entry = rec.get(args.workload, {"about": w["about"], "sha256": bipgen.graph_sha256(g), "counts": {}})
    entry["sha256"] = bipgen.graph_sha256(g)
    entry["machine"] = {"cpu": _cpu_model(), "arch": platform.machine()}
    only = {tuple(int(x) for x in s.split(":")) for s in args.only.split(",") if s}
    if args.store_partial:
        (p, q), = only
        anchor = next(a for pp, qq, a in w["counts"] if (pp, qq) == (p, q))
        entry["counts"][f"{p},{q}"] = partial_record(g, p, q, anchor, args.checkpoint, args.budget_s)
        rec[args.workload] = entry
        with open(OUT + ".tmp", "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)
        return

    def log(msg):
        print(msg, flush=True)

    for p, q, anchor in w["counts"]:
        if only and (p, q) not in only:
            continue
        log(f"{args.workload} ({p},{q}) anchor {anchor} on {args.cores} cores")
        res = run_count(g, w["make"], p, q, anchor, args.cores, args.budget_s, log,
                        checkpoint=args.checkpoint or None)
        entry["counts"][f"{p},{q}"] = res
        rec[args.workload] = entry
        with open(OUT + ".tmp", "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)
        log(f"  -> {res.get('count', res.get('unavailable'))} "
            f"({res.get('oracle_wall_s', '-')} s wall, {res.get('oracle_core_s', '-')} core-s)")


def _cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


if __name__ == "__main__":
    main()
