#!/usr/bin/env python
"""Benchmark: time per exact (p,q)-biclique count on one GB300.

Workload: the Chung-Lu power-law bipartite graph of seed 2 (|U| = 200k,
|V| = 100k, |E| = 2M, degree exponents 2.0 on U and 2.3 on V, int32 CSR on both
sides), counted for p = q in {2, 3, 4, 5, 6}.  One step is that whole sweep
(five counts, every stage of the search on the device).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbc|reference]

Prints one JSON line.  value = device time per count with the graph already
resident in HBM (CUDA events on the library's stream, max over ranks);
e2e = the same through the public API from pinned host CSR arrays (load,
copy, validate, index, count, read back) per step.  --impl reference times
the CPU oracle on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank counts its own replica of the sweep (weak
scaling); only a barrier and the max-time reduction cross ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bipgen  # noqa: E402

WORKLOAD = ("chung-lu seed 2: |U|=200000 |V|=100000 |E|=2000000, exponents 2.0 (U) / 2.3 (V), "
            "int32 CSR both sides; sweep p=q in {2,3,4,5,6}")
METRIC = "time per (p,q) count"
L2_FLUSH_BYTES = 512 << 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbc", choices=["gbc", "reference"])
    ap.add_argument("--pq", default="2,3,4,5,6", help="p = q values of one step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the dense-core timings and the batched-vs-plain comparison of the default line")
    ap.add_argument("--no-roofline", action="store_true",
                    help="skip the untimed statistics pass and microbenchmarks behind the roofline")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "batch", "serve", "ablation", "border"],
                    help="sweep: p=q in 2..6 on the 2M-edge graph; batch: 256 graphs, batched vs plain; "
                         "serve: Poisson query stream over 8 resident graphs; ablation: bitmap vs sorted-list "
                         "(CSR) sets on the 2M-edge and dense-core graphs; border: the per-root position "
                         "orders (most shared first, degree order, Border's order) on the 2M-edge graph")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="size factor of the serving graphs (1 = stated)")
    ap.add_argument("--serve-limit-ms", type=int, default=30_000, help="per-request device deadline when serving")
    ap.add_argument("--serve-per-rate", type=int, default=120, help="queries per arrival rate")
    ap.add_argument("--serve-workers", default="1,4",
                    help="server worker counts to run the rate sweep with (comma-separated)")
    return ap.parse_args()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm).  The oracle counted every
# workload count to completion once, on all roots, with each root's time
# (tests/golden/full_counts.json, written by tests/golden/oracle_full_counts.py).
# Here it re-times a fixed sample of those roots -- the same roots every run,
# drawn with probability proportional to their time -- on this host's cores, and
# scales the full run by the ratio of the two timings of the same roots:
#     est. core-seconds here = (sum of sample times here / sum of their stored
#     times) x stored core-seconds of the full count,
# and wall time on `cores` processes = that / cores.
FULL_COUNTS = os.path.join(ROOT, "tests", "golden", "full_counts.json")


def _oracle_pool_init(graph_fn):
    global _ORC_G
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    _ORC_G = getattr(bipgen, graph_fn)()


def _oracle_root_task(args):
    import oracle
    k, q, anchor, root = args
    t0 = time.perf_counter()
    oracle.count(_ORC_G, k, q, anchor=anchor, roots=(root, root + 1))
    return args, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class OracleSample:
    """The stored fixed samples of a workload's counts, timed on this host's
    cores by one spawned oracle process per core (the graph is drawn once per
    process, before the clock starts)."""

    def __init__(self, workload: str, graph_fn: str, pairs, cores: int):
        rec = json.load(open(FULL_COUNTS))[workload]["counts"]
        self.pairs, self.missing, self.stored, self.partial = [], [], {}, {}
        for p, q in pairs:
            r = rec.get(f"{p},{q}")
            if r is None or "count" not in r:
                self.missing.append((p, q))
                if r is not None and "per_root_done" in r:
                    self.partial[(p, q)] = r  # an unfinished run: its core-seconds are a lower bound
                continue
            self.pairs.append((p, q))
            self.stored[(p, q)] = r
        # p, q as the oracle takes them from the stored anchor
        self.tasks = []
        for p, q in self.pairs:
            r = self.stored[(p, q)]
            for root in r["pps_sample"]["roots"]:
                self.tasks.append((p, q, r["anchor"], int(root)))
        x86 = {(p, q, r["anchor"], int(root)): float(t)
               for (p, q), r in self.stored.items()
               for root, t in zip(r["pps_sample"]["roots"], r["pps_sample"]["oracle_s"])}
        self.stored_s = x86
        self.tasks.sort(key=lambda t: -x86[t])  # longest first
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_pool_init, initargs=(graph_fn,))
        self.pool.map(_oracle_root_task, [self.tasks[-1]] * cores if self.tasks else [])  # workers ready

    def run(self):
        """One timed pass over every sample root: (wall seconds, per-pair estimate of
        the whole count's wall time on `cores` processes, detail)."""
        t0 = time.perf_counter()
        done = self.pool.map(_oracle_root_task, self.tasks, chunksize=1)
        wall = time.perf_counter() - t0
        here = {}
        for args, t in done:
            here.setdefault((args[0], args[1]), []).append((t, self.stored_s[args]))
        est, detail = {}, []
        for p, q in self.pairs:
            r = self.stored[(p, q)]
            h = here.get((p, q), [])
            ratio = sum(t for t, _ in h) / max(1e-12, sum(x for _, x in h))
            core_s = ratio * float(r["oracle_core_s"])
            est[(p, q)] = max(core_s / self.cores, ratio * float(r["max_root_s"]))
            detail.append(f"({p},{q}): {len(h)} roots, here/stored time {ratio:.3f}, "
                          f"est. {core_s:.0f} core-s here; stored full run {r['oracle_wall_s']:.0f} s wall on "
                          f"{r['cores']} cores ({r['oracle_core_s']:.0f} core-s)")
        ratios = [est[pq] * self.cores / float(self.stored[pq]["oracle_core_s"]) for pq in est]
        mean_ratio = statistics.mean(ratios) if ratios else 1.0
        self.lower = {}
        for (p, q), r in self.partial.items():
            # the stored run's finished roots alone: a lower bound of the whole count
            core_s = mean_ratio * float(r["oracle_core_s"])
            self.lower[(p, q)] = core_s / self.cores
            detail.append(f"({p},{q}): at least {core_s:.0f} core-s here (stored run unfinished: "
                          f"{r['roots_done']} of {r['roots_total']} roots, the heaviest-degree first, "
                          f"{r['oracle_core_s']:.0f} core-s, scaled by the mean here/stored ratio {mean_ratio:.3f})")
        return wall, est, detail

    def close(self):
        self.pool.close()
        self.pool.join()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pqs = [int(x) for x in args.pq.split(",")]

    if args.impl == "reference":
        if rank != 0:
            return
        reference_arm(args, pqs)
        return
    if args.workload == "batch":
        batch_workload(args, rank, world, local)
        return
    if args.workload == "serve":
        serve_workload(args, rank, world, local)
        return
    if args.workload == "ablation":
        ablation_workload(args, local)
        return
    if args.workload == "border":
        border_workload(args, local)
        return

    # host-side inputs first: process pools are spawned before CUDA starts
    g = bipgen.workload_powerlaw_2m()
    extras = not args.no_extras and world == 1
    dense = bipgen.workload_dense_core() if extras else None
    batch_jobs = _batch_jobs() if extras else None
    orc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        orc = OracleSample("powerlaw2m", "workload_powerlaw_2m", [(k, k) for k in pqs], host_cores())

    import torch
    import paper_2403_07858_gb300 as gbc
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    gbc.build()

    ctx = gbc.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident graph: counts, then warm-up and timed sweeps
    h = ctx.load(g)
    ref_counts, anchors = {}, {}
    for k in pqs:
        n, info = h.count_ex(k, k)
        ref_counts[k], anchors[k] = n, info["anchor"]
        assert anchors[k] == _auto_anchor(g, k)  # the config states the library's choice
    for _ in range(args.warmup):
        for k in pqs:
            assert h.count(k, k) == ref_counts[k]
    step_ms, enum_ms, enum_words, enum_launches, launches = [], 0.0, 0, 0, 0
    tail = {}  # per p = q: the enumeration launch's longest unit and its warps' exit spread
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush outside the timed region
            barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = []
            for k in pqs:
                n, info = h.count_ex(k, k)
                assert n == ref_counts[k]
                infos.append(info)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            step_ms.append(e0.elapsed_time(e1))
            for k, info in zip(pqs, infos):
                launches += info["launches"]
                if info["set_size"] >= 4 and info["ms_enumerate"] > 0:
                    enum_ms += info["ms_enumerate"]
                    enum_launches += 1
                    tail[str(k)] = {"launch_ms": info["enum_span_ms"],
                                    "longest_unit_ms": info["enum_longest_unit_ms"],
                                    "warp_exit_spread_ms": info["enum_exit_spread_ms"]}
    clocks = clk.summary()
    # Algorithmic work of the enumeration launches (untimed): the model words
    # of the search nodes the enumeration kernel evaluates, counted by the
    # statistics pass of the same counts (equal to the oracle's instrumented
    # traversal on the graphs the tests check).
    # The kernel collapses small-C_R subtrees, so the words it executes (the
    # nodes it evaluates plus each collapsed subtree's C_L and T words) come
    # from a second statistics pass with the collapse on.
    model_words, exec_words, collapsed = {}, {}, 0
    for k in ([] if args.no_roofline else pqs):
        n, sinfo = h.count_ex(k, k, stats=True)
        assert n == ref_counts[k]
        if sinfo["words_enum"] > 0:
            model_words[k] = sinfo["words_enum"]
            enum_words += sinfo["enum_words"]
            n, xinfo = h.count_ex(k, k, stats="exec")
            assert n == ref_counts[k]
            exec_words[k] = xinfo["words_exec"]
            collapsed += xinfo["collapsed"]
    h.close()
    ms_step = statistics.mean(step_ms)
    if dist is not None:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    n_counts = len(pqs) * world
    value = ms_step / n_counts  # whole job: every rank's counts in the max-over-ranks step time

    # ---- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(x).pin_memory() for x in (g.off_u, g.adj_u, g.off_v, g.adj_v)]
        host = [x.numpy() for x in pinned]
        h2d = sum(int(x.nbytes) for x in host)
        e2e_ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = ctx.load_graph(g.n_u, g.n_v, *host)
            for k in pqs:
                assert hh.count(k, k) == ref_counts[k]
            hh.close()
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            barrier()
        em = statistics.mean(e2e_ms)
        if dist is not None:
            t = torch.tensor([em], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            em = float(t.item())
        e2e = {"value": em / n_counts, "unit": "ms", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 16 * len(pqs)}

    # ---- roofline of the dominant kernel (the enumeration).  ncu shows it bound
    # by instruction issue on the integer pipe with its bitmap rows resident in
    # L1/L2, so the roofline is ALU.  Algorithmic work per launch, as the
    # measurement plan defines it independently of the kernel's design: the
    # model words of the search nodes of the full traversal below the roots'
    # children (the oracle's instrumented tree; the statistics pass equals it)
    # -- per evaluated node ceil(d/32) C_R words, plus ceil(c/32) C_L words for
    # internal nodes -- each word one AND and one POPC.  The kernel itself
    # executes fewer: subtrees with a small C_R are counted in closed form, and
    # the words it does execute (evaluated nodes plus each collapsed subtree's
    # C_L and T words) are reported beside, with their own fraction.  Peak: the
    # POPC pipe, the narrower of the two, retires 16 results per SM per clock
    # (the register-only AND + POPC loop of gbc_measure_int_peaks reaches that
    # rate), so the SMs can do at most SMs x 16 x clock words per second.
    peaks = _peaks()
    roof = None
    if enum_launches and model_words:
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        n_sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak_words = n_sms * 16 * sm_max * 1e6
        peak_tops = 2.0 * peak_words / 1e12
        words_per_launch = sum(model_words.values()) / len(model_words)
        exec_per_launch = sum(exec_words.values()) / len(exec_words) if exec_words else None
        ops_per_launch = 2.0 * words_per_launch
        ms_per_launch = enum_ms / enum_launches
        achieved = ops_per_launch / (ms_per_launch * 1e-3) / 1e12
        micro = gbc.measure_int_peaks(local)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved / peak_tops, "traffic": _ncu_traffic(), "kernel": "k_enumerate",
                "peak_source": f"derived: {n_sms} SMs x 16 POPC/clk/SM x {sm_max:.0f} MHz max SM clock "
                               "= words/s, x 2 ops (AND + POPC) per word",
                "algorithmic_ops_per_launch": ops_per_launch, "ops_per_word": 2,
                "model_words_per_launch": words_per_launch,
                "executed_words_per_launch": exec_per_launch,
                "executed_frac": (exec_per_launch / (ms_per_launch * 1e-3) / peak_words) if exec_per_launch else None,
                "collapsed_subtrees_per_launch": collapsed / len(exec_words) if exec_words else None,
                "loaded_words_per_launch_full_traversal": enum_words / len(model_words),
                "launches": enum_launches, "ms_per_launch": ms_per_launch, "tail": tail,
                "int32_lanes_peak_tops": n_sms * 128 * sm_max * 1e6 / 1e12,
                "microbench": {
                    "and_popc_add_loop_words_per_s": micro["and_popc_words_per_s"],
                    "loop_over_derived_peak": micro["and_popc_words_per_s"] / peak_words,
                    "model_words_per_s_over_loop": words_per_launch / (ms_per_launch * 1e-3)
                                                   / micro["and_popc_words_per_s"],
                    "l2_and_popc_stream_gbs": micro["l2_bytes_per_s"] / 1e9}}

    # ---- the dense-core and the 256-graph batch workloads (extra keys of the line)
    dense_line = dense_core_timing(ctx, dense, flush) if extras else None
    batch_line = batch_comparison(ctx, batch_jobs, flush) if extras else None

    cpu = None
    if orc is not None:
        wall, est, detail = orc.run()
        orc.close()
        per_count = [est[(k, k)] if (k, k) in est else orc.lower.get((k, k)) for k in pqs]
        bounded = [k for k in pqs if (k, k) in orc.lower]
        per_count = [x for x in per_count if x is not None]
        none = [pq for pq in orc.missing if pq not in orc.lower]
        cpu = {"value": 1e3 * statistics.mean(per_count) if per_count else None, "unit": "ms",
               "cores": orc.cores, "kind": "oracle",
               "lower_bound": bool(bounded),
               "sample": f"fixed sample of {len(orc.tasks)} roots (the same every run, drawn with probability "
                         f"proportional to their time in the stored full oracle run), timed here in {wall:.1f} s "
                         f"on {orc.cores} processes; each whole count = stored full-run core-seconds x "
                         f"(time here / stored time of the same roots) / cores; " + "; ".join(detail)
                         + (f"; the mean is a lower bound: p=q={bounded} only from the roots an unfinished run "
                            "completed" if bounded else "")
                         + ("; no stored run for " + str(none) if none else "")}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 bitmaps, u128 counts", "data": "synthetic",
            "config": sweep_config(g, pqs, world),
            "counts": {str(k): str(ref_counts[k]) for k in pqs},
            "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": launches,
            "dense_core": dense_line, "batch": batch_line,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def _batch_job(seed):
    return bipgen.batch_job(seed)


def _batch_jobs():
    """The 256 jobs of the batch workload, drawn in a spawned process pool."""
    with mp.get_context("spawn").Pool(min(32, host_cores())) as pool:
        return pool.map(_batch_job, range(100, 356), chunksize=1)


DENSE_PAIRS = [(4, 4), (6, 6), (8, 8), (4, 8)]


def dense_core_timing(ctx, g, flush, reps=2):
    """Device time of each count of the dense-core workload (50k x 50k ER, 5M
    edges, 20 planted K_{40,40}), graph resident, one untimed count first; each
    count checked against the oracle's stored whole count."""
    import torch
    stored = json.load(open(FULL_COUNTS))["dense_core"]
    assert stored["sha256"] == bipgen.graph_sha256(g)
    h = ctx.load(g)
    stream = torch.cuda.current_stream()
    out = {"workload": "Erdos-Renyi seed 3, 50000 x 50000, 5000000 edges + 20 planted K_{40,40} "
                       f"({g.n_edges} edges)", "reps": reps, "pairs": {}}
    for p, q in DENSE_PAIRS:
        n = h.count(p, q)
        ms = []
        for _ in range(reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            assert h.count(p, q) == n
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out["pairs"][f"{p},{q}"] = {"ms": statistics.mean(ms), "count": str(n),
                                    "equals_oracle": n == int(stored["counts"][f"{p},{q}"]["count"])}
    h.close()
    return out


def batch_comparison(ctx, jobs, flush, reps=3):
    """Queries/s of one gbc_count_batch over the 256-graph batch against 256 plain
    gbc_count calls on the same resident graphs (autotuned anchors, identical
    counts asserted), `reps` timed passes each after one untimed pass."""
    import torch
    hs = [ctx.load(g) for g, _, _ in jobs]
    ps = [p for _, p, _ in jobs]
    qs = [q for _, _, q in jobs]
    ctx.autotune(hs, ps, qs, time_limit_ms=30_000)
    ref = [h.count(p, q) for h, p, q in zip(hs, ps, qs)]
    assert ctx.count_batch(hs, ps, qs) == ref

    def timed(fn):
        out = []
        for _ in range(reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
            assert res == ref
        return statistics.mean(out)

    t_batch = timed(lambda: ctx.count_batch(hs, ps, qs))
    t_plain = timed(lambda: [h.count(p, q) for h, p, q in zip(hs, ps, qs)])
    # where the time goes: each job alone (plain), and the comparison again
    # without the ten longest jobs
    alone = []
    for i, (h, p, q) in enumerate(zip(hs, ps, qs)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.count(p, q)
        torch.cuda.synchronize()
        alone.append((time.perf_counter() - t0, i))
    alone.sort(reverse=True)
    rest = sorted(i for _, i in alone[10:])
    sub = ([hs[i] for i in rest], [ps[i] for i in rest], [qs[i] for i in rest])
    ref_rest = [ref[i] for i in rest]

    def timed_rest(fn):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
            assert res == ref_rest
        return statistics.mean(out)

    tb_rest = timed_rest(lambda: ctx.count_batch(*sub))
    tp_rest = timed_rest(lambda: [h.count(p, q) for h, p, q in zip(*sub)])
    total_alone = sum(t for t, _ in alone)
    top = alone[0][1]
    tuned_warps = sum(1 for h, p, q in zip(hs, ps, qs) if h.tuned_warps(p, q))
    for h in hs:
        h.close()
    return {"workload": BATCH_WORKLOAD, "queries": len(jobs), "reps": reps,
            "batched_qps": len(jobs) / t_batch, "plain_qps": len(jobs) / t_plain,
            "batched_over_plain": t_plain / t_batch, "identical_counts": True,
            "largest_job": {"p": ps[top], "q": qs[top], "edges": int(jobs[top][0].n_edges),
                            "share_of_plain": alone[0][0] / total_alone},
            "ten_largest_share_of_plain": sum(t for t, _ in alone[:10]) / total_alone,
            "without_ten_largest": {"queries": len(rest), "batched_qps": len(rest) / tb_rest,
                                    "plain_qps": len(rest) / tp_rest, "batched_over_plain": tp_rest / tb_rest},
            "autotuned_warps_kept": tuned_warps,
            "how": "host wall clock around each pass (synchronised), graphs resident"}


BATCH_WORKLOAD = ("256 chung-lu graphs, seeds 100..355: |E| = 10^U[3,6], |U|:|V| ratio U[0.25,4], "
                  "exponent U[1.9,2.6] on both sides, (p,q) uniform in {2..6}^2")


def batch_workload(args, rank, world, local):
    """Queries/s of one gbc_count_batch over the 256-graph batch against 256 plain
    gbc_count calls on the same resident graphs (same anchors, same counts)."""
    import torch
    import paper_2403_07858_gb300 as gbc
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    gbc.build()
    jobs = [bipgen.batch_job(s) for s in range(100, 356)]
    ctx = gbc.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    hs = [ctx.load(g) for g, _, _ in jobs]
    ps = [p for _, p, _ in jobs]
    qs = [q for _, _, q in jobs]
    ctx.autotune(hs, ps, qs, time_limit_ms=30_000)
    ref = [h.count(p, q) for h, p, q in zip(hs, ps, qs)]
    for _ in range(args.warmup):
        assert ctx.count_batch(hs, ps, qs) == ref
        assert [h.count(p, q) for h, p, q in zip(hs, ps, qs)] == ref

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(fn):
        out = []
        for _ in range(args.steps):
            flush.fill_(1)
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
            assert res == ref
            barrier()
        return statistics.mean(out)

    with ClockSampler(local) as clk:
        t_batch = timed(lambda: ctx.count_batch(hs, ps, qs))
        t_plain = timed(lambda: [h.count(p, q) for h, p, q in zip(hs, ps, qs)])
    clocks = clk.summary()
    if dist is not None:
        t = torch.tensor([t_batch, t_plain], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_batch, t_plain = float(t[0]), float(t[1])
    n_q = len(jobs) * world
    e2e = None
    if not args.no_e2e:
        pinned = [[torch.from_numpy(x).pin_memory().numpy() for x in (g.off_u, g.adj_u, g.off_v, g.adj_v)]
                  for g, _, _ in jobs]
        h2d = sum(int(x.nbytes) for arrs in pinned for x in arrs)
        tt = []
        for _ in range(args.steps):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = [ctx.load_graph(g.n_u, g.n_v, *arrs) for (g, _, _), arrs in zip(jobs, pinned)]
            res = ctx.count_batch(hh, ps, qs)
            for x in hh:
                x.close()
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t0)
            assert res == ref
        e2e = {"value": n_q / statistics.mean(tt), "unit": "queries/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 16 * len(jobs)}
    if rank == 0:
        out = {
            "metric": "batched queries/s", "value": n_q / t_batch, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 bitmaps, u128 counts", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "queries_per_step": len(jobs),
                       "l2": "512 MiB written between timed steps",
                       "anchors": "autotuned (both sides timed once, faster kept)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "plain": {"value": n_q / t_plain, "unit": "queries/s", "ms_per_step": t_plain * 1e3,
                      "how": "256 sequential gbc_count calls on the same resident graphs"},
            "batched_over_plain": t_plain / t_batch,
            "e2e": e2e, "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    for h in hs:
        h.close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def serve_workload(args, rank, world, local):
    """Poisson query streams at rising rates against the continuous-batching
    server; latency = completion - arrival.  The single-stream service rate is
    measured first with sequential plain counts of the same query stream."""
    import concurrent.futures as cf
    import numpy as np
    import torch
    import paper_2403_07858_gb300 as gbc
    torch.cuda.set_device(local)
    gbc.build()
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(8) as pool:
        graphs = pool.starmap(bipgen.serving_graph, [(i, args.serve_scale) for i in range(8)])
    t_gen = time.perf_counter() - t0
    ctx = gbc.Context(local)
    hs = [ctx.load(g) for g in graphs]
    lim = args.serve_limit_ms
    stream = bipgen.serving_queries(24 + 5 * args.serve_per_rate, seed=600)
    # single stream: sequential plain counts of the first 24 queries
    alone, serv_ms, single_answered = {}, [], 0
    for (gi, p, q) in stream[:24]:
        t = time.perf_counter()
        try:
            alone[(gi, p, q)] = hs[gi].count_ex(p, q, time_limit_ms=lim)[0]
            single_answered += 1
        except gbc.CountTimeout:
            alone[(gi, p, q)] = "timeout"
        serv_ms.append((time.perf_counter() - t) * 1e3)
    # queries/s of one stream, every query (answered or past its deadline) taking
    # its time: the base of the offered rates
    mu = 1e3 / statistics.mean(serv_ms)
    # answered queries/s of one stream: the figure the server's answered rate compares with
    single_qps = single_answered / (sum(serv_ms) / 1e3)
    configs = []
    mismatches = 0
    for n_workers in [int(x) for x in args.serve_workers.split(",") if x]:
        ctx.serve_start(workers=n_workers, max_batch=64, max_queue=100_000, time_limit_ms=lim)
        rng = np.random.default_rng(601)
        rates = []
        for ri, f in enumerate([0.25, 0.5, 1.0, 2.0, 4.0]):
            lam = f * mu
            qs = stream[:24] + stream[24 + ri * args.serve_per_rate: 24 + (ri + 1) * args.serve_per_rate]
            # about a minute of arrivals per rate, at least 8 queries
            qs = qs[:int(min(len(qs), max(8, lam * 60)))]
            arrivals = np.cumsum(rng.exponential(1.0 / lam, len(qs)))
            done_at, status = [None] * len(qs), [None] * len(qs)
            pool = cf.ThreadPoolExecutor(max_workers=64)
            start = time.perf_counter()
            futs = []

            def wait(i, ticket):
                try:
                    v = ctx.poll(ticket, -1)
                    status[i] = v
                except gbc.CountTimeout:
                    status[i] = "timeout"
                except gbc.GbcError as e:
                    status[i] = f"error {e.status}: {str(e)[:400]}"
                done_at[i] = time.perf_counter() - start

            for i, (gi, p, q) in enumerate(qs):
                now = time.perf_counter() - start
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                futs.append(pool.submit(wait, i, ctx.submit(hs[gi], p, q)))
            for fu in futs:
                fu.result()
            pool.shutdown()
            lat = [done_at[i] - arrivals[i] for i in range(len(qs))]
            answered = [i for i in range(len(qs)) if isinstance(status[i], int)]
            lat_ok = [lat[i] for i in answered] or [float("nan")]
            for i, key in enumerate(qs[:min(24, len(qs))]):
                # a query that finished alone may pass its deadline in a crowded mix:
                # only two finished counts can disagree
                if isinstance(alone[key], int) and isinstance(status[i], int) and status[i] != alone[key]:
                    mismatches += 1
            span = max(done_at) - arrivals[0]
            rates.append({"offered_qps": lam, "factor": f, "queries": len(qs), "answered": len(answered),
                          "served_qps": len(answered) / span,
                          "p50_ms": 1e3 * float(np.percentile(lat_ok, 50)),
                          "p99_ms": 1e3 * float(np.percentile(lat_ok, 99)),
                          "p99_all_ms": 1e3 * float(np.percentile(lat, 99)),
                          "timeouts": sum(1 for x in status if x == "timeout"),
                          "errors": sum(1 for x in status if isinstance(x, str) and x != "timeout"),
                          "error_kinds": sorted({x for x in status if isinstance(x, str) and x != "timeout"})})
        stats = ctx.serve_stats()
        ctx.serve_stop()
        configs.append({"workers": n_workers, "best_served_qps": max(r["served_qps"] for r in rates),
                        "rates": rates, "server": stats})
    best_cfg = max(configs, key=lambda c: c["best_served_qps"])
    best = best_cfg["best_served_qps"]
    if rank == 0:
        out = {"metric": "batched queries/s, p99 latency", "value": best, "unit": "queries/s",
               "n_gpus": world, "steps": 5 * len(configs), "warmup": 0, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "u32 bitmaps, u128 counts", "data": "synthetic",
               "config": {"workload": f"8 resident chung-lu graphs (exponent 2.1): seed 500 with "
                                      f"{graphs[0].n_u}/{graphs[0].n_v}/{graphs[0].n_edges} vertices/edges, "
                                      f"seeds 501..507 |E| log-uniform in [1e5,1e7] x {args.serve_scale}; "
                                      "queries: graph uniform, p,q uniform in {2..8}, Poisson arrivals",
                          "scale": args.serve_scale, "per_request_limit_ms": lim,
                          "workers": best_cfg["workers"], "graph_generation_s": t_gen},
               "single_stream_qps": single_qps,
               "single_stream": {"queries": 24, "answered": single_answered, "answered_qps": single_qps,
                                 "service_rate_qps": mu,
                                 "how": "the first 24 queries as sequential plain counts with the same deadline; "
                                        "answered_qps counts answered queries only, service_rate_qps every "
                                        "query (the base of the offered rates)"},
               "served_over_single_stream": best / single_qps if single_qps > 0 else None,
               "rates": best_cfg["rates"], "by_workers": configs,
               "served_equals_alone_mismatches": mismatches,
               "value_is": "answered queries/s (requests past their deadline are counted apart, as timeouts), "
                           "best over the rates and worker counts; p50/p99 over answered requests, p99_all over all",
               "server": best_cfg["server"]}
        print(json.dumps(out), flush=True)
    for h in hs:
        h.close()
    ctx.close()


def ablation_workload(args, local, limit_ms=60_000):
    """Device time of the same counts with bitmap sets (the library's kernels)
    and with sorted-list sets intersected by binary search (the CSR
    representation of Sec. III-B), same search trees, graph resident: one
    untimed count, then `steps` timed counts each (the CSR counts stop at
    limit_ms)."""
    import torch
    import paper_2403_07858_gb300 as gbc
    torch.cuda.set_device(local)
    gbc.build()
    ctx = gbc.Context(local)
    rows = []
    for name, g, pairs in [("chung-lu seed 2, 200k x 100k, 2M edges", bipgen.workload_powerlaw_2m(),
                            [(3, 3), (4, 4), (5, 5), (6, 6)]),
                           ("dense core, 50k x 50k ER 5M edges + 20 planted K_{40,40}", bipgen.workload_dense_core(),
                            DENSE_PAIRS)]:
        h = ctx.load(g)
        for p, q in pairs:
            n, info = h.count_ex(p, q)
            row = {"graph": name, "p": p, "q": q, "anchor": info["anchor"], "count": str(n)}
            # the bitmap kernel with its subtree collapse off walks the same tree as
            # the CSR kernel (the representation alone differs); with it on, the
            # library's default, beside
            for kern, collapse in (("bitmap", False), ("csr", False), ("bitmap_collapse", True)):
                ms, ok = [], True
                for rep in range(1 + max(1, args.steps)):
                    try:
                        m, inf = h.count_ex(p, q, anchor=info["anchor"], kernel=kern.split("_")[0],
                                            collapse=collapse,
                                            time_limit_ms=limit_ms if kern == "csr" else 0)
                    except gbc.CountTimeout:
                        ok = False
                        break
                    assert m == n
                    if rep:
                        ms.append((inf["ms_total"], inf["ms_enumerate"]))
                row[kern] = ({"ms_total": statistics.mean(a for a, _ in ms),
                              "ms_enumerate": statistics.mean(b for _, b in ms)} if ok
                             else {"over_limit_ms": limit_ms})
            if "ms_total" in row["csr"]:
                row["csr_over_bitmap"] = row["csr"]["ms_total"] / row["bitmap"]["ms_total"]
            rows.append(row)
            print(json.dumps(row), flush=True)
        h.close()
    ctx.close()
    print(json.dumps({"metric": "time per (p,q) count, bitmap vs sorted-list (CSR) sets", "unit": "ms",
                      "steps": args.steps, "rows": rows,
                      "how": "device time (CUDA events on the library's stream) of gbc_count_ex with "
                             "kernel = bitmap and kernel = csr, the same anchor and search tree (subtree "
                             "collapse off); bitmap_collapse: the bitmap kernel with its default collapse"}),
          flush=True)


def _relabel(g, new_u, new_v):
    """g with vertex u of U renamed new_u[u] and v of V renamed new_v[v]."""
    import numpy as np
    us = np.repeat(np.arange(g.n_u), np.diff(g.off_u))
    return bipgen.from_edges(g.n_u, g.n_v, np.asarray(new_u)[us], np.asarray(new_v)[np.asarray(g.adj_u)])


def border_workload(args, local, iterations=20_000):
    """Bit order of the per-root C_R bitmaps on the 2M-edge graph (Sec. V-B):
    most shared position first (the library's default), the other side's
    degree order, and Border's order of the other side.  For the last two the
    anchor side is renumbered by degree, the other side by degree or by
    gbc_border_order, and the graph is loaded with its ids kept.  Reports the
    enumeration's device time and the C_R words it loads per evaluated child
    (its span-truncated reads, from a statistics pass)."""
    import numpy as np
    import torch
    import paper_2403_07858_gb300 as gbc
    torch.cuda.set_device(local)
    gbc.build()
    g = bipgen.workload_powerlaw_2m()

    def degree_ids(off):
        deg = np.diff(off)
        order = np.argsort(-deg, kind="stable")
        ids = np.empty(len(deg), dtype=np.int64)
        ids[order] = np.arange(len(deg))
        return ids

    ctx = gbc.Context(local)
    rows = []
    for k, anchor in [(4, "U"), (5, "V"), (6, "V")]:
        if anchor == "U":
            a_ids = degree_ids(g.off_u)
            nA, nO, off, adj = g.n_u, g.n_v, g.off_u, g.adj_u
        else:
            a_ids = degree_ids(g.off_v)
            nA, nO, off, adj = g.n_v, g.n_u, g.off_v, g.adj_v
        t0 = time.perf_counter()
        border_ids, ob_before, ob_after = gbc.border_order(nA, nO, off, adj, iterations=iterations, max_cand=64)
        t_border = time.perf_counter() - t0
        deg_ids, _, _ = gbc.border_order(nA, nO, off, adj, iterations=0, max_cand=64)
        variants = [("most shared first (default)", g, False, "shared")]
        for name, o_ids in [("other side's degree order", deg_ids), ("Border's order", border_ids)]:
            gg = _relabel(g, a_ids, o_ids) if anchor == "U" else _relabel(g, o_ids, a_ids)
            variants.append((name, gg, True, "id"))
        want = None
        for name, gg, keep, order in variants:
            h = ctx.load(gg, keep_ids=keep)
            n, info = h.count_ex(k, k, anchor=anchor, position_order=order)
            want = n if want is None else want
            assert n == want
            ms = []
            for _ in range(max(1, args.steps)):
                _, inf = h.count_ex(k, k, anchor=anchor, position_order=order)
                ms.append(inf["ms_enumerate"])
            _, st = h.count_ex(k, k, anchor=anchor, position_order=order, stats=True)
            evals = sum(st["evals"][3:])
            rows.append({"p": k, "q": k, "anchor": anchor, "order": name, "ms_enumerate": statistics.mean(ms),
                         "loaded_words": st["enum_words"], "evaluated_children": evals,
                         "words_per_child": st["enum_words"] / max(1, evals), "count": str(n)})
            print(json.dumps(rows[-1]), flush=True)
            h.close()
        rows.append({"p": k, "q": k, "anchor": anchor, "border_iterations": iterations,
                     "one_blocks_degree_order": ob_before, "one_blocks_border": ob_after, "border_s": t_border})
        print(json.dumps(rows[-1]), flush=True)
    ctx.close()
    print(json.dumps({"metric": "enumeration time and C_R words per evaluated child by position order",
                      "graph": WORKLOAD, "steps": args.steps, "rows": rows}), flush=True)


def kernel_source_digest() -> str:
    """SHA-256 of the enumeration kernels' source with comments and whitespace
    removed: it changes when the code does, not when a comment does."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_2403_07858_gb300", "csrc", "gbc_search.cu")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256("".join(src.split()).encode()).hexdigest()


def _ncu_traffic():
    """dram bytes per launch of the enumeration kernel from the committed ncu
    summary, if it was taken on the current kernel code; else None."""
    path = os.path.join(ROOT, "profiles", "enumerate_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("source_digest") != kernel_source_digest():
        return None
    return rec.get("dram_bytes_per_launch_scaled")


def _auto_anchor(g, k):
    """The library's anchor rule for p = q = k (the oracle counts the same from
    either side): up to k = 4 the side whose 2-hop wedges through the other side
    are fewer, from k = 5 the side with the lighter own degree tail."""
    import numpy as np
    du = np.diff(g.off_u).astype(np.int64)
    dv = np.diff(g.off_v).astype(np.int64)
    if k == 1:
        return "U"
    wedges_u = int((du * (du - 1) // 2).sum())  # wedges centred on U vertices
    wedges_v = int((dv * (dv - 1) // 2).sum())
    if k <= 4:
        return "U" if wedges_v <= wedges_u else "V"
    return "U" if wedges_u <= wedges_v else "V"


def sweep_config(g, pqs, world=1):
    """The config object of the sweep line (both arms print the same)."""
    return {"workload": WORKLOAD, "graph_sha256": bipgen.graph_sha256(g), "counts_per_step": len(pqs),
            "anchor": {str(k): _auto_anchor(g, k) for k in pqs},
            "l2": "512 MiB written between timed steps (outside the events); per-count "
                  "scratch also exceeds L2",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def reference_arm(args, pqs):
    """The oracle on this host's cores.  Each step times the same fixed sample of
    roots of every count (stored with the oracle's full run) and scales the full
    run's core-seconds by the ratio of the two timings of those roots; the value
    is the resulting time per whole count on all host cores, and ms_per_step is
    the measured wall time of the step (the sample)."""
    g = bipgen.workload_powerlaw_2m()
    cores = host_cores()
    orc = OracleSample("powerlaw2m", "workload_powerlaw_2m", [(k, k) for k in pqs], cores)
    for _ in range(args.warmup):
        orc.run()
    walls, values, detail = [], [], []
    for _ in range(args.steps):
        wall, est, detail = orc.run()
        walls.append(wall)
        per = [est[(k, k)] if (k, k) in est else orc.lower.get((k, k)) for k in pqs]
        values.append(1e3 * statistics.mean(x for x in per if x is not None))
    orc.close()
    v = statistics.mean(values)
    bounded = [k for k in pqs if (k, k) in orc.lower]
    none = [pq for pq in orc.missing if pq not in orc.lower]
    sample = (f"per step: the fixed sample of {len(orc.tasks)} roots (the same every step, drawn with probability "
              f"proportional to their time in the stored full oracle run) timed on {cores} processes; each whole "
              f"count = stored full-run core-seconds x (time here / stored time of the same roots) / cores; "
              f"steps' values range {min(values):.0f}..{max(values):.0f} ms; " + "; ".join(detail)
              + (f"; the mean is a lower bound: p=q={bounded} only from the roots an unfinished run completed"
                 if bounded else "")
              + ("; no stored run for " + str(none) if none else ""))
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u128 (CPU oracle)",
        "data": "synthetic", "config": sweep_config(g, pqs),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
