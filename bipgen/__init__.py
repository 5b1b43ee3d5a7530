"""Seeded synthetic bipartite graphs, shared by the oracle tests and the GPU path.

This module draws graphs and nothing else: it holds none of the counting
method's arithmetic (no intersections, no binomials, no ordering of roots).
Both sides of every parity test take their inputs from here.

Determinism across machines (x86_64 here, aarch64 on the GPU host) is part of
the contract: every float used to place an edge comes from correctly rounded
IEEE-754 operations (+, -, *, /, frexp/ldexp) in a fixed order, so the same
seed gives the same graph bit for bit on both.  ``graph_sha256`` fingerprints a
graph so stored expected values can be tied to the exact input they were
computed on.

Random numbers come from SplitMix64 (S. Vigna, public domain), used in its
counter form: draw k of a stream with initial state s is mix(s + (k+1)*GAMMA).

Graph families (the workload recipes, Table 2 stand-ins):
  * ``chung_lu``   power-law bipartite graph, weights (i+1)^(-1/(gamma-1)) per
                   side clipped at sqrt(|E|), endpoints drawn independently,
                   duplicates rejected until exactly |E| distinct edges remain.
  * ``er_planted`` uniform random bipartite graph plus planted K_{k,k} blocks.
  * ``tiny_random``/``complete``/``disjoint_union``/``permute``/``swap_sides``
                   small structural helpers for the oracle's pins.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _mix_int(x: int) -> int:
    x &= _MASK
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK
    return x ^ (x >> 31)


def stream_state(seed: int, tag: str) -> int:
    """Initial SplitMix64 state of the sub-stream ``tag`` of ``seed``."""
    h = 0
    for ch in tag.encode():
        h = _mix_int(h * 131 + ch + 1)
    return _mix_int((seed & _MASK) ^ h)


def splitmix64(state: int, start: int, n: int) -> np.ndarray:
    """Draws start .. start+n-1 of the SplitMix64 stream with initial ``state``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(state) + k * _GAMMA
        return _mix(z)


def uniform(state: int, start: int, n: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    return (splitmix64(state, start, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Deterministic x^(-a) for x >= 1 from basic IEEE operations only (libm's pow,
# log and exp are not guaranteed to round identically on both machines).
# log: x = m*2^e with m in [sqrt(1/2), sqrt(2)); log m = 2*atanh(s), s=(m-1)/(m+1).
# exp: y = k*ln2 + r, |r| <= ln2/2, exp(r) by its Taylor series.
_LN2 = 0.6931471805599453


def _det_log(x: np.ndarray) -> np.ndarray:
    m, e = np.frexp(x)  # x = m * 2^e, m in [0.5, 1)
    m = m * 2.0
    e = e.astype(np.float64) - 1.0
    big = m >= 1.4142135623730951
    m = np.where(big, m * 0.5, m)
    e = np.where(big, e + 1.0, e)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    acc = np.zeros_like(s)
    for k in range(41, 0, -2):  # s^(k-1)/k Horner over odd terms
        acc = acc * s2 + 1.0 / k
    return 2.0 * s * acc + e * _LN2


def _det_exp(y: np.ndarray) -> np.ndarray:
    k = np.rint(y / _LN2)
    r = y - k * _LN2
    acc = np.ones_like(r)
    for n in range(27, 0, -1):
        acc = 1.0 + acc * r / n
    return np.ldexp(acc, k.astype(np.int64))


def powerlaw_weights(n: int, gamma: float) -> np.ndarray:
    """w_i = (i+1)^(-1/(gamma-1)), i = 0..n-1."""
    a = 1.0 / (gamma - 1.0)
    x = np.arange(1, n + 1, dtype=np.float64)
    return _det_exp(-a * _det_log(x))


def clip_rescale(w: np.ndarray, total: float, wmax: float) -> np.ndarray:
    """Scale w to sum to ``total``, then clip at ``wmax`` and rescale, repeated."""
    w = w.copy()
    for _ in range(500):
        s = math.fsum(w.tolist())
        w = w * (total / s)
        if float(w.max()) <= wmax * (1.0 + 1e-12):
            break
        w = np.minimum(w, wmax)
    return w


# ---------------------------------------------------------------------------
@dataclass
class BipartiteGraph:
    """Canonical CSR on both sides: rows sorted, no duplicates, int32."""
    n_u: int
    n_v: int
    off_u: np.ndarray  # int32 [n_u+1]
    adj_u: np.ndarray  # int32 [|E|], neighbours in V
    off_v: np.ndarray  # int32 [n_v+1]
    adj_v: np.ndarray  # int32 [|E|], neighbours in U

    @property
    def n_edges(self) -> int:
        return int(self.adj_u.shape[0])

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        us = np.repeat(np.arange(self.n_u, dtype=np.int64), np.diff(self.off_u))
        return us, self.adj_u.astype(np.int64)


def from_edges(n_u: int, n_v: int, us, vs) -> BipartiteGraph:
    """Canonical CSR pair from an edge list (duplicates removed)."""
    us = np.asarray(us, dtype=np.int64)
    vs = np.asarray(vs, dtype=np.int64)
    if us.size:
        if us.min() < 0 or us.max() >= n_u or vs.min() < 0 or vs.max() >= n_v:
            raise ValueError("edge endpoint out of range")
    key = np.unique(us * max(n_v, 1) + vs)
    us = key // max(n_v, 1)
    vs = key % max(n_v, 1)
    off_u = np.zeros(n_u + 1, dtype=np.int64)
    np.add.at(off_u, us + 1, 1)
    off_u = np.cumsum(off_u)
    adj_u = vs  # key order is (u, v) ascending
    order = np.lexsort((us, vs))
    off_v = np.zeros(n_v + 1, dtype=np.int64)
    np.add.at(off_v, vs + 1, 1)
    off_v = np.cumsum(off_v)
    adj_v = us[order]
    return BipartiteGraph(n_u, n_v, off_u.astype(np.int32), adj_u.astype(np.int32),
                          off_v.astype(np.int32), adj_v.astype(np.int32))


def graph_sha256(g: BipartiteGraph) -> str:
    h = hashlib.sha256()
    h.update(np.array([g.n_u, g.n_v, g.n_edges], dtype=np.int64).tobytes())
    for a in (g.off_u, g.adj_u, g.off_v, g.adj_v):
        h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    return h.hexdigest()


def _distinct_pairs(seed: int, n_u: int, n_v: int, n_edges: int, draw_u, draw_v):
    """First ``n_edges`` distinct (u, v) pairs of the draw sequence, in draw order."""
    keys = np.zeros(0, dtype=np.int64)
    drawn = 0
    while True:
        need = n_edges - (np.unique(keys).size if keys.size else 0)
        batch = int(need * 1.25) + 1024
        us = draw_u(drawn, batch)
        vs = draw_v(drawn, batch)
        drawn += batch
        keys = np.concatenate([keys, us.astype(np.int64) * n_v + vs.astype(np.int64)])
        _, first = np.unique(keys, return_index=True)
        if first.size >= n_edges:
            first.sort()
            keys = keys[first[:n_edges]]
            return keys // n_v, keys % n_v


def _random_perm(state: int, n: int) -> np.ndarray:
    return np.argsort(splitmix64(state, 0, n), kind="stable").astype(np.int64)


def chung_lu(seed: int, n_u: int, n_v: int, n_edges: int, gamma_u: float,
             gamma_v: float) -> BipartiteGraph:
    """Chung-Lu power-law bipartite graph with exactly ``n_edges`` distinct edges."""
    if n_edges > n_u * n_v:
        raise ValueError("more edges than vertex pairs")
    wmax = math.sqrt(n_edges)
    cum = []
    for n, g in ((n_u, gamma_u), (n_v, gamma_v)):
        w = clip_rescale(powerlaw_weights(n, g), float(n_edges), wmax)
        cum.append(np.cumsum(w))
    su, sv = stream_state(seed, "U"), stream_state(seed, "V")

    def draw(cw, st, n):
        def f(start, k):
            t = uniform(st, start, k) * cw[-1]
            return np.minimum(np.searchsorted(cw, t, side="right"), n - 1)
        return f

    us, vs = _distinct_pairs(seed, n_u, n_v, n_edges, draw(cum[0], su, n_u), draw(cum[1], sv, n_v))
    pu = _random_perm(stream_state(seed, "PU"), n_u)
    pv = _random_perm(stream_state(seed, "PV"), n_v)
    return from_edges(n_u, n_v, pu[us], pv[vs])


def er_planted(seed: int, n_u: int, n_v: int, n_edges: int, n_planted: int,
               k: int) -> BipartiteGraph:
    """Uniform random bipartite graph with ``n_edges`` distinct edges, united with
    ``n_planted`` complete K_{k,k} on random k-subsets of each side."""
    su, sv = stream_state(seed, "U"), stream_state(seed, "V")

    def draw(st, n):
        return lambda start, m: (splitmix64(st, start, m) % np.uint64(n)).astype(np.int64)

    us, vs = _distinct_pairs(seed, n_u, n_v, n_edges, draw(su, n_u), draw(sv, n_v))
    extra_u, extra_v = [], []
    for lu, lv in planted_blocks(seed, n_u, n_v, n_planted, k):
        gu, gv = np.meshgrid(lu, lv, indexing="ij")
        extra_u.append(gu.ravel())
        extra_v.append(gv.ravel())
    if extra_u:
        us = np.concatenate([us] + extra_u)
        vs = np.concatenate([vs] + extra_v)
    return from_edges(n_u, n_v, us, vs)


def planted_blocks(seed: int, n_u: int, n_v: int, n_planted: int, k: int):
    """The vertex sets (U part, V part) of the blocks ``er_planted`` plants."""
    sp = stream_state(seed, "PLANT")
    out = []
    for b in range(n_planted):
        base = 2 * b
        lu = np.argsort(splitmix64(sp, base * max(n_u, n_v), n_u), kind="stable")[:k]
        lv = np.argsort(splitmix64(sp, (base + 1) * max(n_u, n_v), n_v), kind="stable")[:k]
        out.append((lu, lv))
    return out


def tiny_random(seed: int, n_u: int, n_v: int, density: float) -> BipartiteGraph:
    """Each of the n_u*n_v pairs present independently with probability ``density``."""
    r = uniform(stream_state(seed, "TINY"), 0, n_u * n_v).reshape(n_u, n_v)
    us, vs = np.nonzero(r < density)
    return from_edges(n_u, n_v, us, vs)


def complete(m: int, n: int) -> BipartiteGraph:
    us, vs = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return from_edges(m, n, us.ravel(), vs.ravel())


def disjoint_union(*gs: BipartiteGraph) -> BipartiteGraph:
    us_all, vs_all = [], []
    ou = ov = 0
    for g in gs:
        us, vs = g.edges()
        us_all.append(us + ou)
        vs_all.append(vs + ov)
        ou += g.n_u
        ov += g.n_v
    return from_edges(ou, ov, np.concatenate(us_all) if us_all else [],
                      np.concatenate(vs_all) if vs_all else [])


def permute(g: BipartiteGraph, seed: int) -> BipartiteGraph:
    """Relabel both sides by seeded random permutations."""
    pu = _random_perm(stream_state(seed, "RELABEL_U"), g.n_u)
    pv = _random_perm(stream_state(seed, "RELABEL_V"), g.n_v)
    us, vs = g.edges()
    return from_edges(g.n_u, g.n_v, pu[us], pv[vs])


def swap_sides(g: BipartiteGraph) -> BipartiteGraph:
    return BipartiteGraph(g.n_v, g.n_u, g.off_v.copy(), g.adj_v.copy(),
                          g.off_u.copy(), g.adj_u.copy())


def add_edges(g: BipartiteGraph, us, vs) -> BipartiteGraph:
    u0, v0 = g.edges()
    return from_edges(g.n_u, g.n_v, np.concatenate([u0, np.asarray(us, np.int64)]),
                      np.concatenate([v0, np.asarray(vs, np.int64)]))


# ---------------------------------------------------------------------------
# The workloads (Table 2 stand-ins; the paper's KONECT graphs are not used).
def workload_small() -> BipartiteGraph:
    """Chung-Lu seed 1: |U|=2000, |V|=3000, |E|=20000, exponent 2.1 both sides."""
    return chung_lu(1, 2000, 3000, 20000, 2.1, 2.1)


def workload_powerlaw_2m() -> BipartiteGraph:
    """Chung-Lu seed 2: |U|=200k, |V|=100k, |E|=2M, exponents 2.0 (U) / 2.3 (V)."""
    return chung_lu(2, 200_000, 100_000, 2_000_000, 2.0, 2.3)


def workload_dense_core() -> BipartiteGraph:
    """ER seed 3: 50k x 50k, 5M uniform edges, plus 20 planted K_{40,40}."""
    return er_planted(3, 50_000, 50_000, 5_000_000, 20, 40)


def batch_job(seed: int) -> tuple[BipartiteGraph, int, int]:
    """One job of the 256-graph batch: |E| = 10^U[3,6], |U|:|V| ratio U[0.25,4],
    one exponent U[1.9,2.6] for both sides, (p, q) uniform in {2..6}^2;
    |U|+|V| = ceil(|E|/5) (mean degree 10 over all vertices)."""
    st = stream_state(seed, "JOB")
    r = uniform(st, 0, 5)
    n_edges = int(round(10.0 ** (3.0 + 3.0 * float(r[0]))))
    ratio = 0.25 + 3.75 * float(r[1])
    gamma = 1.9 + 0.7 * float(r[2])
    p = 2 + int(float(r[3]) * 5)
    q = 2 + int(float(r[4]) * 5)
    n_tot = -(-n_edges // 5)
    n_u = max(2, int(round(n_tot * ratio / (1.0 + ratio))))
    n_v = max(2, n_tot - n_u)
    n_edges = min(n_edges, n_u * n_v // 2)
    return chung_lu(seed, n_u, n_v, n_edges, gamma, gamma), p, q


def serving_graph(i: int, scale: float = 1.0) -> BipartiteGraph:
    """Graph i (0..7) of the serving set.  0: Chung-Lu seed 500, |U|=10M, |V|=5M,
    |E|=100M, exponent 2.1; 1..7: seeds 501..507, |E| log-uniform in [1e5, 1e7],
    |U|+|V| = ceil(|E|/5) split by a ratio U[0.25, 4], exponent 2.1.  ``scale``
    multiplies every size (1.0 = the stated workload)."""
    if i == 0:
        return chung_lu(500, int(10_000_000 * scale), int(5_000_000 * scale), int(100_000_000 * scale), 2.1, 2.1)
    seed = 500 + i
    r = uniform(stream_state(seed, "SERVE"), 0, 2)
    n_edges = int(round(10.0 ** (5.0 + 2.0 * float(r[0]))) * scale)
    ratio = 0.25 + 3.75 * float(r[1])
    n_tot = -(-n_edges // 5)
    n_u = max(2, int(round(n_tot * ratio / (1.0 + ratio))))
    n_v = max(2, n_tot - n_u)
    return chung_lu(seed, n_u, n_v, min(n_edges, n_u * n_v // 2), 2.1, 2.1)


def serving_queries(n: int, seed: int = 600) -> list[tuple[int, int, int]]:
    """n queries (graph index 0..7, p, q) with p, q uniform in {2..8}."""
    r = uniform(stream_state(seed, "QUERIES"), 0, 3 * n).reshape(n, 3)
    return [(int(a * 8), 2 + int(b * 7), 2 + int(c * 7)) for a, b, c in r]
