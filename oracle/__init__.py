"""Oracle for exact (p,q)-biclique counting -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It wraps the plain C enumerator in ``gbc_oracle.c``
(Sec. III-A Basic model, Def. 2 priority, Alg. 1 pruning) and adds two pure
Python references for tiny inputs:

  * ``brute_force``    Def. 1 taken literally: every p-subset L of U and every
                       q-subset R of V, counted when L x R is inside E;
  * ``by_definition``  sum over p-subsets L of C(|common neighbourhood|, q).

It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_ERR_ARG, ORC_OVERFLOW, ORC_NOMEM = 0, 1, 2, 3
MAXK = 16


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("roots_expanded", ctypes.c_int64),
        ("evals", ctypes.c_int64 * (MAXK + 1)),
        ("passed", ctypes.c_int64 * (MAXK + 1)),
        ("words_r", ctypes.c_int64),
        ("words_l", ctypes.c_int64),
        ("cand_total", ctypes.c_int64),
        ("words_lvl2", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {
            "roots_expanded": int(self.roots_expanded),
            "evals": [int(x) for x in self.evals],
            "passed": [int(x) for x in self.passed],
            "words_r": int(self.words_r),
            "words_l": int(self.words_l),
            "cand_total": int(self.cand_total),
            "words_lvl2": int(self.words_lvl2),
        }


class OracleOverflow(ArithmeticError):
    """The count (or one binomial term) exceeds 2^128 - 1."""


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no vector flags)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.orc_count.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int32, ctypes.c_int32, u64p, u64p,
                                  ctypes.POINTER(OracleStats)]
        lib.orc_count.restype = ctypes.c_int
        lib.orc_binomial.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
        lib.orc_binomial.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def count(g, p: int, q: int, anchor: str = "U", roots: tuple[int, int] | None = None,
          per_root: bool = False, stats: bool = False):
    """Exact (p,q)-biclique count of ``g`` (a ``bipgen.BipartiteGraph``).

    anchor "U": L on U (size p), R on V (size q).  anchor "V": the search runs
    from V; the result is still the (p,q) count of g (|L|=p on U, |R|=q on V).
    roots: half-open range of anchor-side vertex ids to use as roots (default
    all); the result is then the sum over those roots of the per-root counts
    (bicliques whose lowest-ranked anchor-side vertex is the root).
    Returns an int, or (int, per_root_list, stats_dict) per the flags.
    """
    lib = _load()
    if anchor == "U":
        a_flag, pp, qq, n_a = 0, p, q, g.n_u
    elif anchor == "V":
        a_flag, pp, qq, n_a = 1, q, p, g.n_v
    else:
        raise ValueError("anchor must be 'U' or 'V'")
    r0, r1 = (0, n_a) if roots is None else roots
    r0, r1 = max(0, r0), min(n_a, r1)
    offu, pou = _i32(g.off_u)
    adju, pau = _i32(g.adj_u if g.n_edges else np.zeros(1, np.int32))
    offv, pov = _i32(g.off_v)
    adjv, pav = _i32(g.adj_v if g.n_edges else np.zeros(1, np.int32))
    tot = (ctypes.c_uint64 * 2)()
    pr = (ctypes.c_uint64 * (2 * max(1, r1 - r0)))() if per_root else None
    st = OracleStats()
    rc = lib.orc_count(g.n_u, g.n_v, pou, pau, pov, pav, pp, qq, a_flag, r0, r1,
                       ctypes.cast(pr, ctypes.POINTER(ctypes.c_uint64)) if pr is not None else None,
                       ctypes.cast(tot, ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(st))
    if rc == ORC_ERR_ARG:
        raise ValueError(f"oracle: bad arguments p={p} q={q}")
    if rc == ORC_NOMEM:
        raise MemoryError("oracle: out of host memory")
    if rc == ORC_OVERFLOW:
        raise OracleOverflow(f"(p,q)=({p},{q}) count exceeds 2^128-1")
    value = int(tot[0]) | (int(tot[1]) << 64)
    if not per_root and not stats:
        return value
    out = [value]
    if per_root:
        out.append([int(pr[2 * i]) | (int(pr[2 * i + 1]) << 64) for i in range(r1 - r0)])
    if stats:
        out.append(st.as_dict())
    return tuple(out)


def binomial(n: int, k: int) -> int | None:
    """C(n, k) from the oracle's checked Pascal table; None if above 2^128-1."""
    out = (ctypes.c_uint64 * 2)()
    rc = _load().orc_binomial(n, k, ctypes.cast(out, ctypes.POINTER(ctypes.c_uint64)))
    if rc < 0:
        raise ValueError("bad binomial arguments")
    return None if rc else int(out[0]) | (int(out[1]) << 64)


# ---------------------------------------------------------------------------
# Pure-Python references for tiny graphs (at most about 12 + 12 vertices).
def _neighbour_masks(g) -> list[int]:
    masks = []
    for u in range(g.n_u):
        m = 0
        for v in g.adj_u[g.off_u[u]:g.off_u[u + 1]]:
            m |= 1 << int(v)
        masks.append(m)
    return masks


def brute_force(g, p: int, q: int) -> int:
    """Def. 1 literally: count pairs (L, R) with |L|=p, |R|=q and L x R in E."""
    masks = _neighbour_masks(g)
    total = 0
    for L in itertools.combinations(range(g.n_u), p):
        for R in itertools.combinations(range(g.n_v), q):
            if all((masks[u] >> v) & 1 for u in L for v in R):
                total += 1
    return total


def by_definition(g, p: int, q: int) -> int:
    """Sum over p-subsets L of U of C(|common neighbourhood of L|, q)."""
    masks = _neighbour_masks(g)
    full = (1 << g.n_v) - 1
    total = 0
    for L in itertools.combinations(range(g.n_u), p):
        m = full
        for u in L:
            m &= masks[u]
        total += math.comb(bin(m).count("1"), q)
    return total
