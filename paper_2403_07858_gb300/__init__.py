"""GB300 (sm_103a) exact (p,q)-biclique counting: Python binding of libgbc.so.

The binding only marshals arguments: every step of a count runs in the CUDA
kernels behind the C ABI of include/gbc.h.  There is no CPU fallback; if the
library has not been built, or no GPU is present, the calls raise.

    import paper_2403_07858_gb300 as gbc
    ctx = gbc.Context()                       # device 0
    g = ctx.load_graph(n_u, n_v, off_u, adj_u, off_v, adj_v)   # host arrays
    n = g.count(4, 4)                         # Python int, exact
    n, info = g.count_ex(4, 4, anchor="V", stats=True)

Arrays may be numpy arrays (host) or CUDA torch tensors (``load_graph`` copies
either way; torch is only used for device memory and streams).
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbc.so")
MAX_PQ = 16

GBC_OK, GBC_ERR_ARG, GBC_ERR_INVALID_GRAPH, GBC_ERR_OOM, GBC_ERR_OVERFLOW = 0, 1, 2, 3, 4
GBC_ERR_TIMEOUT, GBC_ERR_CUDA, GBC_PENDING, GBC_ERR_REJECTED = 5, 6, 7, 8
ANCHORS = {"auto": 0, "U": 1, "V": 2}
_ANCHOR_NAMES = {1: "U", 2: "V"}


class GbcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class InvalidGraph(GbcError):
    pass


class CountOverflow(GbcError, ArithmeticError):
    pass


class CountTimeout(GbcError, TimeoutError):
    pass


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self) -> int:
        return int(self.lo) | (int(self.hi) << 64)


class CountOptions(ctypes.Structure):
    _fields_ = [("anchor", ctypes.c_int32), ("collect_stats", ctypes.c_int32),
                ("enum_warps", ctypes.c_int32), ("time_limit_ms", ctypes.c_int32),
                ("root_begin", ctypes.c_int32), ("root_end", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("position_order", ctypes.c_int32),
                ("collapse_skip", ctypes.c_int32)]


class CountInfo(ctypes.Structure):
    _fields_ = [("anchor_used", ctypes.c_int32), ("set_size", ctypes.c_int32),
                ("roots", ctypes.c_int64), ("candidates", ctypes.c_int64), ("units", ctypes.c_int64),
                ("evals", ctypes.c_int64 * (MAX_PQ + 1)), ("passed", ctypes.c_int64 * (MAX_PQ + 1)),
                ("words_r", ctypes.c_int64), ("words_l", ctypes.c_int64),
                ("scratch_bytes", ctypes.c_int64),
                ("ms_candidates", ctypes.c_float), ("ms_pairs", ctypes.c_float),
                ("ms_enumerate", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("enum_words", ctypes.c_int64), ("launches", ctypes.c_int32), ("pieces", ctypes.c_int32),
                ("words_enum", ctypes.c_int64), ("enum_span_ms", ctypes.c_float),
                ("enum_longest_unit_ms", ctypes.c_float), ("enum_exit_spread_ms", ctypes.c_float),
                ("reserved_t", ctypes.c_int32), ("words_exec", ctypes.c_int64), ("collapsed", ctypes.c_int64),
                ("enum_phase_cycles", ctypes.c_int64 * 10)]

    def as_dict(self) -> dict:
        return {
            "anchor": _ANCHOR_NAMES.get(self.anchor_used, "?"),
            "set_size": int(self.set_size),
            "roots": int(self.roots),
            "candidates": int(self.candidates),
            "units": int(self.units),
            "evals": [int(x) for x in self.evals],
            "passed": [int(x) for x in self.passed],
            "words_r": int(self.words_r),
            "words_l": int(self.words_l),
            "scratch_bytes": int(self.scratch_bytes),
            "ms_candidates": float(self.ms_candidates),
            "ms_pairs": float(self.ms_pairs),
            "ms_enumerate": float(self.ms_enumerate),
            "ms_total": float(self.ms_total),
            "enum_words": int(self.enum_words),
            "words_enum": int(self.words_enum),
            "launches": int(self.launches),
            "pieces": int(self.pieces),
            "enum_span_ms": float(self.enum_span_ms),
            "enum_longest_unit_ms": float(self.enum_longest_unit_ms),
            "enum_exit_spread_ms": float(self.enum_exit_spread_ms),
            "words_exec": int(self.words_exec),
            "collapsed": int(self.collapsed),
            "enum_phase_cycles": [int(x) for x in self.enum_phase_cycles],
        }


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("rejected", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("peak_in_flight_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("peak_running_batches", ctypes.c_int32),
                ("reserved_i", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved_i"}


_lib = None
_lib_lock = threading.Lock()

# name -> (restype, argtypes); the full C ABI of include/gbc.h
_vp, _i32, _i64, _i32p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "gbc_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "gbc_ctx_set_stream": (ctypes.c_int, [_vp, _vp]),
    "gbc_ctx_destroy": (None, [_vp]),
    "gbc_load_graph": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "gbc_load_graph_device": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "gbc_load_graph_ex": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    "gbc_free_graph": (None, [_vp]),
    "gbc_graph_info": (ctypes.c_int, [_vp, _i32p, _i32p, ctypes.POINTER(_i64), _i32p, _i32p]),
    "gbc_count": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(U128)]),
    "gbc_count_ex": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(CountOptions),
                                    ctypes.POINTER(U128), ctypes.POINTER(CountInfo)]),
    "gbc_count_per_root": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(U128), ctypes.POINTER(U128)]),
    "gbc_count_p2_noalloc": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _vp, ctypes.c_int, _vp,
                                            ctypes.POINTER(U128)]),
    "gbc_count_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(U128),
                                       ctypes.POINTER(ctypes.c_int)]),
    "gbc_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "gbc_tuned_anchor": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "gbc_tuned_warps": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "gbc_serve_start": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gbc_serve_stop": (ctypes.c_int, [_vp]),
    "gbc_serve_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(ServeStats)]),
    "gbc_footprint": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_int)]),
    "gbc_list_begin": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp),
                                      ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "gbc_list_next": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                     ctypes.POINTER(ctypes.c_int)]),
    "gbc_list_end": (None, [_vp]),
    "gbc_submit": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "gbc_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(U128)]),
    "gbc_border_order": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i64)]),
    "gbc_measure_int_peaks": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    "gbc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gbc_last_error": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return LIB_PATH


def load_library(path: str | None = None):
    """Load libgbc.so (built by ``build()``); raises if it is missing."""
    global _lib
    with _lib_lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libgbc.so not built ({p}); run paper_2403_07858_gb300.build()")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def build(force: bool = False) -> str:
    """Compile libgbc.so for sm_103a if it is missing or stale; returns its path."""
    import importlib
    return importlib.import_module(__name__ + ".buildlib").build(force=force)


def _check(status: int, what: str):
    if status == GBC_OK:
        return
    lib = load_library()
    msg = (lib.gbc_last_error() or b"").decode(errors="replace") or what
    if status == GBC_ERR_INVALID_GRAPH:
        raise InvalidGraph(status, msg)
    if status == GBC_ERR_OVERFLOW:
        raise CountOverflow(status, msg)
    if status == GBC_ERR_TIMEOUT:
        raise CountTimeout(status, msg)
    raise GbcError(status, msg)


def _ptr_host(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


class Graph:
    """A graph resident on the device (freed by ``close`` or garbage collection)."""

    def __init__(self, ctx: "Context", handle: int):
        self._ctx = ctx
        self._h = ctypes.c_void_p(handle)
        ctx._graphs.add(self)
        n_u, n_v, mu, mv = _i32(), _i32(), _i32(), _i32()
        n_e = _i64()
        _check(load_library().gbc_graph_info(self._h, ctypes.byref(n_u), ctypes.byref(n_v), ctypes.byref(n_e),
                                             ctypes.byref(mu), ctypes.byref(mv)), "gbc_graph_info")
        self.n_u, self.n_v, self.n_edges = n_u.value, n_v.value, n_e.value
        self.max_deg_u, self.max_deg_v = mu.value, mv.value

    def close(self):
        if self._h:
            load_library().gbc_free_graph(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def count(self, p: int, q: int) -> int:
        out = U128()
        _check(load_library().gbc_count(self._h, p, q, ctypes.byref(out)), "gbc_count")
        return out.value()

    def count_ex(self, p: int, q: int, anchor: str = "auto", stats: bool = False,
                 enum_warps: int = 0, time_limit_ms: int = 0,
                 roots: tuple[int, int] | None = None, kernel: str = "bitmap",
                 position_order: str = "shared", collapse: bool | int = True) -> tuple[int, dict]:
        """roots: count only the search trees rooted in this half-open range of
        anchor vertices (give the anchor explicitly when splitting a count).
        kernel: "bitmap" (the default) or "csr" (the sorted-list ablation).
        position_order: "shared" (most shared position first, the default) or
        "id" (the other side's id order).
        stats: False, True (the full traversal's counters) or "exec" (the
        executed traversal's words and collapsed subtrees).
        collapse: count small-C_R subtrees in closed form: True (the default
        slack), False (enter every node) or the slack s = 1..4 (nodes with
        |C_R| <= q' + s collapse)."""
        opt = CountOptions()
        opt.kernel = {"bitmap": 0, "csr": 1}[kernel]
        opt.position_order = {"shared": 0, "id": 1}[position_order]
        opt.anchor = ANCHORS[anchor]
        opt.collect_stats = 2 if stats == "exec" else (1 if stats else 0)
        opt.collapse_skip = 0 if collapse is True else (-1 if collapse is False else int(collapse))
        opt.enum_warps = enum_warps
        opt.time_limit_ms = time_limit_ms
        if roots is not None:
            opt.root_begin, opt.root_end = int(roots[0]), int(roots[1])
        out, info = U128(), CountInfo()
        _check(load_library().gbc_count_ex(self._h, p, q, ctypes.byref(opt), ctypes.byref(out),
                                           ctypes.byref(info)), "gbc_count_ex")
        return out.value(), info.as_dict()

    def footprint(self, p: int, q: int) -> tuple[int, bool]:
        """Scratch bytes the (p,q) count holds: (bytes, exact); exact once the
        same count ran on this context, else a load-time upper bound."""
        b, e = ctypes.c_size_t(), ctypes.c_int()
        _check(load_library().gbc_footprint(self._h, p, q, ctypes.byref(b), ctypes.byref(e)), "gbc_footprint")
        return int(b.value), bool(e.value)

    def list_records(self, p: int, q: int, buffer=None, anchor: str = "U", min_words: int = 4096,
                     calls: list | None = None):
        """Yield the listed bicliques as (L, C_R) tuples of caller ids, filling the
        int32 CUDA tensor ``buffer`` one gbc_list_next call at a time (None: one
        of max(min_words, the largest root's records) words).  ``calls``, if
        given, receives the (words, records) of every call."""
        lib = load_library()
        h = ctypes.c_void_p()
        tw, tr, mx = _i64(), _i64(), _i64()
        _check(lib.gbc_list_begin(self._h, p, q, ANCHORS[anchor], ctypes.byref(h), ctypes.byref(tw),
                                  ctypes.byref(tr), ctypes.byref(mx)), "gbc_list_begin")
        k = p if anchor == "U" else q
        try:
            if buffer is None:
                import torch
                buffer = torch.zeros(max(min_words, mx.value, 1), dtype=torch.int32, device="cuda")
            done = ctypes.c_int(0)
            while not done.value:
                w, r = _i64(), _i64()
                _check(lib.gbc_list_next(h, ctypes.c_void_p(buffer.data_ptr()), buffer.numel(), ctypes.byref(w),
                                         ctypes.byref(r), ctypes.byref(done)), "gbc_list_next")
                if calls is not None:
                    calls.append((w.value, r.value))
                words = buffer[:w.value].cpu().tolist()
                at = 0
                for _ in range(r.value):
                    m = words[at + k]
                    yield tuple(words[at:at + k]), tuple(words[at + k + 1:at + k + 1 + m])
                    at += k + 1 + m
        finally:
            lib.gbc_list_end(h)

    def tuned_anchor(self, p: int, q: int) -> str | None:
        return _ANCHOR_NAMES.get(load_library().gbc_tuned_anchor(self._h, p, q))

    def tuned_warps(self, p: int, q: int) -> int:
        """Enumeration warps the autotuner kept for (p, q); 0 = the default."""
        return int(load_library().gbc_tuned_warps(self._h, p, q))

    def count_per_root(self, p: int, q: int, anchor: str) -> tuple[int, list[int]]:
        n_a = self.n_u if anchor == "U" else self.n_v
        per = (U128 * max(1, n_a))()
        tot = U128()
        _check(load_library().gbc_count_per_root(self._h, p, q, ANCHORS[anchor], per, ctypes.byref(tot)),
               "gbc_count_per_root")
        return tot.value(), [per[i].value() for i in range(n_a)]


class Context:
    """One CUDA device, its stream and a device-memory budget for search scratch."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.gbc_ctx_create(device, mem_budget_bytes, ctypes.byref(h)), "gbc_ctx_create")
        self._h = h
        self.device = device
        self._graphs = weakref.WeakSet()  # graphs still loaded, freed before the context

    def set_stream(self, stream) -> None:
        """Run later calls on ``stream`` (a torch.cuda.Stream, a raw handle, or None)."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(load_library().gbc_ctx_set_stream(self._h, ctypes.c_void_p(handle or 0)), "gbc_ctx_set_stream")

    def close(self):
        """Stop serving, free the graphs still loaded on this context, then the context."""
        if self._h:
            lib = load_library()
            lib.gbc_serve_stop(self._h)
            for g in list(self._graphs):
                g.close()
            lib.gbc_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def load_graph(self, n_u: int, n_v: int, off_u, adj_u, off_v, adj_v, keep_ids: bool = False) -> Graph:
        """keep_ids: keep the caller's vertex ids on the device (host arrays only)
        instead of renumbering each side by degree; the counts are the same."""
        lib = load_library()
        h = ctypes.c_void_p()
        arrays = (off_u, adj_u, off_v, adj_v)
        if keep_ids:
            keep = [_ptr_host(x) for x in arrays]
            ptrs = [ctypes.c_void_p(p) for _, p in keep]
            _check(lib.gbc_load_graph_ex(self._h, n_u, n_v, *ptrs, 1, ctypes.byref(h)), "gbc_load_graph_ex")
            return Graph(self, h.value)
        if all(_is_cuda_tensor(x) for x in arrays):
            ptrs = [ctypes.c_void_p(x.data_ptr()) for x in arrays]
            _check(lib.gbc_load_graph_device(self._h, n_u, n_v, *ptrs, ctypes.byref(h)), "gbc_load_graph_device")
        else:
            keep = [_ptr_host(x) for x in arrays]
            ptrs = [ctypes.c_void_p(p) for _, p in keep]
            _check(lib.gbc_load_graph(self._h, n_u, n_v, *ptrs, ctypes.byref(h)), "gbc_load_graph")
        return Graph(self, h.value)

    def count_batch(self, graphs, ps, qs):
        """Counts of (graphs[i], ps[i], qs[i]) in one batched pipeline; returns a list
        whose entries are ints, or GbcError instances for jobs that failed."""
        n = len(graphs)
        hs = (ctypes.c_void_p * max(1, n))(*[g._h.value for g in graphs])
        pa = (ctypes.c_int * max(1, n))(*ps)
        qa = (ctypes.c_int * max(1, n))(*qs)
        out = (U128 * max(1, n))()
        st = (ctypes.c_int * max(1, n))()
        _check(load_library().gbc_count_batch(self._h, n, hs, pa, qa, out, st), "gbc_count_batch")
        res = []
        for i in range(n):
            if st[i] == GBC_OK:
                res.append(out[i].value())
            else:
                res.append(GbcError(st[i], load_library().gbc_status_string(st[i]).decode()))
        return res

    def autotune(self, graphs, ps, qs, time_limit_ms: int = 60_000) -> None:
        """Time both anchors for each (graph, p, q) and keep the faster for later counts."""
        n = len(graphs)
        hs = (ctypes.c_void_p * max(1, n))(*[g._h.value for g in graphs])
        pa = (ctypes.c_int * max(1, n))(*ps)
        qa = (ctypes.c_int * max(1, n))(*qs)
        _check(load_library().gbc_autotune(self._h, n, hs, pa, qa, time_limit_ms), "gbc_autotune")

    # ---- serving
    def serve_start(self, workers: int = 0, max_batch: int = 0, max_queue: int = 0, time_limit_ms: int = 0):
        _check(load_library().gbc_serve_start(self._h, workers, max_batch, max_queue, time_limit_ms),
               "gbc_serve_start")

    def serve_stop(self):
        _check(load_library().gbc_serve_stop(self._h), "gbc_serve_stop")

    def serve_stats(self) -> dict:
        st = ServeStats()
        _check(load_library().gbc_serve_stats_get(self._h, ctypes.byref(st)), "gbc_serve_stats_get")
        return st.as_dict()

    def submit(self, graph: "Graph", p: int, q: int) -> int:
        t = ctypes.c_uint64()
        _check(load_library().gbc_submit(self._h, graph._h, p, q, ctypes.byref(t)), "gbc_submit")
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """The count of a ticket, or None while it is pending (timeout reached)."""
        out = U128()
        s = load_library().gbc_poll(self._h, ticket, timeout_ms, ctypes.byref(out))
        if s == GBC_PENDING:
            return None
        _check(s, "gbc_poll")
        return out.value()

    def load(self, g, keep_ids: bool = False) -> Graph:
        """Load a ``bipgen.BipartiteGraph`` (or anything with the same fields)."""
        return self.load_graph(g.n_u, g.n_v, g.off_u, g.adj_u, g.off_v, g.adj_v, keep_ids=keep_ids)


def count_p2_noalloc(n_u: int, n_v: int, off_u, adj_u, off_v, adj_v, q: int, stream=None) -> int:
    """(2,q)-biclique count from CUDA tensors through the entry point that
    allocates nothing (its scratch is a fixed static device array).  The four
    arrays must be int32 CUDA tensors on the current device."""
    arrays = (off_u, adj_u, off_v, adj_v)
    if not all(_is_cuda_tensor(x) for x in arrays):
        raise TypeError("count_p2_noalloc takes int32 CUDA tensors")
    handle = getattr(stream, "cuda_stream", stream)
    out = U128()
    _check(load_library().gbc_count_p2_noalloc(n_u, n_v, *[ctypes.c_void_p(x.data_ptr()) for x in arrays], q,
                                               ctypes.c_void_p(handle or 0), ctypes.byref(out)),
           "gbc_count_p2_noalloc")
    return out.value()


def border_order(n_a: int, n_o: int, off_a, adj_a, iterations: int = 10_000, max_cand: int = 64):
    """Border (Sec. V-B, Alg. 2) on the A -> O CSR (host arrays): the new id of
    every O vertex, and the 1-blocks before (degree order) and after."""
    off, p_off = _ptr_host(off_a)
    adj, p_adj = _ptr_host(adj_a if len(adj_a) else np.zeros(1, np.int32))
    out = np.zeros(max(1, n_o), dtype=np.int32)
    before, after = _i64(), _i64()
    _check(load_library().gbc_border_order(n_a, n_o, ctypes.c_void_p(p_off), ctypes.c_void_p(p_adj), iterations,
                                           max_cand, ctypes.c_void_p(out.ctypes.data), ctypes.byref(before),
                                           ctypes.byref(after)), "gbc_border_order")
    return out[:n_o], int(before.value), int(after.value)


def measure_int_peaks(device: int = 0) -> dict:
    """Integer-pipe and L2 microbenchmarks on one GPU: words/s of a register-only
    AND + POPC + ADD loop and bytes/s of an L2-resident AND + popcount stream."""
    alu, l2 = ctypes.c_double(), ctypes.c_double()
    _check(load_library().gbc_measure_int_peaks(device, ctypes.byref(alu), ctypes.byref(l2)), "gbc_measure_int_peaks")
    return {"and_popc_words_per_s": alu.value, "l2_bytes_per_s": l2.value}
