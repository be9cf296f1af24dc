"""Python binding of the GB300 CL-DIAM library (``include/cldiam.h``).

Argument marshalling only: every step of the method runs in the CUDA library
``libcldiam.so`` built from ``csrc/`` for sm_103a.  There is no CPU fallback;
if the library cannot be loaded, :func:`load` raises.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the library
copies through unified addressing.  Names follow the C ABI:
``build_csr``, ``cluster``, ``quotient_build``, ``estimate``, ``sssp_delta`` ...
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["load", "CldiamError", "Graph", "Clustering", "Quotient", "Result", "Opts", "build_csr", "cluster",
           "quotient_build", "estimate", "apsp_max", "sssp_source", "sssp_delta", "run", "lib_path"]

OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "OVERFLOW", -4: "TIMEOUT", -5: "CUDA", -6: "BUSY",
          -7: "CANCELLED", -8: "DIVERGED", -9: "UNSUPPORTED"}
CSR_LCC = 1
DELTA0_AVG, DELTA0_MIN, DELTA0_EXPLICIT = 0, 1, 2
QUOTIENT_AUTO, QUOTIENT_SORT, QUOTIENT_DENSE = 0, 1, 2
CONTRACT_RESET, CONTRACT_CUMULATIVE = 0, 1


class CldiamError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


class Opts(ctypes.Structure):
    _fields_ = [("delta0_mode", ctypes.c_int32), ("delta0", ctypes.c_uint32), ("contract_mode", ctypes.c_int32),
                ("step_cap", ctypes.c_uint32), ("max_fw_k", ctypes.c_uint32), ("quotient_mode", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


class Tuning(ctypes.Structure):
    """cldiam_tuning: result-invariant launch shapes and cut-overs (0 = library default)."""
    _fields_ = [("pull_ratio", ctypes.c_float), ("relax_ctas_per_sm", ctypes.c_uint32),
                ("dense_quotient_k", ctypes.c_uint32), ("apsp_sources_per_cta", ctypes.c_uint32),
                ("apsp_fw_density", ctypes.c_uint32), ("batch_fw_k", ctypes.c_uint32),
                ("sssp_delta_scale", ctypes.c_float), ("batch_split", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 8)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# cldiam_tune_measure_fn: (const cldiam_tuning*, void* user, double* seconds, uint64_t* result_hash) -> status
TUNE_MEASURE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.POINTER(Tuning), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64))
KNOBS = ["pull_ratio", "relax_ctas_per_sm", "dense_quotient_k", "apsp_sources_per_cta", "apsp_fw_density",
         "batch_fw_k", "sssp_delta_scale", "batch_split"]


class Result(ctypes.Structure):
    _fields_ = [("phi_gc", ctypes.c_uint64), ("radius", ctypes.c_uint64), ("phi_approx", ctypes.c_uint64),
                ("k", ctypes.c_uint32), ("stages", ctypes.c_uint32), ("steps", ctypes.c_uint32),
                ("doublings", ctypes.c_uint32), ("delta_end", ctypes.c_uint32), ("guard_exits", ctypes.c_uint32),
                ("node_updates", ctypes.c_uint64), ("edges_scanned", ctypes.c_uint64),
                ("quotient_edges", ctypes.c_uint64), ("centers_drawn", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_lib_file = None


def lib_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load libcldiam.so (building it with nvcc if needed).  Raises if it cannot be loaded."""
    global _lib, _lib_file
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        PP = ctypes.POINTER(ctypes.c_void_p)
        st = ctypes.c_int32
        sig = {
            "cldiam_status_string": (ctypes.c_char_p, [st]),
            "cldiam_last_error": (ctypes.c_char_p, []),
            "cldiam_version": (st, [P, P]),
            "cldiam_build_csr": (st, [P, P, P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P, PP]),
            "cldiam_graph_info": (st, [P, P, P]),
            "cldiam_graph_copy": (st, [P, P, P, P, P]),
            "cldiam_graph_free": (None, [P]),
            "cldiam_delta0": (st, [P, ctypes.c_int32, P]),
            "cldiam_cluster": (st, [P, ctypes.c_double, ctypes.c_uint64, P, PP]),
            "cldiam_cluster2": (st, [P, ctypes.c_double, ctypes.c_uint64, P, PP]),
            "cldiam_clustering_info": (st, [P, P]),
            "cldiam_clustering_copy": (st, [P, P, P, P]),
            "cldiam_clustering_free": (None, [P]),
            "cldiam_quotient_build": (st, [P, PP]),
            "cldiam_quotient_info": (st, [P, P, P]),
            "cldiam_quotient_copy": (st, [P, P, P, P]),
            "cldiam_quotient_free": (None, [P]),
            "cldiam_estimate": (st, [P, P]),
            "cldiam_apsp_max": (st, [ctypes.c_uint32, P, P, P, P, P]),
            "cldiam_apsp_max_noalloc": (st, [ctypes.c_uint32, P, P, P, P, P]),
            "cldiam_sssp_source": (st, [P, ctypes.c_uint64, P]),
            "cldiam_sssp_delta": (st, [P, ctypes.c_uint32, ctypes.c_uint32, P, P, P, P]),
            "cldiam_run": (st, [P, P, P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                ctypes.c_uint64, P, P, P]),
            "cldiam_arena_create": (st, [ctypes.c_uint64, P, PP]),
            "cldiam_arena_add": (st, [P, P, P, P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P]),
            "cldiam_arena_info": (st, [P, P, P]),
            "cldiam_arena_graph": (st, [P, ctypes.c_uint32, PP]),
            "cldiam_batch_run": (st, [P, P, P, P, ctypes.c_uint32, P, P, P]),
            "cldiam_arena_job_times": (st, [P, ctypes.c_uint32, P, P]),
            "cldiam_arena_free": (None, [P]),
            "cldiam_server_create": (st, [P, P, PP]),
            "cldiam_server_submit": (st, [P, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, P]),
            "cldiam_server_poll": (st, [P, ctypes.c_uint64, P]),
            "cldiam_server_replay": (st, [P, P, P, P, P, ctypes.c_uint32, ctypes.c_int32, P, P, P]),
            "cldiam_server_free": (None, [P]),
            "cldiam_tuning_get": (st, [P]),
            "cldiam_tuning_set": (st, [P]),
            "cldiam_autotune_graph": (st, [P, ctypes.c_double, ctypes.c_uint64, P, ctypes.c_uint32, P]),
            "cldiam_autotune_batch": (st, [P, P, P, P, ctypes.c_uint32, P, ctypes.c_uint32, P]),
            "cldiam_autotune_sssp": (st, [P, ctypes.c_uint32, ctypes.c_uint32, P]),
            "cldiam_autotune_search": (st, [P, ctypes.c_uint32, TUNE_MEASURE_FN, P, P, P]),
            "cldiam_size_class": (ctypes.c_uint32, [ctypes.c_uint64]),
            "cldiam_tuning_effective": (st, [ctypes.c_int32, ctypes.c_uint32, P]),
            "cldiam_tuning_cache_put": (st, [ctypes.c_int32, ctypes.c_uint32, P]),
            "cldiam_tuning_cache_get": (st, [ctypes.c_int32, ctypes.c_uint32, P]),
            "cldiam_tuning_cache_clear": (None, []),
            "cldiam_tuning_cache_save": (st, [ctypes.c_char_p]),
            "cldiam_tuning_cache_load": (st, [ctypes.c_char_p]),
            "cldiam_profile_set_timing": (st, [ctypes.c_uint32]),
            "cldiam_profile_reset": (st, []),
            "cldiam_profile_num_classes": (ctypes.c_uint32, []),
            "cldiam_profile_get": (st, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_char_p), P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib, _lib_file = lib, path
        return lib


def _check(status: int, where: str):
    if status != OK:
        msg = (load().cldiam_last_error() or b"").decode(errors="replace")
        raise CldiamError(status, where, msg)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device); None passes through."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _u32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.uint32)


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


class _Handle:
    _free = None

    def __init__(self, h):
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("handle already freed")
        return self._h

    def free(self):
        if self._h is not None:
            getattr(load(), self._free)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Graph(_Handle):
    _free = "cldiam_graph_free"

    @property
    def n(self) -> int:
        n = ctypes.c_uint32()
        _check(load().cldiam_graph_info(self.handle, ctypes.byref(n), None), "cldiam_graph_info")
        return n.value

    @property
    def nnz(self) -> int:
        z = ctypes.c_uint64()
        _check(load().cldiam_graph_info(self.handle, None, ctypes.byref(z)), "cldiam_graph_info")
        return z.value

    def copy(self):
        """(off uint64[n+1], col uint32[nnz], w uint32[nnz], orig uint32[n]) on the host."""
        n, z = self.n, self.nnz
        off = np.empty(n + 1, np.uint64); col = np.empty(z, np.uint32); w = np.empty(z, np.uint32)
        orig = np.empty(n, np.uint32)
        _check(load().cldiam_graph_copy(self.handle, off.ctypes.data, col.ctypes.data if z else None,
                                        w.ctypes.data if z else None, orig.ctypes.data), "cldiam_graph_copy")
        return off, col, w, orig

    def delta0(self, mode: int = DELTA0_AVG) -> int:
        d = ctypes.c_uint32()
        _check(load().cldiam_delta0(self.handle, mode, ctypes.byref(d)), "cldiam_delta0")
        return d.value


class Clustering(_Handle):
    _free = "cldiam_clustering_free"

    def __init__(self, h, graph):
        super().__init__(h)
        self.graph = graph  # keep the graph alive

    def info(self) -> dict:
        r = Result()
        _check(load().cldiam_clustering_info(self.handle, ctypes.byref(r)), "cldiam_clustering_info")
        return r.as_dict()

    def copy(self):
        """(center, D, cid) as uint32 host arrays."""
        n = self.graph.n
        c = np.empty(n, np.uint32); D = np.empty(n, np.uint32); cid = np.empty(n, np.uint32)
        _check(load().cldiam_clustering_copy(self.handle, c.ctypes.data, D.ctypes.data, cid.ctypes.data),
               "cldiam_clustering_copy")
        return c, D, cid


class Quotient(_Handle):
    _free = "cldiam_quotient_free"

    def __init__(self, h, clustering):
        super().__init__(h)
        self.clustering = clustering

    def info(self):
        k = ctypes.c_uint32(); z = ctypes.c_uint64()
        _check(load().cldiam_quotient_info(self.handle, ctypes.byref(k), ctypes.byref(z)), "cldiam_quotient_info")
        return k.value, z.value

    def copy(self):
        k, z = self.info()
        off = np.empty(k + 1, np.uint64); col = np.empty(z, np.uint32); w = np.empty(z, np.uint32)
        _check(load().cldiam_quotient_copy(self.handle, off.ctypes.data, col.ctypes.data if z else None,
                                           w.ctypes.data if z else None), "cldiam_quotient_copy")
        return off, col, w


class ArenaGraph(Graph):
    """A graph handle viewing one arena graph (keeps the arena alive)."""

    def __init__(self, h, arena):
        super().__init__(h)
        self.arena = arena


class Arena(_Handle):
    """Many graphs in one device CSR arena, run as one persistent batch (cldiam_arena_* / cldiam_batch_run)."""
    _free = "cldiam_arena_free"

    def add(self, src, dst, w, n: int, lcc: bool = True) -> int:
        src, dst, w = _u32(src), _u32(dst), _u32(w)
        gid = ctypes.c_uint32()
        _check(load().cldiam_arena_add(self.handle, _ptr(src), _ptr(dst), _ptr(w), int(src.shape[0]), n,
                                       CSR_LCC if lcc else 0, ctypes.byref(gid)), "cldiam_arena_add")
        return gid.value

    def info(self):
        g = ctypes.c_uint32(); b = ctypes.c_uint64()
        _check(load().cldiam_arena_info(self.handle, ctypes.byref(g), ctypes.byref(b)), "cldiam_arena_info")
        return g.value, b.value

    def graph(self, gid: int) -> "ArenaGraph":
        h = ctypes.c_void_p()
        _check(load().cldiam_arena_graph(self.handle, gid, ctypes.byref(h)), "cldiam_arena_graph")
        return ArenaGraph(h.value, self)

    def run(self, ids, taus, seeds, delta0_mode=DELTA0_AVG, raise_on_error=True, contract_mode=CONTRACT_RESET,
            step_cap=0):
        """Batch of jobs; returns (list of result dicts, list of statuses)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        cnt = int(ids.size)
        res = (Result * max(cnt, 1))()
        sts = np.zeros(max(cnt, 1), np.int32)
        o = make_opts(delta0_mode, contract_mode=contract_mode, step_cap=step_cap)
        st = load().cldiam_batch_run(self.handle, ids.ctypes.data, taus.ctypes.data, seeds.ctypes.data, cnt,
                                     ctypes.byref(o), ctypes.cast(res, ctypes.c_void_p), sts.ctypes.data)
        if raise_on_error:
            _check(st, "cldiam_batch_run")
        return [res[i].as_dict() for i in range(cnt)], [int(x) for x in sts[:cnt]]

    def job_times(self, count: int):
        """cldiam_arena_job_times: (start, end) seconds of each job of the last batch, in job order."""
        a = np.zeros(count, np.float64); b = np.zeros(count, np.float64)
        _check(load().cldiam_arena_job_times(self.handle, count, a.ctypes.data, b.ctypes.data),
               "cldiam_arena_job_times")
        return a, b

    def autotune(self, ids, taus, seeds, reps: int = 3) -> dict:
        """cldiam_autotune_batch: tune the many-graph knobs on these jobs; cached for the batch's size class."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        t = Tuning()
        _check(load().cldiam_autotune_batch(self.handle, ids.ctypes.data, taus.ctypes.data, seeds.ctypes.data,
                                            int(ids.size), None, reps, ctypes.byref(t)), "cldiam_autotune_batch")
        return t.as_dict()


class ServerOpts(ctypes.Structure):
    _fields_ = [("ctas", ctypes.c_uint32), ("capacity", ctypes.c_uint32), ("big_nodes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64), ("idle_seconds", ctypes.c_double)]


class Server(_Handle):
    """Continuous-batching query server over an arena (cldiam_server_*)."""
    _free = "cldiam_server_free"

    def __init__(self, h, arena):
        super().__init__(h)
        self.arena = arena

    def submit(self, graph_id: int, tau: float, seed: int) -> int:
        t = ctypes.c_uint64()
        _check(load().cldiam_server_submit(self.handle, graph_id, float(tau), seed, ctypes.byref(t)),
               "cldiam_server_submit")
        return t.value

    def poll(self, ticket: int):
        """Result dict when finished, None while busy."""
        r = Result()
        st = load().cldiam_server_poll(self.handle, ticket, ctypes.byref(r))
        if st == -6:
            return None
        _check(st, "cldiam_server_poll")
        return r.as_dict()

    def replay(self, ids, taus, seeds, arrivals, plain=False):
        """Native trace replay; returns (results, latencies in s, elapsed s)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        arr = np.ascontiguousarray(arrivals, dtype=np.float64)
        cnt = int(ids.size)
        res = (Result * max(cnt, 1))()
        lat = np.zeros(max(cnt, 1), np.float64)
        el = ctypes.c_double()
        _check(load().cldiam_server_replay(self.handle, ids.ctypes.data, taus.ctypes.data, seeds.ctypes.data,
                                           arr.ctypes.data, cnt, 1 if plain else 0, ctypes.cast(res, ctypes.c_void_p),
                                           lat.ctypes.data, ctypes.byref(el)), "cldiam_server_replay")
        return [res[i].as_dict() for i in range(cnt)], lat[:cnt], el.value


def server_create(arena: "Arena", ctas=0, capacity=0, big_nodes=0, hbm_budget_bytes=0, idle_seconds=0.0) -> Server:
    o = ServerOpts(ctas, capacity, big_nodes, 0, hbm_budget_bytes, idle_seconds)
    h = ctypes.c_void_p()
    _check(load().cldiam_server_create(arena.handle, ctypes.byref(o), ctypes.byref(h)), "cldiam_server_create")
    return Server(h.value, arena)


def arena_create(hbm_budget_bytes: int = 0, stream=None) -> Arena:
    h = ctypes.c_void_p()
    _check(load().cldiam_arena_create(hbm_budget_bytes, _stream_ptr(stream), ctypes.byref(h)), "cldiam_arena_create")
    return Arena(h.value)


def build_csr(src, dst, w, n: int, lcc: bool = True, stream=None) -> Graph:
    """cldiam_build_csr: device CSR of an undirected weighted graph (host or device edge arrays)."""
    lib = load()
    src, dst, w = _u32(src), _u32(dst), _u32(w)
    m = int(src.shape[0])
    h = ctypes.c_void_p()
    st = lib.cldiam_build_csr(_ptr(src), _ptr(dst), _ptr(w), m, n, CSR_LCC if lcc else 0, _stream_ptr(stream),
                              ctypes.byref(h))
    _check(st, "cldiam_build_csr")
    return Graph(h.value)


def make_opts(delta0_mode=DELTA0_AVG, delta0=0, max_fw_k=0, quotient_mode=QUOTIENT_AUTO,
              contract_mode=CONTRACT_RESET, step_cap=0) -> Opts:
    o = Opts()
    o.delta0_mode = delta0_mode
    o.delta0 = delta0
    o.max_fw_k = max_fw_k
    o.quotient_mode = quotient_mode
    o.contract_mode = contract_mode
    o.step_cap = step_cap
    return o


def cluster(g: Graph, tau: float, seed: int, delta0_mode=DELTA0_AVG, delta0=0, max_fw_k=0,
            quotient_mode=QUOTIENT_AUTO, contract_mode=CONTRACT_RESET, step_cap=0) -> Clustering:
    """cldiam_cluster: CLUSTER(G, tau) of Algorithm 1 (options: contract mode, growing-step cap)."""
    o = make_opts(delta0_mode, delta0, max_fw_k, quotient_mode, contract_mode, step_cap)
    h = ctypes.c_void_p()
    _check(load().cldiam_cluster(g.handle, float(tau), seed, ctypes.byref(o), ctypes.byref(h)), "cldiam_cluster")
    return Clustering(h.value, g)


def cluster2(g: Graph, tau: float, seed: int, delta0_mode=DELTA0_AVG, delta0=0, max_fw_k=0,
             quotient_mode=QUOTIENT_AUTO, contract_mode=CONTRACT_RESET, step_cap=0) -> Clustering:
    """cldiam_cluster2: CLUSTER2(G, tau) of Algorithm 2 (CLUSTER for R_CL, then log n iterations of
    PartialGrowth2 / Contract2); the options apply to the first CLUSTER run."""
    o = make_opts(delta0_mode, delta0, max_fw_k, quotient_mode, contract_mode, step_cap)
    h = ctypes.c_void_p()
    _check(load().cldiam_cluster2(g.handle, float(tau), seed, ctypes.byref(o), ctypes.byref(h)), "cldiam_cluster2")
    return Clustering(h.value, g)


def quotient_build(c: Clustering) -> Quotient:
    """cldiam_quotient_build: the weighted quotient graph of Section 4."""
    h = ctypes.c_void_p()
    _check(load().cldiam_quotient_build(c.handle, ctypes.byref(h)), "cldiam_quotient_build")
    return Quotient(h.value, c)


def estimate(q: Quotient) -> dict:
    """cldiam_estimate: Phi(G_C), R and Phi_approx = Phi(G_C) + 2R (Section 4)."""
    r = Result()
    _check(load().cldiam_estimate(q.handle, ctypes.byref(r)), "cldiam_estimate")
    return r.as_dict()


def apsp_max(k: int, off, col, w, stream=None) -> int:
    """cldiam_apsp_max: largest finite distance of a k-node symmetric CSR graph."""
    phi = ctypes.c_uint64()
    off = off if hasattr(off, "data_ptr") else np.ascontiguousarray(off, dtype=np.uint64)
    _check(load().cldiam_apsp_max(k, _ptr(off), _ptr(_u32(col)), _ptr(_u32(w)), _stream_ptr(stream),
                                  ctypes.byref(phi)), "cldiam_apsp_max")
    return phi.value


def apsp_max_noalloc(k: int, off, col, w, stream=None) -> int:
    """cldiam_apsp_max_noalloc: same as apsp_max, device tensors only, no device allocation."""
    phi = ctypes.c_uint64()
    _check(load().cldiam_apsp_max_noalloc(k, _ptr(off), _ptr(col), _ptr(w), _stream_ptr(stream), ctypes.byref(phi)),
           "cldiam_apsp_max_noalloc")
    return phi.value


def sssp_source(g: Graph, seed: int) -> int:
    s = ctypes.c_uint32()
    _check(load().cldiam_sssp_source(g.handle, seed, ctypes.byref(s)), "cldiam_sssp_source")
    return s.value


def sssp_delta(g: Graph, source: int, delta: int = 0, want_dist: bool = True, with_scanned: bool = False):
    """cldiam_sssp_delta: (dist or None, ecc, rounds) of Delta-stepping from `source`; with_scanned adds the
    adjacency entries the phases read as a fourth element."""
    dist = np.empty(g.n, np.uint32) if want_dist else None
    ecc = ctypes.c_uint64(); rounds = ctypes.c_uint64(); scanned = ctypes.c_uint64()
    _check(load().cldiam_sssp_delta(g.handle, source, delta, _ptr(dist), ctypes.byref(ecc), ctypes.byref(rounds),
                                    ctypes.byref(scanned)), "cldiam_sssp_delta")
    if with_scanned:
        return dist, ecc.value, rounds.value, scanned.value
    return dist, ecc.value, rounds.value


def tuning_get() -> dict:
    """cldiam_tuning_get: the process-wide knobs in effect (defaults filled in)."""
    t = Tuning()
    _check(load().cldiam_tuning_get(ctypes.byref(t)), "cldiam_tuning_get")
    return t.as_dict()


def tuning_set(**knobs) -> None:
    """cldiam_tuning_set: replace the process-wide knobs (unnamed ones = library default);
    no arguments restores every default."""
    if not knobs:
        _check(load().cldiam_tuning_set(None), "cldiam_tuning_set")
        return
    t = _tuning_of(knobs)
    _check(load().cldiam_tuning_set(ctypes.byref(t)), "cldiam_tuning_set")


def _tuning_of(knobs: dict) -> Tuning:
    t = Tuning()
    for k, v in knobs.items():
        if k not in KNOBS:
            raise KeyError(k)
        setattr(t, k, v if k in ("pull_ratio", "sssp_delta_scale") else int(v))
    return t


def autotune_graph(g: "Graph", tau: float, seed: int, reps: int = 3, **opts) -> dict:
    """cldiam_autotune_graph: tune the one-graph knobs on this graph's CLUSTER + quotient + estimate;
    the choice is cached for the graph's size class and returned."""
    o = make_opts(**opts) if opts else None
    t = Tuning()
    _check(load().cldiam_autotune_graph(g.handle, float(tau), seed, ctypes.byref(o) if o else None, reps,
                                        ctypes.byref(t)), "cldiam_autotune_graph")
    return t.as_dict()


def autotune_sssp(g: "Graph", source: int, reps: int = 3) -> dict:
    """cldiam_autotune_sssp: tune Delta-stepping's bucket width on this graph and source."""
    t = Tuning()
    _check(load().cldiam_autotune_sssp(g.handle, source, reps, ctypes.byref(t)), "cldiam_autotune_sssp")
    return t.as_dict()


def autotune_search(measure, knobs, start: dict | None = None):
    """cldiam_autotune_search with a Python measure(knobs: dict) -> (seconds, result_hash); returns
    (best knobs, best seconds)."""
    mask = 0
    for k in knobs:
        mask |= 1 << KNOBS.index(k)
    err = []

    def cb(tp, user, sec, h):
        try:
            s_, h_ = measure(tp.contents.as_dict())
        except Exception as ex:  # a failing candidate is skipped by the search
            err.append(ex)
            return -1
        sec[0] = float(s_)
        h[0] = int(h_) & 0xFFFFFFFFFFFFFFFF
        return 0

    fn = TUNE_MEASURE_FN(cb)
    best = Tuning()
    bs = ctypes.c_double()
    st0 = _tuning_of(start or {})
    _check(load().cldiam_autotune_search(ctypes.byref(st0), mask, fn, None, ctypes.byref(best), ctypes.byref(bs)),
           "cldiam_autotune_search")
    return best.as_dict(), bs.value


def size_class(entries: int) -> int:
    return int(load().cldiam_size_class(entries))


def tuning_effective(device: int, size_class_: int) -> dict:
    t = Tuning()
    _check(load().cldiam_tuning_effective(device, size_class_, ctypes.byref(t)), "cldiam_tuning_effective")
    return t.as_dict()


def tuning_cache_put(device: int, size_class_: int, **knobs) -> None:
    t = _tuning_of(knobs)
    _check(load().cldiam_tuning_cache_put(device, size_class_, ctypes.byref(t)), "cldiam_tuning_cache_put")


def tuning_cache_get(device: int, size_class_: int) -> dict:
    t = Tuning()
    _check(load().cldiam_tuning_cache_get(device, size_class_, ctypes.byref(t)), "cldiam_tuning_cache_get")
    return t.as_dict()


def tuning_cache_clear() -> None:
    load().cldiam_tuning_cache_clear()


def tuning_cache_save(path: str) -> None:
    _check(load().cldiam_tuning_cache_save(path.encode()), "cldiam_tuning_cache_save")


def tuning_cache_load(path: str) -> None:
    _check(load().cldiam_tuning_cache_load(path.encode()), "cldiam_tuning_cache_load")


KERNEL_CLASSES = ["relax", "snapshot", "rebuild", "select", "finalize", "growable", "radix_hist", "radix_scatter",
                  "scan", "csr", "components", "quotient", "floyd_warshall", "delta_stepping", "reduce", "misc",
                  "relax_pull"]


def profile_set_timing(classes) -> None:
    """Time every launch of the named kernel classes with CUDA events (empty = off)."""
    mask = 0
    for c in classes:
        mask |= 1 << KERNEL_CLASSES.index(c)
    _check(load().cldiam_profile_set_timing(mask), "cldiam_profile_set_timing")


def profile_reset() -> None:
    _check(load().cldiam_profile_reset(), "cldiam_profile_reset")


def profile_get() -> dict:
    """{class: {"launches", "ms", "bytes"}} since the last reset."""
    lib = load()
    out = {}
    for i in range(lib.cldiam_profile_num_classes()):
        name = ctypes.c_char_p(); L = ctypes.c_uint64(); ms = ctypes.c_double(); b = ctypes.c_double()
        _check(lib.cldiam_profile_get(i, ctypes.byref(name), ctypes.byref(L), ctypes.byref(ms), ctypes.byref(b)),
               "cldiam_profile_get")
        out[name.value.decode()] = {"launches": L.value, "ms": ms.value, "bytes": b.value}
    return out


def run(src, dst, w, n: int, tau: float, seed: int, lcc: bool = True, delta0_mode=DELTA0_AVG, stream=None) -> dict:
    """cldiam_run: the whole method from an edge list."""
    src, dst, w = _u32(src), _u32(dst), _u32(w)
    o = make_opts(delta0_mode)
    r = Result()
    _check(load().cldiam_run(_ptr(src), _ptr(dst), _ptr(w), int(src.shape[0]), n, CSR_LCC if lcc else 0,
                             float(tau), seed, ctypes.byref(o), _stream_ptr(stream), ctypes.byref(r)), "cldiam_run")
    return r.as_dict()
