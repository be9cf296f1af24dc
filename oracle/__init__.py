"""CPU oracle for CL-DIAM (test infrastructure only).

A plain sequential C restatement of the method (``cldiam_oracle.c``), loaded
with ctypes.  Only the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package; the product library never does, and shares no code with it.

Each wrapper names the passage of the paper it follows (arXiv 1506.03265).
Parity status: see the header of ``cldiam_oracle.c``; CLUSTER's random
trajectory is pinned by invariants and special cases only.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cldiam_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

INF_KEY = 0xFFFFFFFFFFFFFFFF
NONE = 0xFFFFFFFF
UNREACHABLE = np.iinfo(np.uint64).max

DELTA0_AVG = 0
DELTA0_MIN = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single-threaded, no fp contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    tag = hashlib.sha1(open(_SRC, "rb").read()).hexdigest()[:12]
    out = os.path.join(_BUILD, f"libcldiam_oracle_{tag}.so")
    if force or not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, out)
    return out


class Stats(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_uint32), ("steps", ctypes.c_uint32), ("doublings", ctypes.c_uint32),
                ("delta_end", ctypes.c_uint32), ("guard_exits", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("node_updates", ctypes.c_uint64), ("edges_examined", ctypes.c_uint64),
                ("centers_drawn", ctypes.c_uint64)]


TRACE_DTYPE = np.dtype([("kind", np.uint32), ("stage", np.uint32), ("delta", np.uint32), ("pad", np.uint32),
                        ("a", np.uint64), ("b", np.uint64)])
TRACE_STEP, TRACE_DOUBLE, TRACE_FINALIZE, TRACE_GUARD, TRACE_STAGE = 0, 1, 2, 3, 4


def _lib_load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_philox4x32_10.argtypes = [ctypes.c_uint64, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_build_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, P, P, P, ctypes.c_int, P, P, P, P, P]
            lib.orc_build_csr.restype = ctypes.c_int64
            lib.orc_delta0.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_int]
            lib.orc_delta0.restype = ctypes.c_uint32
            lib.orc_growth_steps.argtypes = [ctypes.c_uint32, P, P, P, P, P, P, P, ctypes.c_uint32, ctypes.c_uint32, P]
            lib.orc_growth_steps.restype = None
            lib.orc_cluster.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                        P, P, ctypes.POINTER(Stats), P, ctypes.c_uint64, P]
            lib.orc_cluster.restype = ctypes.c_int
            lib.orc_cluster_opts.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_double, ctypes.c_uint64,
                                             ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32, P, P,
                                             ctypes.POINTER(Stats), P, ctypes.c_uint64, P]
            lib.orc_cluster_opts.restype = ctypes.c_int
            lib.orc_cluster2.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_uint32, P, P, ctypes.POINTER(C2Stats)]
            lib.orc_cluster2.restype = ctypes.c_int
            lib.orc_quotient.argtypes = [ctypes.c_uint32, P, P, P, P, P, P, P, P, P, P]
            lib.orc_quotient.restype = ctypes.c_int64
            lib.orc_dijkstra.argtypes = [ctypes.c_uint32, P, P, P, P, ctypes.c_uint32, P]
            lib.orc_dijkstra.restype = ctypes.c_int
            lib.orc_apsp_max.argtypes = [ctypes.c_uint32, P, P, P, P]
            lib.orc_apsp_max.restype = ctypes.c_int
            lib.orc_sssp_source.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            lib.orc_sssp_source.restype = ctypes.c_uint32
            lib.orc_lower_bound.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_uint32, ctypes.c_uint32, P, P]
            lib.orc_lower_bound.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class CSR:
    """Symmetric CSR of an undirected weighted graph (oracle layout: separate col / wt arrays)."""
    n: int
    off: np.ndarray   # uint64[n+1]
    col: np.ndarray   # uint32[nnz]
    wt: np.ndarray    # uint32[nnz]
    orig: np.ndarray  # uint32[n] original id of each kept node

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2


def philox4x32_10(seed: int, ctr) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al. SC'11), the draw behind Algorithm 1's center selection."""
    c = _c(ctr, np.uint32)
    o = np.empty(4, np.uint32)
    _lib_load().orc_philox4x32_10(seed, _ptr(c), _ptr(o))
    return o


def build_csr(n, src, dst, w, lcc=True) -> CSR:
    """Graph model of Section 2: dedup (min weight), no self-loops, symmetric, optional LCC."""
    lib = _lib_load()
    src = _c(src, np.uint32); dst = _c(dst, np.uint32); w = _c(w, np.uint32)
    m = src.shape[0]
    off = np.empty(n + 1, np.uint64)
    col = np.empty(max(2 * m, 1), np.uint32)
    wt = np.empty(max(2 * m, 1), np.uint32)
    orig = np.empty(n, np.uint32)
    nout = ctypes.c_uint32()
    nnz = lib.orc_build_csr(n, m, _ptr(src), _ptr(dst), _ptr(w), 1 if lcc else 0, ctypes.addressof(nout),
                            _ptr(off), _ptr(col), _ptr(wt), _ptr(orig))
    if nnz < 0:
        raise ValueError(f"orc_build_csr failed: {nnz}")
    k = nout.value
    return CSR(k, off[:k + 1].copy(), col[:nnz].copy(), wt[:nnz].copy(), orig[:k].copy())


def delta0(g: CSR, mode: int = DELTA0_AVG) -> int:
    """Initial Delta: minimum weight (Algorithm 1) or average weight (Section 5)."""
    return int(_lib_load().orc_delta0(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), mode))


def growth_steps(g: CSR, key, frozen, center, delta: int, steps: int, D=None):
    """t synchronous Delta-growing steps (Section 3) at fixed Delta; returns (key, updated-per-step).
    D (optional): bounds of the frozen nodes for the cumulative contract mode."""
    key = _c(key, np.uint64).copy()
    frozen = _c(frozen, np.uint8)
    center = _c(center, np.uint32)
    Dp = _c(D, np.uint64) if D is not None else None
    upd = np.zeros(max(steps, 1), np.uint64)
    _lib_load().orc_growth_steps(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), _ptr(key), _ptr(frozen),
                                 _ptr(center), _ptr(Dp) if Dp is not None else None, delta, steps, _ptr(upd))
    return key, upd[:steps]


@dataclass
class Clustering:
    center: np.ndarray  # uint32[n] center node id of each node
    D: np.ndarray       # uint64[n] upper bound on dist(center, v)
    stats: dict
    trace: np.ndarray


CONTRACT_RESET = 0       # contracted clusters relax as (0, c_u) (Procedure Contract)
CONTRACT_CUMULATIVE = 1  # contracted nodes relax with their own bound D_u


def cluster(g: CSR, tau: float, seed: int, delta0_value: int, trace_cap: int = 1 << 16,
            contract_mode: int = CONTRACT_RESET, step_cap: int = 0) -> Clustering:
    """CLUSTER(G, tau) of Algorithm 1 with the Section 5 initial Delta passed in; optionally the
    cumulative contract mode and the O(n / tau) cap on growing steps per PartialGrowth (end of Section 3)."""
    lib = _lib_load()
    center = np.empty(g.n, np.uint32)
    D = np.empty(g.n, np.uint64)
    st = Stats()
    tr = np.zeros(trace_cap, TRACE_DTYPE)
    tl = ctypes.c_uint64()
    rc = lib.orc_cluster_opts(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), float(tau), seed, delta0_value,
                              int(contract_mode), int(step_cap), _ptr(center), _ptr(D), ctypes.byref(st), _ptr(tr),
                              trace_cap, ctypes.addressof(tl))
    if rc != 0:
        raise RuntimeError(f"orc_cluster failed: {rc}")
    stats = {f: getattr(st, f) for f, _ in Stats._fields_ if f != "pad"}
    return Clustering(center, D, stats, tr[:min(tl.value, trace_cap)].copy())


class C2Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("steps", ctypes.c_uint32), ("centers_drawn", ctypes.c_uint64),
                ("node_updates", ctypes.c_uint64), ("r_cl", ctypes.c_uint64)]


def cluster2(g: CSR, tau: float, seed: int, delta0_value: int, contract_mode: int = CONTRACT_RESET,
             step_cap: int = 0) -> Clustering:
    """CLUSTER2(G, tau) of Algorithm 2 (Section 4): CLUSTER for R_CL, then log n iterations drawing new
    centers with probability 2^i / n, PartialGrowth2 with Delta = 2 R_CL and Contract2 on an explicit
    contracted edge list.  D_v is the length of the path the growth followed from c_v."""
    lib = _lib_load()
    center = np.empty(g.n, np.uint32)
    D = np.empty(g.n, np.uint64)
    st = C2Stats()
    rc = lib.orc_cluster2(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), float(tau), seed, delta0_value,
                          int(contract_mode), int(step_cap), _ptr(center), _ptr(D), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"orc_cluster2 failed: {rc}")
    stats = {f: getattr(st, f) for f, _ in C2Stats._fields_}
    return Clustering(center, D, stats, np.zeros(0, TRACE_DTYPE))


@dataclass
class Quotient:
    k: int
    cid: np.ndarray   # uint32[n]
    off: np.ndarray   # uint64[k+1]
    col: np.ndarray   # uint32[nq]
    w: np.ndarray     # uint64[nq]


def quotient(g: CSR, cl: Clustering) -> Quotient:
    """Weighted quotient graph G_C of Section 4 (edge weight w(u,v) + d_u + d_v, min per pair)."""
    lib = _lib_load()
    cid = np.empty(g.n, np.uint32)
    k = ctypes.c_uint32()
    qoff = np.empty(g.n + 1, np.uint64)
    cap = max(g.nnz, 1)
    qcol = np.empty(cap, np.uint32)
    qw = np.empty(cap, np.uint64)
    center = _c(cl.center, np.uint32); D = _c(cl.D, np.uint64)
    nq = lib.orc_quotient(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), _ptr(center), _ptr(D), _ptr(cid),
                          ctypes.addressof(k), _ptr(qoff), _ptr(qcol), _ptr(qw))
    if nq < 0:
        raise RuntimeError(f"orc_quotient failed: {nq}")
    kk = k.value
    return Quotient(kk, cid, qoff[:kk + 1].copy(), qcol[:nq].copy(), qw[:nq].copy())


def dijkstra(g: CSR, source: int) -> np.ndarray:
    d = np.empty(g.n, np.uint64)
    rc = _lib_load().orc_dijkstra(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), None, source, _ptr(d))
    if rc:
        raise RuntimeError(rc)
    return d


def apsp_max(q: Quotient) -> int:
    """Phi(G_C): largest finite distance of the quotient graph (Section 4)."""
    phi = ctypes.c_uint64()
    rc = _lib_load().orc_apsp_max(q.k, _ptr(q.off), _ptr(q.col), _ptr(q.w), ctypes.addressof(phi))
    if rc:
        raise RuntimeError(rc)
    return phi.value


def sssp_source(seed: int, n: int) -> int:
    return int(_lib_load().orc_sssp_source(seed, n))


def lower_bound(g: CSR, source: int, sweeps: int = 4):
    """(LB, ecc(source)): repeated farthest-node SSSP sweeps (Table 2 caption)."""
    lb = ctypes.c_uint64(); e0 = ctypes.c_uint64()
    rc = _lib_load().orc_lower_bound(g.n, _ptr(g.off), _ptr(g.col), _ptr(g.wt), source, sweeps,
                                     ctypes.addressof(lb), ctypes.addressof(e0))
    if rc:
        raise RuntimeError(rc)
    return lb.value, e0.value


@dataclass
class Result:
    k: int
    phi_gc: int
    radius: int
    phi_approx: int
    stats: dict


def estimate(q: Quotient, cl: Clustering) -> Result:
    """Phi_approx = Phi(G_C) + 2R with R the largest D of the clustering (Section 4)."""
    phi = apsp_max(q)
    R = int(cl.D.max()) if cl.D.size else 0
    return Result(q.k, phi, R, phi + 2 * R, cl.stats)


def cldiam(g: CSR, tau: float, seed: int, delta0_mode: int = DELTA0_AVG):
    """Whole CL-DIAM pipeline on a built CSR: CLUSTER -> G_C -> Phi_approx."""
    d0 = delta0(g, delta0_mode)
    cl = cluster(g, tau, seed, d0)
    q = quotient(g, cl)
    return estimate(q, cl), cl, q
