"""Seeded synthetic inputs for CL-DIAM (edge lists with uint32 weights).

This module is the only code shared by the CPU oracle and the CUDA path: it
generates graphs and holds none of the diameter method's arithmetic.  The
generators live in ``gen.c`` (Philox4x32-10 counter-based draws, so output is a
pure function of the seed) and are compiled on first use with gcc.

Workloads mirror the paper's synthetic graph families (Section 5, Table 1):
square meshes, R-MAT power-law graphs, and a road-like mesh standing in for
the road networks, which are not available here.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (cached by source hash)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = open(_SRC, "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    out = os.path.join(_BUILD, f"libcldiam_inputs_{tag}.so")
    if force or not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.gen_grid.restype = ctypes.c_int64
            lib.gen_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u32p]
            lib.gen_road_mesh_max_edges.restype = ctypes.c_int64
            lib.gen_road_mesh_max_edges.argtypes = [ctypes.c_uint32, ctypes.c_double]
            lib.gen_road_mesh.restype = ctypes.c_int64
            lib.gen_road_mesh.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                          ctypes.c_uint64, u32p, u32p, u32p]
            lib.gen_rmat.restype = ctypes.c_int64
            lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     u32p, u32p, u32p, u32p]
            lib.gen_mix_params.restype = None
            lib.gen_mix_params.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p, u32p, u32p,
                                           ctypes.POINTER(ctypes.c_uint64)]
            lib.gen_queries.restype = None
            lib.gen_queries.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint32, ctypes.POINTER(ctypes.c_double), u32p]
            lib.gen_philox4x32.restype = None
            lib.gen_philox4x32.argtypes = [ctypes.c_uint64, u32p, u32p]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class EdgeList:
    """An undirected multigraph as parallel uint32 arrays (src, dst, w) on n nodes."""

    def __init__(self, n, src, dst, w, name=""):
        self.n = int(n)
        self.src = src
        self.dst = dst
        self.w = w
        self.name = name

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def __repr__(self):
        return f"EdgeList({self.name!r}, n={self.n}, m={self.m})"


def grid(side: int, W: int, seed: int) -> EdgeList:
    lib = _load()
    m = 2 * side * (side - 1)
    src = np.empty(m, np.uint32); dst = np.empty(m, np.uint32); w = np.empty(m, np.uint32)
    got = lib.gen_grid(side, W, seed, _p(src), _p(dst), _p(w))
    assert got == m
    return EdgeList(side * side, src, dst, w, f"grid{side}")


def road_mesh(side: int, W: int, seed: int, p_del: float = 0.1, chord_frac: float = 0.001) -> EdgeList:
    lib = _load()
    cap = lib.gen_road_mesh_max_edges(side, chord_frac)
    src = np.empty(cap, np.uint32); dst = np.empty(cap, np.uint32); w = np.empty(cap, np.uint32)
    m = lib.gen_road_mesh(side, p_del, chord_frac, W, seed, _p(src), _p(dst), _p(w))
    return EdgeList(side * side, src[:m].copy(), dst[:m].copy(), w[:m].copy(), f"roadmesh{side}")


def rmat(scale: int, ef: int, W: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True) -> EdgeList:
    lib = _load()
    n = 1 << scale
    m = ef * n
    src = np.empty(m, np.uint32); dst = np.empty(m, np.uint32); w = np.empty(m, np.uint32)
    perm = np.empty(n, np.uint32)
    got = lib.gen_rmat(scale, ef, W, seed, a, b, c, 1 if permute else 0, _p(src), _p(dst), _p(w), _p(perm))
    assert got == m
    return EdgeList(n, src, dst, w, f"rmat{scale}")


def mix_params(seed: int, g: int):
    """(kind, scale, side, subseed) of graph g in the many-graph mixture; kind 0 = R-MAT, 1 = mesh."""
    lib = _load()
    k = ctypes.c_uint32(); s = ctypes.c_uint32(); sd = ctypes.c_uint32(); ss = ctypes.c_uint64()
    lib.gen_mix_params(seed, g, ctypes.byref(k), ctypes.byref(s), ctypes.byref(sd), ctypes.byref(ss))
    return k.value, s.value, sd.value, ss.value


def mix_graph(seed: int, g: int, W: int = 1000) -> EdgeList:
    kind, scale, side, sub = mix_params(seed, g)
    if kind == 0:
        e = rmat(scale, 8, W, sub)
        e.name = f"mix{g}:rmat{scale}"
    else:
        e = grid(side, W, sub)
        e.name = f"mix{g}:grid{side}"
    return e


def queries(seed: int, count: int, rate: float, p_big: float, n_small: int):
    lib = _load()
    arr = np.empty(count, np.float64); g = np.empty(count, np.uint32)
    lib.gen_queries(seed, count, rate, p_big, n_small, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _p(g))
    return arr, g


def philox4x32(seed: int, ctr) -> np.ndarray:
    lib = _load()
    c = np.asarray(ctr, np.uint32)
    o = np.empty(4, np.uint32)
    lib.gen_philox4x32(seed, _p(c), _p(o))
    return o
