"""Seeded synthetic graph inputs shared by the oracle tests, the CUDA parity
tests and the benchmark.

This package holds no arithmetic of the partitioning method: it only builds
CSR graphs (undirected, no self-loops, no parallel edges, positive integer
weights) shaped like the paper's workloads (Sec. 5 "Test Graphs": meshes such
as the 2000x4000 grid and the 200^3 cube; power-law and geometric graphs as
stand-ins for the irregular classes).  Generation is a pure function of the
parameters and the seed (splitmix64 counter streams in ``graphgen.c``).

    g = graphgen.grid3d(128, 128, 128, vw=(1, 4), ew=(1, 10), seed=1)
    g.n, g.xadj (int64[n+1]), g.adjncy (int32[2m]), g.vwgt, g.adjwgt (int32)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library next to this file."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            out = [P(ctypes.c_int32), P(P(ctypes.c_int64)), P(P(ctypes.c_int32)),
                   P(P(ctypes.c_int32)), P(P(ctypes.c_int32))]
            i32, u64, f64 = ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.gg_grid.argtypes = [i32, i32, i32, i32, i32, i32, i32, u64] + out
            lib.gg_rmat.argtypes = [i32, i32, f64, f64, f64, u64, i32, i32, i32, i32] + out
            lib.gg_rgg.argtypes = [i32, f64, u64, i32, i32, i32, i32] + out
            lib.gg_gnp.argtypes = [i32, f64, u64, i32, i32, i32, i32] + out
            lib.gg_from_edges.argtypes = [i32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          i32, i32, i32, i32, u64] + out
            lib.gg_free.argtypes = [ctypes.c_void_p]
            for f in (lib.gg_grid, lib.gg_rmat, lib.gg_rgg, lib.gg_gnp, lib.gg_from_edges):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """CSR graph.  ``xadj`` int64[n+1], ``adjncy``/``adjwgt`` int32[2m],
    ``vwgt`` int32[n].  ``name`` describes the generator call."""
    n: int
    xadj: np.ndarray
    adjncy: np.ndarray
    vwgt: np.ndarray
    adjwgt: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.xadj[-1]) // 2

    @property
    def nnz(self) -> int:
        return int(self.xadj[-1])


def _call(fn, *args, name=""):
    lib = _load()
    n = ctypes.c_int32()
    px = ctypes.POINTER(ctypes.c_int64)()
    pa, pv, pw = (ctypes.POINTER(ctypes.c_int32)() for _ in range(3))
    rc = fn(*args, ctypes.byref(n), ctypes.byref(px), ctypes.byref(pa), ctypes.byref(pv), ctypes.byref(pw))
    if rc != 0:
        raise MemoryError(f"graphgen: {name} failed ({rc})")
    nv = n.value
    try:
        xadj = np.ctypeslib.as_array(px, shape=(nv + 1,)).copy()
        nnz = int(xadj[-1])
        adj = np.ctypeslib.as_array(pa, shape=(max(nnz, 1),))[:nnz].copy()
        ew = np.ctypeslib.as_array(pw, shape=(max(nnz, 1),))[:nnz].copy()
        vw = np.ctypeslib.as_array(pv, shape=(max(nv, 1),))[:nv].copy()
    finally:
        for p in (px, pa, pv, pw):
            lib.gg_free(ctypes.cast(p, ctypes.c_void_p))
    return Graph(nv, xadj, adj, vw, ew, name)


def _rng(r):
    return (int(r[0]), int(r[1])) if isinstance(r, (tuple, list)) else (int(r), int(r))


def grid2d(nx: int, ny: int, vw=1, ew=1, seed: int = 1) -> Graph:
    """nx*ny mesh, 5-point stencil."""
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_grid, nx, ny, 1, vlo, vhi, elo, ehi, seed,
                 name=f"grid2d_{nx}x{ny}_vw{vlo}-{vhi}_ew{elo}-{ehi}_s{seed}")


def grid3d(nx: int, ny: int, nz: int, vw=1, ew=1, seed: int = 1) -> Graph:
    """nx*ny*nz mesh, 7-point stencil."""
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_grid, nx, ny, nz, vlo, vhi, elo, ehi, seed,
                 name=f"grid3d_{nx}x{ny}x{nz}_vw{vlo}-{vhi}_ew{elo}-{ehi}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed: int = 1, vw=1, ew=1) -> Graph:
    """R-MAT, symmetrised, self-loops and duplicates removed, isolated vertices kept."""
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_rmat, scale, edge_factor, a, b, c, seed, vlo, vhi, elo, ehi,
                 name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def rgg(n: int, radius: float | None = None, seed: int = 1, vw=1, ew=1, mean_degree: float = 8.0) -> Graph:
    """Random geometric graph in the unit square; default radius gives the
    requested mean degree (boundary effect ignored): r = sqrt(d / (pi n))."""
    if radius is None:
        radius = float(np.sqrt(mean_degree / (np.pi * max(n, 1))))
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_rgg, n, radius, seed, vlo, vhi, elo, ehi, name=f"rgg_n{n}_s{seed}")


def gnp(n: int, p: float, seed: int = 1, vw=1, ew=1) -> Graph:
    """Erdos-Renyi G(n, p) (small test graphs)."""
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_gnp, n, p, seed, vlo, vhi, elo, ehi, name=f"gnp_n{n}_p{p}_s{seed}")


def from_edges(n: int, edges, vw=1, ew=1, seed: int = 1, name: str = "edges") -> Graph:
    """CSR from an undirected edge list [(u, v), ...]; weights drawn per edge."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0]); dst = np.ascontiguousarray(e[:, 1])
    (vlo, vhi), (elo, ehi) = _rng(vw), _rng(ew)
    return _call(_load().gg_from_edges, n, len(e), src.ctypes.data, dst.ctypes.data,
                 vlo, vhi, elo, ehi, seed, name=name)


def with_weights(g: Graph, vwgt=None, adjwgt=None, name: str | None = None) -> Graph:
    """Copy of ``g`` with explicit weight arrays (adjwgt must be symmetric)."""
    return Graph(g.n, g.xadj.copy(), g.adjncy.copy(),
                 g.vwgt.copy() if vwgt is None else np.asarray(vwgt, dtype=np.int32).copy(),
                 g.adjwgt.copy() if adjwgt is None else np.asarray(adjwgt, dtype=np.int32).copy(),
                 name or g.name)


def disjoint_union(*gs: Graph, name: str = "union") -> Graph:
    """Disjoint union (vertex ids of later graphs shifted)."""
    xs, adjs, vws, ews, off, eoff = [np.zeros(1, np.int64)], [], [], [], 0, 0
    for g in gs:
        xs.append(g.xadj[1:] + eoff)
        adjs.append(g.adjncy + off); vws.append(g.vwgt); ews.append(g.adjwgt)
        off += g.n; eoff += g.nnz
    return Graph(off, np.concatenate(xs).astype(np.int64), np.concatenate(adjs).astype(np.int32),
                 np.concatenate(vws).astype(np.int32), np.concatenate(ews).astype(np.int32), name)
