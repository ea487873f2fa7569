"""The oracle: a plain, single-threaded C statement of the Jet partitioner's
definitions (``jet_oracle.c``), loaded through ctypes.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers; the CUDA library and its
Python binding never import this package, and the two share no code.

Graphs are any object with ``n``, ``xadj`` (int64[n+1]), ``adjncy`` (int32),
``vwgt`` and ``adjwgt`` (int32 arrays or None for unit weights), e.g.
``graphgen.Graph``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jet_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libjet_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_LP, KIND_RW, KIND_RS = 0, 1, 2
ABL_NO_LOCKS, ABL_NO_AFTERBURN, ABL_WEAK_AFTERBURN, ABL_BASELINE_LP = 1, 2, 4, 8
ABL_STRICT_GAIN = 32     # first filter keeps only F > 0
TWO_HOP = 16             # coarsening: add two-hop matches after heavy-edge matching (Sec. 3.1)
MATCHMAKER_MAX_DEG = 1024
NONE = np.iinfo(np.int64).min  # the "negative infinity" gain


def build(force: bool = False) -> str:
    """Compile jet_oracle.c (plain C11, -O2, single-threaded)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("xadj", ctypes.c_void_p), ("adjncy", ctypes.c_void_p),
                ("vwgt", ctypes.c_void_p), ("adjwgt", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in (
        "c_fine_q16", "c_coarse_q16", "phi_ppm", "max_no_improve", "weak_limit",
        "coarsen_target", "max_levels", "max_iters", "hem_rounds", "flags")]


class _Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32),
                ("n", ctypes.c_int64 * 64), ("m", ctypes.c_int64 * 64),
                ("it_lp", ctypes.c_int32 * 64), ("it_rw", ctypes.c_int32 * 64), ("it_rs", ctypes.c_int32 * 64),
                ("cut_level", ctypes.c_int64 * 64),
                ("edge_iters", ctypes.c_int64), ("fin_edge_iters", ctypes.c_int64),
                ("cut", ctypes.c_int64), ("maxw", ctypes.c_int64),
                ("sec_coarsen", ctypes.c_double), ("sec_init", ctypes.c_double),
                ("sec_refine", ctypes.c_double), ("sec_refine_finest", ctypes.c_double)]


@dataclass
class Options:
    """The paper's hyper-parameters with its defaults (Sec. 3, 4, 4.1.2, 4.2.2)."""
    c_fine: float = 0.25
    c_coarse: float = 0.75
    phi: float = 0.999
    max_no_improve: int = 12
    weak_limit: int = 2
    coarsen_target: int = 0
    max_levels: int = 64
    max_iters: int = 10000
    hem_rounds: int = 8
    flags: int = 0

    def c_struct(self) -> _Opts:
        return _Opts(int(round(self.c_fine * 65536)), int(round(self.c_coarse * 65536)),
                     int(round(self.phi * 1e6)), self.max_no_improve, self.weak_limit,
                     self.coarsen_target, self.max_levels, self.max_iters, self.hem_rounds, self.flags)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            G = ctypes.POINTER(_Graph)
            vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.or_cut.argtypes = [G, vp]; L.or_cut.restype = i64
            L.or_part_weights.argtypes = [G, vp, i32, vp]
            L.or_limit.argtypes = [i64, i32, f64, vp]; L.or_limit.restype = i64
            L.or_sigma.argtypes = [i64, i64]; L.or_sigma.restype = i64
            L.or_slot.argtypes = [i64]; L.or_slot.restype = i32
            L.or_splitmix64.argtypes = [u64]; L.or_splitmix64.restype = u64
            L.or_level_seed.argtypes = [u64, i32]; L.or_level_seed.restype = u64
            L.or_jetlp.argtypes = [G, i32, vp, vp, i32, i32, vp, vp, vp, vp, vp]
            L.or_jetrw.argtypes = [G, i32, vp, vp, i64, i64, i64, u64, i32, vp, vp, vp]; L.or_jetrw.restype = i64
            L.or_jetrs.argtypes = [G, i32, vp, vp, i64, i64, i64, vp, vp, vp]; L.or_jetrs.restype = i64
            L.or_refine.argtypes = [G, i32, f64, i32, u64, ctypes.POINTER(_Opts), vp, vp, vp,
                                    i32, vp, vp, vp, vp, vp, vp, vp]
            L.or_refine.restype = ctypes.c_int
            L.or_hem.argtypes = [G, u64, i32, i32, vp]; L.or_hem.restype = i64
            L.or_two_hop.argtypes = [G, vp, vp]; L.or_two_hop.restype = i64
            L.or_twin_key.argtypes = [G, i32]; L.or_twin_key.restype = u64
            L.or_coarse_map.argtypes = [i32, vp, vp]; L.or_coarse_map.restype = i32
            L.or_contract.argtypes = [G, vp, i32, vp, vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]
            L.or_initial_partition.argtypes = [G, i32, vp]
            L.or_coarsen_target.argtypes = [i32, ctypes.POINTER(_Opts)]; L.or_coarsen_target.restype = i32
            L.or_coarsen.argtypes = [G, i32, u64, ctypes.POINTER(_Opts)]; L.or_coarsen.restype = vp
            L.or_hier_free.argtypes = [vp]
            L.or_hier_levels.argtypes = [vp]; L.or_hier_levels.restype = i32
            P = ctypes.POINTER
            L.or_hier_get.argtypes = [vp, i32, P(i32), P(vp), P(vp), P(vp), P(vp), P(vp)]
            L.or_uncoarsen.argtypes = [vp, i32, f64, u64, P(_Opts), vp, vp, P(_Stats)]
            L.or_uncoarsen.restype = ctypes.c_int
            L.or_partition.argtypes = [G, i32, f64, u64, P(_Opts), vp, vp, P(_Stats)]
            L.or_partition.restype = ctypes.c_int
            L.or_free.argtypes = [vp]
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


class _GraphRef:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, g):
        self.n = int(g.n)
        self.xadj = np.ascontiguousarray(g.xadj, dtype=np.int64)
        self.adjncy = _i32(g.adjncy)
        self.vwgt = None if g.vwgt is None else _i32(g.vwgt)
        self.adjwgt = None if g.adjwgt is None else _i32(g.adjwgt)
        self.s = _Graph(self.n, self.xadj.ctypes.data, self.adjncy.ctypes.data,
                        _ptr(self.vwgt), _ptr(self.adjwgt))

    @property
    def p(self):
        return ctypes.byref(self.s)

    def total_weight(self) -> int:
        return self.n if self.vwgt is None else int(self.vwgt.astype(np.int64).sum())


def splitmix64(x: int) -> int:
    return int(_load().or_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def level_seed(seed: int, level: int) -> int:
    return int(_load().or_level_seed(seed, level))


def cut(g, part) -> int:
    """Sec. 2.1 cost of a partition."""
    gr = _GraphRef(g); p = _i32(part)
    return int(_load().or_cut(gr.p, p.ctypes.data))


def part_weights(g, part, k: int) -> np.ndarray:
    gr = _GraphRef(g); p = _i32(part); pw = np.zeros(k, np.int64)
    _load().or_part_weights(gr.p, p.ctypes.data, k, pw.ctypes.data)
    return pw


def limit(W: int, k: int, eps: float) -> tuple[int, int]:
    """(L, opt): the integer balance limit and opt = ceil(W/k)."""
    opt = ctypes.c_int64()
    L = _load().or_limit(W, k, eps, ctypes.addressof(opt))
    return int(L), int(opt.value)


def sigma(opt: int, L: int) -> int:
    return int(_load().or_sigma(opt, L))


def slot(x: int) -> int:
    return int(_load().or_slot(x))


def jetlp(g, k: int, part, locked=None, c: float = 0.25, ablation: int = 0) -> dict:
    """One Jetlp pass (Alg. 4); arrays per vertex: Pd, F (NONE = -inf), inX, F2, inM."""
    gr = _GraphRef(g); n = gr.n; p = _i32(part)
    lk = None if locked is None else np.ascontiguousarray(locked, dtype=np.uint8)
    Pd = np.zeros(n, np.int32); F = np.zeros(n, np.int64); inX = np.zeros(n, np.uint8)
    F2 = np.zeros(n, np.int64); inM = np.zeros(n, np.uint8)
    _load().or_jetlp(gr.p, k, p.ctypes.data, _ptr(lk), int(round(c * 65536)), ablation,
                     Pd.ctypes.data, F.ctypes.data, inX.ctypes.data, F2.ctypes.data, inM.ctypes.data)
    return dict(Pd=Pd, F=F, inX=inX.astype(bool), F2=F2, inM=inM.astype(bool))


def _balance(gr, k, eps, pw):
    L, opt = limit(gr.total_weight(), k, eps)
    return L, opt, sigma(opt, L)


def jetrw(g, k: int, part, eps: float = 0.03, seed: int = 1, it: int = 0) -> dict:
    """One Jetrw pass (Alg. 5): dest (-1 = stays), loss (NONE for non-candidates)."""
    gr = _GraphRef(g); n = gr.n; p = _i32(part)
    pw = part_weights(g, p, k)
    L, opt, sg = _balance(gr, k, eps, pw)
    dest = np.zeros(n, np.int32); loss = np.zeros(n, np.int64); nc = ctypes.c_int64()
    nm = _load().or_jetrw(gr.p, k, p.ctypes.data, pw.ctypes.data, L, opt, sg, seed, it,
                          dest.ctypes.data, loss.ctypes.data, ctypes.addressof(nc))
    return dict(dest=dest, loss=loss, nmoves=int(nm), ncand=int(nc.value), L=L, opt=opt, sigma=sg, pw=pw)


def jetrs(g, k: int, part, eps: float = 0.03) -> dict:
    """One Jetrs pass (Sec. 4.2.2): dest (-1 = stays), loss."""
    gr = _GraphRef(g); n = gr.n; p = _i32(part)
    pw = part_weights(g, p, k)
    L, opt, sg = _balance(gr, k, eps, pw)
    dest = np.zeros(n, np.int32); loss = np.zeros(n, np.int64); nc = ctypes.c_int64()
    nm = _load().or_jetrs(gr.p, k, p.ctypes.data, pw.ctypes.data, L, opt, sg,
                          dest.ctypes.data, loss.ctypes.data, ctypes.addressof(nc))
    return dict(dest=dest, loss=loss, nmoves=int(nm), ncand=int(nc.value), L=L, opt=opt, sigma=sg, pw=pw)


@dataclass
class RefineResult:
    part: np.ndarray
    cut: int
    maxw: int
    status: int
    iters: int
    kinds: list = field(default_factory=list)
    trace: dict = field(default_factory=dict)


def refine(g, k: int, part, eps: float = 0.03, c: float | None = None, is_finest: bool = True,
           seed: int = 1, opts: Options | None = None, trace_cap: int = 100000) -> RefineResult:
    """Jet refinement of one level (Alg. 3) starting from ``part``."""
    o = opts or Options()
    if c is None:
        c = o.c_fine if is_finest else o.c_coarse
    gr = _GraphRef(g); p = _i32(part).copy()
    cs = o.c_struct()
    cut_ = ctypes.c_int64(); mw = ctypes.c_int64(); it = ctypes.c_int32(); kc = (ctypes.c_int32 * 3)()
    tk = np.zeros(trace_cap, np.int32); tx = np.zeros(trace_cap, np.int64); tm = np.zeros(trace_cap, np.int64)
    tc = np.zeros(trace_cap, np.int64); tw = np.zeros(trace_cap, np.int64)
    st = _load().or_refine(gr.p, k, eps, int(round(c * 65536)), seed, ctypes.byref(cs), p.ctypes.data,
                           ctypes.addressof(cut_), ctypes.addressof(mw), trace_cap, tk.ctypes.data,
                           tx.ctypes.data, tm.ctypes.data, tc.ctypes.data, tw.ctypes.data,
                           ctypes.addressof(it), ctypes.addressof(kc))
    ni = int(it.value); nt = min(ni, trace_cap)
    return RefineResult(p, int(cut_.value), int(mw.value), int(st), ni, [kc[0], kc[1], kc[2]],
                        dict(kind=tk[:nt], nx=tx[:nt], nm=tm[:nt], cut=tc[:nt], maxw=tw[:nt]))


def hem(g, seed: int = 1, level: int = 0, rounds: int = 8) -> np.ndarray:
    """Heavy-edge matching (Sec. 3.1 reading): mate[v] or -1."""
    gr = _GraphRef(g); mate = np.zeros(gr.n, np.int32)
    _load().or_hem(gr.p, seed, level, rounds, mate.ctypes.data)
    return mate


def two_hop(g, mate) -> tuple[np.ndarray, list[int]]:
    """Two-hop matching after heavy-edge matching (Sec. 3.1 reading): leaves,
    twins, relatives, each stage while > 25% of vertices are unmatched.
    Returns the new mate array and the vertices matched by each stage."""
    gr = _GraphRef(g); m = _i32(mate).copy(); added = np.zeros(3, np.int64)
    _load().or_two_hop(gr.p, m.ctypes.data, added.ctypes.data)
    return m, [int(x) for x in added]


def twin_key(g, v: int) -> int:
    """Order-free neighbourhood hash that identifies twins."""
    gr = _GraphRef(g)
    return int(_load().or_twin_key(gr.p, int(v)))


def coarse_map(mate) -> tuple[np.ndarray, int]:
    m = _i32(mate); cmap = np.zeros(len(m), np.int32)
    nc = _load().or_coarse_map(len(m), m.ctypes.data, cmap.ctypes.data)
    return cmap, int(nc)


@dataclass
class CGraph:
    n: int
    xadj: np.ndarray
    adjncy: np.ndarray
    vwgt: np.ndarray
    adjwgt: np.ndarray

    @property
    def m(self) -> int:
        return int(self.xadj[-1]) // 2


def contract(g, cmap, nc: int) -> CGraph:
    """Alg. 2 edge contraction (rows sorted, self-loops dropped)."""
    gr = _GraphRef(g); cm = _i32(cmap)
    xc = np.zeros(nc + 1, np.int64); vc = np.zeros(max(nc, 1), np.int32)
    pa, pw = ctypes.c_void_p(), ctypes.c_void_p()
    L = _load()
    L.or_contract(gr.p, cm.ctypes.data, nc, xc.ctypes.data, vc.ctypes.data, ctypes.byref(pa), ctypes.byref(pw))
    nnz = int(xc[-1])
    try:
        adj = np.ctypeslib.as_array(ctypes.cast(pa, ctypes.POINTER(ctypes.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
        w = np.ctypeslib.as_array(ctypes.cast(pw, ctypes.POINTER(ctypes.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    finally:
        L.or_free(pa); L.or_free(pw)
    return CGraph(nc, xc, adj, vc[:nc].copy(), w)


def initial_partition(g, k: int) -> np.ndarray:
    gr = _GraphRef(g); part = np.zeros(gr.n, np.int32)
    _load().or_initial_partition(gr.p, k, part.ctypes.data)
    return part


def coarsen_target(k: int, opts: Options | None = None) -> int:
    cs = (opts or Options()).c_struct()
    return int(_load().or_coarsen_target(k, ctypes.byref(cs)))


@dataclass
class Level:
    graph: CGraph
    cmap: np.ndarray | None  # level i -> level i+1


def coarsen(g, k: int, seed: int = 1, opts: Options | None = None) -> list[Level]:
    """MLCoarsen (Alg. 1): the hierarchy as a list of levels (copies)."""
    gr = _GraphRef(g); cs = (opts or Options()).c_struct()
    L = _load()
    h = L.or_coarsen(gr.p, k, seed, ctypes.byref(cs))
    try:
        out = []
        for i in range(L.or_hier_levels(h)):
            n = ctypes.c_int32(); px, pa, pv, pw, pc = (ctypes.c_void_p() for _ in range(5))
            L.or_hier_get(h, i, ctypes.byref(n), ctypes.byref(px), ctypes.byref(pa), ctypes.byref(pv),
                          ctypes.byref(pw), ctypes.byref(pc))
            nv = n.value
            xadj = np.ctypeslib.as_array(ctypes.cast(px, ctypes.POINTER(ctypes.c_int64)), shape=(nv + 1,)).copy()
            nnz = int(xadj[-1])

            def arr(p, cnt):
                if cnt == 0 or not p.value:
                    return np.zeros(0, np.int32)
                return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_int32)), shape=(cnt,)).copy()
            cm = arr(pc, nv) if pc.value else None
            out.append(Level(CGraph(nv, xadj, arr(pa, nnz), arr(pv, nv), arr(pw, nnz)), cm))
        return out
    finally:
        L.or_hier_free(h)


@dataclass
class PartitionResult:
    part: np.ndarray
    cut: int
    status: int
    stats: dict


def _stats_dict(s: _Stats) -> dict:
    lv = s.levels
    return dict(levels=lv, n=list(s.n[:lv]), m=list(s.m[:lv]), it_lp=list(s.it_lp[:lv]),
                it_rw=list(s.it_rw[:lv]), it_rs=list(s.it_rs[:lv]), cut_level=list(s.cut_level[:lv]),
                edge_iters=s.edge_iters, fin_edge_iters=s.fin_edge_iters, cut=s.cut, maxw=s.maxw,
                sec_coarsen=s.sec_coarsen, sec_init=s.sec_init, sec_refine=s.sec_refine,
                sec_refine_finest=s.sec_refine_finest)


def partition(g, k: int, eps: float = 0.03, seed: int = 1, opts: Options | None = None) -> PartitionResult:
    """Alg. 1 end to end: coarsen, initial partition, refine, project, refine."""
    gr = _GraphRef(g); cs = (opts or Options()).c_struct()
    part = np.zeros(gr.n, np.int32); cut_ = ctypes.c_int64(); st = _Stats()
    status = _load().or_partition(gr.p, k, eps, seed, ctypes.byref(cs), part.ctypes.data,
                                  ctypes.addressof(cut_), ctypes.byref(st))
    return PartitionResult(part, int(cut_.value), int(status), _stats_dict(st))
