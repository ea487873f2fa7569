"""ctypes binding of libjet.so (the C ABI in include/jet.h).

Marshalling only: tensors are passed as raw device pointers plus sizes, the
context enqueues on the CUDA stream it was created with, and every call
returns after the library has synchronised that stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

JET_MAX_K = 1024
JET_MAX_LEVELS = 64
FLAG_VALIDATE, FLAG_HOSTLOOP, FLAG_PROFILE = 1, 2, 4
FLAG_NO_LOCKS, FLAG_NO_AFTERBURN, FLAG_WEAK_AFTERBURN, FLAG_BASELINE_LP = 16, 32, 64, 128
FLAG_TWO_HOP = 256
FLAG_STRICT_GAIN = 512
FLAG_NO_PDL = 1024
FLAG_GRID_LOOP = 2048
KIND_LP, KIND_RW, KIND_RS = 0, 1, 2
NONE_GAIN = -(2 ** 31)
JET_KERNELS = 16      # size of the per-kernel statistics rows (JET_K_* indices)
JET_K_COUNT = 10      # refinement kernels in use

EXPORTED_SYMBOLS = [
    "jet_options_default", "jet_ctx_create", "jet_ctx_destroy", "jet_coarsen", "jet_hier_destroy",
    "jet_hier_info", "jet_hier_level", "jet_uncoarsen", "jet_refine", "jet_last_trace", "jet_partition",
    "jet_partition_host", "jet_cut", "jet_lp_pass", "jet_rebalance_pass", "jet_hem", "jet_initial_partition",
    "jet_status_string", "jet_last_error", "jet_lp_pass_noalloc", "jet_two_hop", "jet_partition_batch",
    "jet_coarsest_refined", "jet_lip_num_params", "jet_lip_create", "jet_lip_destroy", "jet_lip_get_params",
    "jet_lip_set_params", "jet_lip_features", "jet_lip_labels", "jet_lip_forward", "jet_lip_loss_grad",
    "jet_lip_train_step", "jet_lip_decode", "jet_lip_initial_partition", "jet_partition_learned", "jet_autotune",
    "jet_kernel_name", "jet_alloc_count", "jet_debug_fail_alloc",
]
LIP_FEATURES, LIP_HIDDEN, LIP_MAX_K, LIP_MAX_N = 16, 64, 256, 1 << 20
JET_NOALLOC_MAX_N = 262144

_STATUS = {0: "JET_OK", 1: "JET_WUNBALANCED", 2: "JET_WITERLIMIT", -1: "JET_EINVAL", -2: "JET_EGRAPH",
           -3: "JET_ENOMEM", -4: "JET_ECUDA", -5: "JET_ETIMEOUT", -6: "JET_EOVERFLOW"}


class JetError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)} ({status_string(status)}) {detail}".strip())


class Options(ctypes.Structure):
    """jet_options (defaults from jet_options_default)."""
    _fields_ = [("c_fine", ctypes.c_double), ("c_coarse", ctypes.c_double), ("phi", ctypes.c_double),
                ("max_no_improve", ctypes.c_int32), ("weak_limit", ctypes.c_int32),
                ("coarsen_target", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("max_iters_per_level", ctypes.c_int32), ("hem_rounds", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("cluster_max_n", ctypes.c_int32), ("cluster_blocks", ctypes.c_int32),
                ("barrier_polls", ctypes.c_int32), ("list_blocks_per_sm", ctypes.c_int32),
                ("list_items_per_block", ctypes.c_int32), ("apply_blocks_per_sm", ctypes.c_int32),
                ("scan_blocks_per_sm", ctypes.c_int32), ("hub_degree", ctypes.c_int32)]

    @classmethod
    def default(cls, **kw) -> "Options":
        o = cls()
        load_library().jet_options_default(ctypes.byref(o))
        for key, val in kw.items():
            if not hasattr(o, key):
                raise AttributeError(key)
            setattr(o, key, val)
        return o


class _CStats(ctypes.Structure):
    L = JET_MAX_LEVELS
    _fields_ = [("levels", ctypes.c_int32),
                ("n", ctypes.c_int64 * L), ("m", ctypes.c_int64 * L),
                ("iters_lp", ctypes.c_int32 * L), ("iters_rw", ctypes.c_int32 * L), ("iters_rs", ctypes.c_int32 * L),
                ("cut_level", ctypes.c_int64 * L),
                ("edge_iters", ctypes.c_int64), ("fin_edge_iters", ctypes.c_int64),
                ("ms_coarsen", ctypes.c_float), ("ms_init", ctypes.c_float), ("ms_refine", ctypes.c_float),
                ("ms_refine_finest", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("cut", ctypes.c_int64), ("max_part_w", ctypes.c_int64),
                ("bytes_model", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("sel_launches", ctypes.c_int64 * L), ("sel_bytes", ctypes.c_int64 * L),
                ("sel_ms", ctypes.c_float * L), ("ms_level", ctypes.c_float * L),
                ("cluster_blocks", ctypes.c_int32 * L),
                ("kern_launches", (ctypes.c_int64 * JET_KERNELS) * L),
                ("kern_bytes", (ctypes.c_int64 * JET_KERNELS) * L),
                ("kern_ms", (ctypes.c_float * JET_KERNELS) * L)]


@dataclass
class Stats:
    levels: int = 0
    n: list = field(default_factory=list)
    m: list = field(default_factory=list)
    iters_lp: list = field(default_factory=list)
    iters_rw: list = field(default_factory=list)
    iters_rs: list = field(default_factory=list)
    cut_level: list = field(default_factory=list)
    edge_iters: int = 0
    fin_edge_iters: int = 0
    ms_coarsen: float = 0.0
    ms_init: float = 0.0
    ms_refine: float = 0.0
    ms_refine_finest: float = 0.0
    ms_total: float = 0.0
    cut: int = 0
    max_part_w: int = 0
    bytes_model: int = 0
    kernel_launches: int = 0
    sel_launches: list = field(default_factory=list)
    sel_bytes: list = field(default_factory=list)
    sel_ms: list = field(default_factory=list)
    ms_level: list = field(default_factory=list)
    cluster_blocks: list = field(default_factory=list)
    # per level, one entry per refinement kernel (JET_K_* order, kernel_names())
    kern_launches: list = field(default_factory=list)
    kern_bytes: list = field(default_factory=list)
    kern_ms: list = field(default_factory=list)

    @classmethod
    def from_c(cls, s: _CStats) -> "Stats":
        lv = s.levels
        rows = lambda a: [list(a[i][:JET_K_COUNT]) for i in range(lv)]   # noqa: E731
        return cls(lv, list(s.n[:lv]), list(s.m[:lv]), list(s.iters_lp[:lv]), list(s.iters_rw[:lv]),
                   list(s.iters_rs[:lv]), list(s.cut_level[:lv]), s.edge_iters, s.fin_edge_iters, s.ms_coarsen,
                   s.ms_init, s.ms_refine, s.ms_refine_finest, s.ms_total, s.cut, s.max_part_w, s.bytes_model,
                   s.kernel_launches, list(s.sel_launches[:lv]), list(s.sel_bytes[:lv]), list(s.sel_ms[:lv]),
                   list(s.ms_level[:lv]), list(s.cluster_blocks[:lv]), rows(s.kern_launches), rows(s.kern_bytes),
                   rows(s.kern_ms))


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libjet.so, building it first if the in-tree copy is missing or
    stale.  Raises if it cannot be built or loaded (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib_path = path or os.environ.get("JET_LIBRARY") or _build.build()
        L = ctypes.CDLL(lib_path)
        vp, i32, i64, u32, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_double)
        P = ctypes.POINTER
        sig = {
            "jet_options_default": (None, [P(Options)]),
            "jet_ctx_create": (ctypes.c_int, [ctypes.c_int, vp, P(Options), P(vp)]),
            "jet_ctx_destroy": (None, [vp]),
            "jet_coarsen": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, u64, P(vp)]),
            "jet_hier_destroy": (None, [vp]),
            "jet_hier_info": (ctypes.c_int, [vp, P(i32), vp, vp]),
            "jet_hier_level": (ctypes.c_int, [vp, i32, P(i32), P(vp), P(vp), P(vp), P(vp), P(vp)]),
            "jet_uncoarsen": (ctypes.c_int, [vp, vp, i32, f64, u64, vp, P(i64), P(_CStats)]),
            "jet_refine": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, f64, i32, u64, vp, P(i64)]),
            "jet_last_trace": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp, P(i32)]),
            "jet_partition": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, f64, u64, vp, P(i64), P(_CStats)]),
            "jet_partition_host": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, f64, u64, vp, P(i64), P(_CStats)]),
            "jet_cut": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, vp, P(i64), vp]),
            "jet_lp_pass": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, vp, vp, f64, u32, vp, vp, vp, vp, vp]),
            "jet_lp_pass_noalloc": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, vp, vp, f64, u32, vp, vp, vp, vp,
                                                   vp]),
            "jet_rebalance_pass": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, i32, f64, i32, u64, i32, vp, vp, vp,
                                                  P(i64), P(i64)]),
            "jet_hem": (ctypes.c_int, [vp, i32, vp, vp, vp, u64, i32, i32, vp]),
            "jet_two_hop": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
            "jet_partition_batch": (ctypes.c_int, [vp, i32, vp, i32]),
            "jet_initial_partition": (ctypes.c_int, [vp, i32, vp, vp, vp, i32, vp]),
            "jet_coarsest_refined": (ctypes.c_int, [vp, vp, i32, f64, u64, vp, P(i64)]),
            "jet_lip_num_params": (i64, [i32]),
            "jet_lip_create": (ctypes.c_int, [vp, i32, vp, P(vp)]),
            "jet_lip_destroy": (None, [vp]),
            "jet_lip_get_params": (ctypes.c_int, [vp, vp, vp]),
            "jet_lip_set_params": (ctypes.c_int, [vp, vp, vp]),
            "jet_lip_features": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp]),
            "jet_lip_labels": (ctypes.c_int, [vp, i32, vp, vp, i32, vp, vp]),
            "jet_lip_forward": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp]),
            "jet_lip_loss_grad": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp, P(ctypes.c_float), vp]),
            "jet_lip_train_step": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp, ctypes.c_float, P(ctypes.c_float)]),
            "jet_lip_decode": (ctypes.c_int, [vp, i32, vp, vp, i32, i64, vp]),
            "jet_lip_initial_partition": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp, f64, vp]),
            "jet_partition_learned": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp, f64, u64, vp, P(i64), P(_CStats),
                                                     P(_LearnedInfo)]),
            "jet_autotune": (ctypes.c_int, [vp, i32, vp, i32, P(_TuneReport)]),
            "jet_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "jet_kernel_name": (ctypes.c_char_p, [i32]),
            "jet_alloc_count": (i64, []),
            "jet_debug_fail_alloc": (None, [i64]),
            "jet_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def debug_fail_alloc(nth: int) -> None:
    """Make the nth device allocation the library attempts from now on fail
    with JET_ENOMEM (host-side injection, one shot); 0 disarms."""
    load_library().jet_debug_fail_alloc(int(nth))


def alloc_count() -> int:
    """Device allocations the library has made in this process so far."""
    return int(load_library().jet_alloc_count())


def kernel_names() -> list[str]:
    """Names of the refinement kernels, in the order of Stats.kern_* rows."""
    L = load_library()
    return [L.jet_kernel_name(i).decode() for i in range(JET_K_COUNT)]


def status_string(status: int) -> str:
    if _lib is None:
        return _STATUS.get(status, str(status))
    return _lib.jet_status_string(status).decode()


def _check(status: int, where: str) -> int:
    if status < 0:
        detail = load_library().jet_last_error().decode()
        raise JetError(status, where, detail)
    return status


def _torch():
    import torch  # imported lazily: the binding needs torch only for tensors
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _DevArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


class _BatchItem(ctypes.Structure):
    """jet_batch_item."""
    _fields_ = [("n", ctypes.c_int32), ("xadj", ctypes.c_void_p), ("adjncy", ctypes.c_void_p),
                ("vwgt", ctypes.c_void_p), ("adjwgt", ctypes.c_void_p), ("k", ctypes.c_int32), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("part_out", ctypes.c_void_p), ("cut", ctypes.c_int64),
                ("status", ctypes.c_int32), ("ms", ctypes.c_float)]


TUNE_MAX_CAND = 48
TUNE_STAGES = ["cluster_blocks", "cluster_max_n", "workers", "list_blocks_per_sm", "apply_blocks_per_sm",
               "list_items_per_block", "scan_blocks_per_sm", "hub_degree"]   # JET_TUNE_* order


class _TuneReport(ctypes.Structure):
    """jet_tune_report."""
    _fields_ = [(f, ctypes.c_int32) for f in ("cluster_max_n", "cluster_blocks", "workers", "list_blocks_per_sm",
                                             "apply_blocks_per_sm", "list_items_per_block", "scan_blocks_per_sm",
                                             "hub_degree", "ncand")] + \
               [("cand_stage", ctypes.c_int32 * TUNE_MAX_CAND), ("cand_value", ctypes.c_int32 * TUNE_MAX_CAND),
                ("cand_ms", ctypes.c_float * TUNE_MAX_CAND)]


class _LearnedInfo(ctypes.Structure):
    """jet_learned_info."""
    _fields_ = [("cut_plain", ctypes.c_int64), ("cut_learned", ctypes.c_int64), ("status_plain", ctypes.c_int32),
                ("status_learned", ctypes.c_int32), ("chosen", ctypes.c_int32), ("n_coarsest", ctypes.c_int32),
                ("ms_coarsen", ctypes.c_float), ("ms_plain", ctypes.c_float), ("ms_proposal", ctypes.c_float),
                ("ms_learned", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class LearnedPartitioner:
    """A jet_lip model (the learned initial partition's network) for k parts
    on a context's device.  ``params`` is the initial parameter vector
    (float32, jet_lip_num_params(k) entries, drawn by the caller)."""

    def __init__(self, ctx: "Context", k: int, params):
        self._ctx, self.k = ctx, int(k)
        self.num_params = num_lip_params(k)
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError(f"params: expected {self.num_params} entries, got {p.size}")
        h = ctypes.c_void_p()
        _check(load_library().jet_lip_create(ctx._h, self.k, ctypes.c_void_p(p.ctypes.data), ctypes.byref(h)),
               "jet_lip_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().jet_lip_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, np.float32)
        _check(load_library().jet_lip_get_params(self._ctx._h, self._h, ctypes.c_void_p(out.ctypes.data)),
               "jet_lip_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError("params size")
        _check(load_library().jet_lip_set_params(self._ctx._h, self._h, ctypes.c_void_p(p.ctypes.data)),
               "jet_lip_set_params")

    def forward(self, xadj, adjncy, x):
        """Logits (float32 tensor n x k) of graph (xadj, adjncy) with features x (n x 16)."""
        torch = _torch()
        c = self._ctx
        n, xadj, adjncy, _, _ = c._graph(xadj, adjncy, None, None)
        x = c._dev(x, torch.float32, "x", n * LIP_FEATURES)
        out = c._out(n * self.k, torch.float32)
        _check(load_library().jet_lip_forward(c._h, self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(x), _ptr(out)),
               "jet_lip_forward")
        return out.view(n, self.k)

    def loss_grad(self, xadj, adjncy, x, labels):
        """(mean cross-entropy, gradient float32 tensor in parameter order)."""
        torch = _torch()
        c = self._ctx
        n, xadj, adjncy, _, _ = c._graph(xadj, adjncy, None, None)
        x = c._dev(x, torch.float32, "x", n * LIP_FEATURES)
        y = c._dev(labels, torch.int32, "labels", n)
        grad = c._out(self.num_params, torch.float32)
        loss = ctypes.c_float()
        _check(load_library().jet_lip_loss_grad(c._h, self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(x), _ptr(y),
                                                ctypes.byref(loss), _ptr(grad)), "jet_lip_loss_grad")
        return loss.value, grad

    def train_step(self, xadj, adjncy, x, labels, lr=1e-3) -> float:
        """One Adam step; returns the loss before it."""
        torch = _torch()
        c = self._ctx
        n, xadj, adjncy, _, _ = c._graph(xadj, adjncy, None, None)
        x = c._dev(x, torch.float32, "x", n * LIP_FEATURES)
        y = c._dev(labels, torch.int32, "labels", n)
        loss = ctypes.c_float()
        _check(load_library().jet_lip_train_step(c._h, self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(x), _ptr(y),
                                                 float(lr), ctypes.byref(loss)), "jet_lip_train_step")
        return loss.value

    def initial_partition(self, xadj, adjncy, vwgt=None, adjwgt=None, eps=0.03):
        """The network's proposal (features, forward, balanced decode)."""
        c = self._ctx
        n, xadj, adjncy, vwgt, adjwgt = c._graph(xadj, adjncy, vwgt, adjwgt)
        part = c._out(n)
        _check(load_library().jet_lip_initial_partition(c._h, self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt),
                                                        _ptr(adjwgt), float(eps), _ptr(part)),
               "jet_lip_initial_partition")
        return part

    def partition(self, xadj, adjncy, vwgt=None, adjwgt=None, eps=0.03, seed=1, return_stats=False):
        """jet_partition_learned: (part, cut, info dict[, Stats])."""
        c = self._ctx
        n, xadj, adjncy, vwgt, adjwgt = c._graph(xadj, adjncy, vwgt, adjwgt)
        part = c._out(n)
        cut = ctypes.c_int64()
        st = _CStats()
        info = _LearnedInfo()
        c.last_status = _check(load_library().jet_partition_learned(
            c._h, self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), float(eps), int(seed), _ptr(part),
            ctypes.byref(cut), ctypes.byref(st), ctypes.byref(info)), "jet_partition_learned")
        out = (part, cut.value, info.as_dict())
        return out + (Stats.from_c(st),) if return_stats else out


def num_lip_params(k: int) -> int:
    v = load_library().jet_lip_num_params(int(k))
    if v < 0:
        raise ValueError(f"k = {k} outside [2, {LIP_MAX_K}]")
    return int(v)


class Hierarchy:
    """Device-resident multilevel hierarchy (jet_coarsen).  Level 0 refers to
    the caller's tensors, which must outlive this object."""

    def __init__(self, ctx: "Context", handle, keep):
        self._ctx, self._h, self._keep = ctx, handle, keep

    def close(self):
        if self._h:
            load_library().jet_hier_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        lv = ctypes.c_int32()
        n = (ctypes.c_int64 * JET_MAX_LEVELS)()
        m = (ctypes.c_int64 * JET_MAX_LEVELS)()
        _check(load_library().jet_hier_info(self._h, ctypes.byref(lv), n, m), "jet_hier_info")
        return lv.value, list(n[:lv.value]), list(m[:lv.value])

    def level(self, i: int) -> dict:
        """Copies of level i's CSR and coarse map as torch tensors."""
        torch = _torch()
        n = ctypes.c_int32()
        px, pa, pv, pw, pc = (ctypes.c_void_p() for _ in range(5))
        _check(load_library().jet_hier_level(self._h, i, ctypes.byref(n), ctypes.byref(px), ctypes.byref(pa),
                                             ctypes.byref(pv), ctypes.byref(pw), ctypes.byref(pc)), "jet_hier_level")
        nv = n.value
        dev = torch.device("cuda", self._ctx.device)

        def view(p, cnt, ts, dt):
            if cnt == 0 or not p.value:
                return torch.zeros(0, dtype=dt, device=dev) if cnt == 0 else None
            return torch.as_tensor(_DevArray(p.value, cnt, ts), device=dev).clone()
        xadj = view(px, nv + 1, "<i8", torch.int64)
        nnz = int(xadj[-1].item())
        return dict(n=nv, xadj=xadj, adjncy=view(pa, nnz, "<i4", torch.int32),
                    vwgt=view(pv, nv, "<i4", torch.int32), adjwgt=view(pw, nnz, "<i4", torch.int32),
                    cmap=view(pc, nv, "<i4", torch.int32) if pc.value else None)


class Context:
    """A jet_ctx bound to one CUDA device and stream."""

    def __init__(self, device: int | None = None, stream=None, options: Options | None = None, **opts):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2304_13194_gb300 needs a CUDA GPU (no CPU fallback)")
        self.device = torch.cuda.current_device() if device is None else int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        o = options if options is not None else Options.default()
        for key, val in opts.items():
            setattr(o, key, val)
        self.options = o
        h = ctypes.c_void_p()
        _check(load_library().jet_ctx_create(self.device, ctypes.c_void_p(raw), ctypes.byref(o), ctypes.byref(h)),
               "jet_ctx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().jet_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers ------------------------------------------------------------
    def _dev(self, t, dtype, name, n=None, allow_none=False):
        torch = _torch()
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        if not isinstance(t, torch.Tensor):
            t = torch.as_tensor(np.asarray(t))
        t = t.to(device=torch.device("cuda", self.device), dtype=dtype).contiguous()
        if n is not None and t.numel() != n:
            raise ValueError(f"{name}: expected {n} entries, got {t.numel()}")
        return t

    def _graph(self, xadj, adjncy, vwgt, adjwgt):
        torch = _torch()
        xadj = self._dev(xadj, torch.int64, "xadj")
        n = xadj.numel() - 1
        adjncy = self._dev(adjncy, torch.int32, "adjncy")
        vwgt = self._dev(vwgt, torch.int32, "vwgt", n, allow_none=True)
        adjwgt = self._dev(adjwgt, torch.int32, "adjwgt", adjncy.numel(), allow_none=True)
        return n, xadj, adjncy, vwgt, adjwgt

    def _out(self, n, dtype=None):
        torch = _torch()
        return torch.empty(max(n, 0), dtype=dtype or torch.int32, device=torch.device("cuda", self.device))

    # -- API ----------------------------------------------------------------
    def partition(self, xadj, adjncy, vwgt=None, adjwgt=None, k=2, eps=0.03, seed=1, return_stats=False):
        """jet_partition: returns (part int32 tensor, cut[, Stats])."""
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        part = self._out(n)
        cut = ctypes.c_int64()
        st = _CStats()
        self.last_status = _check(load_library().jet_partition(
            self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), int(k), float(eps), int(seed),
            _ptr(part), ctypes.byref(cut), ctypes.byref(st)), "jet_partition")
        return (part, cut.value, Stats.from_c(st)) if return_stats else (part, cut.value)

    def partition_batch(self, graphs, workers=8):
        """jet_partition_batch: ``graphs`` is a list of dicts with keys xadj,
        adjncy and optionally vwgt, adjwgt, k, eps, seed.  Returns a list of
        (part int32 tensor, cut, status, ms) in the same order."""
        items = (_BatchItem * max(len(graphs), 1))()
        keep = []
        for i, gd in enumerate(graphs):
            n, xadj, adjncy, vwgt, adjwgt = self._graph(gd["xadj"], gd["adjncy"], gd.get("vwgt"), gd.get("adjwgt"))
            part = self._out(n)
            keep.append((xadj, adjncy, vwgt, adjwgt, part))
            it = items[i]
            it.n = n
            it.xadj, it.adjncy, it.vwgt, it.adjwgt = _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt)
            it.k = int(gd.get("k", 2)); it.eps = float(gd.get("eps", 0.03)); it.seed = int(gd.get("seed", 1))
            it.part_out = _ptr(part)
        self.last_status = _check(load_library().jet_partition_batch(self._h, len(graphs), items, int(workers)),
                                  "jet_partition_batch")
        return [(keep[i][4], items[i].cut, items[i].status, items[i].ms) for i in range(len(graphs))]

    def autotune(self, graphs, reps=3):
        """jet_autotune over a batch (list of dicts as in partition_batch):
        times each candidate execution choice, keeps the fastest
        cluster_max_n in this context's options and returns the report
        (chosen cluster_max_n and workers, every candidate's median ms)."""
        items = (_BatchItem * max(len(graphs), 1))()
        keep = []
        for i, gd in enumerate(graphs):
            n, xadj, adjncy, vwgt, adjwgt = self._graph(gd["xadj"], gd["adjncy"], gd.get("vwgt"), gd.get("adjwgt"))
            part = self._out(n)
            keep.append((xadj, adjncy, vwgt, adjwgt, part))
            it = items[i]
            it.n = n
            it.xadj, it.adjncy, it.vwgt, it.adjwgt = _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt)
            it.k = int(gd.get("k", 2)); it.eps = float(gd.get("eps", 0.03)); it.seed = int(gd.get("seed", 1))
            it.part_out = _ptr(part)
        rep = _TuneReport()
        _check(load_library().jet_autotune(self._h, len(graphs), items, int(reps), ctypes.byref(rep)), "jet_autotune")
        chosen = {f: getattr(rep, f) for f in TUNE_STAGES}
        for f, v in chosen.items():
            if f != "workers":
                setattr(self.options, f, v)
        m = rep.ncand
        return dict(chosen, candidates=[dict(stage=TUNE_STAGES[rep.cand_stage[i]], value=rep.cand_value[i],
                                             ms=rep.cand_ms[i]) for i in range(m)],
                    parts=[(keep[i][4], items[i].cut) for i in range(len(graphs))])

    def partition_host(self, xadj, adjncy, vwgt=None, adjwgt=None, k=2, eps=0.03, seed=1, part_out=None,
                       return_stats=False):
        """jet_partition_host on host (numpy / CPU-tensor) arrays; part_out may
        be a preallocated int32 host array (e.g. pinned)."""
        def host(a, dt):
            if a is None:
                return None
            if hasattr(a, "numpy"):
                a = a.numpy()
            return np.ascontiguousarray(a, dtype=dt)
        xadj = host(xadj, np.int64); adjncy = host(adjncy, np.int32)
        vwgt = host(vwgt, np.int32); adjwgt = host(adjwgt, np.int32)
        n = len(xadj) - 1
        if part_out is None:
            part_out = np.zeros(n, np.int32)
        pp = part_out.ctypes.data if isinstance(part_out, np.ndarray) else part_out.data_ptr()
        cut = ctypes.c_int64()
        st = _CStats()
        hp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self.last_status = _check(load_library().jet_partition_host(
            self._h, n, hp(xadj), hp(adjncy), hp(vwgt), hp(adjwgt), int(k), float(eps), int(seed),
            ctypes.c_void_p(pp), ctypes.byref(cut), ctypes.byref(st)), "jet_partition_host")
        return (part_out, cut.value, Stats.from_c(st)) if return_stats else (part_out, cut.value)

    def coarsen(self, xadj, adjncy, vwgt=None, adjwgt=None, k=2, seed=1) -> Hierarchy:
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        h = ctypes.c_void_p()
        _check(load_library().jet_coarsen(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), int(k),
                                          int(seed), ctypes.byref(h)), "jet_coarsen")
        return Hierarchy(self, h, (xadj, adjncy, vwgt, adjwgt))

    def uncoarsen(self, hier: Hierarchy, k=2, eps=0.03, seed=1, part_out=None, return_stats=False):
        n = hier.info()[1][0]
        part = part_out if part_out is not None else self._out(n)
        cut = ctypes.c_int64()
        st = _CStats()
        self.last_status = _check(load_library().jet_uncoarsen(self._h, hier._h, int(k), float(eps), int(seed),
                                                               _ptr(part), ctypes.byref(cut), ctypes.byref(st)),
                                  "jet_uncoarsen")
        return (part, cut.value, Stats.from_c(st)) if return_stats else (part, cut.value)

    def refine(self, xadj, adjncy, vwgt, adjwgt, k, part, eps=0.03, is_finest=True, seed=1):
        """jet_refine on a copy of ``part``: returns (P_best, cut)."""
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        p = self._dev(part, torch.int32, "part", n).clone()
        cut = ctypes.c_int64()
        self.last_status = _check(load_library().jet_refine(
            self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), int(k), float(eps),
            1 if is_finest else 0, int(seed), _ptr(p), ctypes.byref(cut)), "jet_refine")
        return p, cut.value

    def last_trace(self, cap: int = 4096) -> dict:
        kind = np.zeros(cap, np.int32); nx = np.zeros(cap, np.int64); nm = np.zeros(cap, np.int64)
        cut = np.zeros(cap, np.int64); maxw = np.zeros(cap, np.int64); it = ctypes.c_int32()
        _check(load_library().jet_last_trace(self._h, cap, kind.ctypes.data, nx.ctypes.data, nm.ctypes.data,
                                             cut.ctypes.data, maxw.ctypes.data, ctypes.byref(it)), "jet_last_trace")
        m = min(it.value, cap)
        return dict(iters=it.value, kind=kind[:m], nx=nx[:m], nm=nm[:m], cut=cut[:m], maxw=maxw[:m])

    def cut(self, xadj, adjncy, vwgt, adjwgt, k, part):
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        p = self._dev(part, torch.int32, "part", n)
        pw = self._out(k, torch.int64)
        c = ctypes.c_int64()
        _check(load_library().jet_cut(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), int(k), _ptr(p),
                                      ctypes.byref(c), _ptr(pw)), "jet_cut")
        return c.value, pw

    def lp_pass(self, xadj, adjncy, vwgt, adjwgt, k, part, locked=None, c=0.25, flags=0):
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        p = self._dev(part, torch.int32, "part", n)
        lk = self._dev(locked, torch.uint8, "locked", n, allow_none=True)
        pd, gain, f2 = self._out(n), self._out(n), self._out(n)
        inx, inm = self._out(n, torch.uint8), self._out(n, torch.uint8)
        _check(load_library().jet_lp_pass(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt), int(k),
                                          _ptr(p), _ptr(lk), float(c), int(flags), _ptr(pd), _ptr(gain), _ptr(inx),
                                          _ptr(f2), _ptr(inm)), "jet_lp_pass")
        return dict(Pd=pd, F=gain, inX=inx.bool(), F2=f2, inM=inm.bool())

    def lp_pass_noalloc(self, xadj, adjncy, vwgt, adjwgt, k, part, locked=None, c=0.25, flags=0, out=None):
        """jet_lp_pass_noalloc: the Jetlp pass of lp_pass with the library's
        scratch in its fixed device array (n <= JET_NOALLOC_MAX_N).  ``out``
        may hold preallocated output tensors (keys Pd, F, inX, F2, inM)."""
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        p = self._dev(part, torch.int32, "part", n)
        lk = self._dev(locked, torch.uint8, "locked", n, allow_none=True)
        if out is None:
            out = dict(Pd=self._out(n), F=self._out(n), inX=self._out(n, torch.uint8), F2=self._out(n),
                       inM=self._out(n, torch.uint8))
        _check(load_library().jet_lp_pass_noalloc(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt),
                                                  int(k), _ptr(p), _ptr(lk), float(c), int(flags), _ptr(out["Pd"]),
                                                  _ptr(out["F"]), _ptr(out["inX"]), _ptr(out["F2"]),
                                                  _ptr(out["inM"])), "jet_lp_pass_noalloc")
        return dict(Pd=out["Pd"], F=out["F"], inX=out["inX"].bool(), F2=out["F2"], inM=out["inM"].bool())

    def rebalance_pass(self, xadj, adjncy, vwgt, adjwgt, k, part, eps=0.03, strong=False, seed=1, it=0):
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        p = self._dev(part, torch.int32, "part", n)
        dest, loss = self._out(n), self._out(n)
        nm, nc = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().jet_rebalance_pass(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt),
                                                 int(k), float(eps), 1 if strong else 0, int(seed), int(it), _ptr(p),
                                                 _ptr(dest), _ptr(loss), ctypes.byref(nm), ctypes.byref(nc)),
               "jet_rebalance_pass")
        return dict(dest=dest, loss=loss, nmoves=nm.value, ncand=nc.value)

    def hem(self, xadj, adjncy, adjwgt=None, seed=1, level=0, rounds=8):
        n, xadj, adjncy, _, adjwgt = self._graph(xadj, adjncy, None, adjwgt)
        mate = self._out(n)
        _check(load_library().jet_hem(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(adjwgt), int(seed), int(level),
                                      int(rounds), _ptr(mate)), "jet_hem")
        return mate

    def two_hop(self, xadj, adjncy, mate):
        """jet_two_hop on a copy of ``mate``: returns (mate, vertices matched per stage)."""
        torch = _torch()
        n, xadj, adjncy, _, _ = self._graph(xadj, adjncy, None, None)
        m = self._dev(mate, torch.int32, "mate", n).clone()
        added = (ctypes.c_int64 * 3)()
        _check(load_library().jet_two_hop(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(m), added), "jet_two_hop")
        return m, [int(x) for x in added]

    def initial_partition(self, xadj, adjncy, vwgt, k):
        n, xadj, adjncy, vwgt, _ = self._graph(xadj, adjncy, vwgt, None)
        part = self._out(n)
        _check(load_library().jet_initial_partition(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), int(k),
                                                    _ptr(part)), "jet_initial_partition")
        return part

    def coarsest_refined(self, hier: Hierarchy, k=2, eps=0.03, seed=1):
        """jet_coarsest_refined: the plain pipeline's refined partition of the
        coarsest level (part tensor, cut)."""
        n = hier.info()[1][-1]
        part = self._out(n)
        cut = ctypes.c_int64()
        _check(load_library().jet_coarsest_refined(self._h, hier._h, int(k), float(eps), int(seed), _ptr(part),
                                                   ctypes.byref(cut)), "jet_coarsest_refined")
        return part, cut.value

    def lip_features(self, xadj, adjncy, vwgt=None, adjwgt=None):
        """jet_lip_features: float32 tensor n x 16."""
        torch = _torch()
        n, xadj, adjncy, vwgt, adjwgt = self._graph(xadj, adjncy, vwgt, adjwgt)
        x = self._out(n * LIP_FEATURES, torch.float32)
        _check(load_library().jet_lip_features(self._h, n, _ptr(xadj), _ptr(adjncy), _ptr(vwgt), _ptr(adjwgt),
                                               _ptr(x)), "jet_lip_features")
        return x.view(n, LIP_FEATURES)

    def lip_labels(self, xadj, adjncy, k, part):
        """jet_lip_labels: canonical labels of ``part``."""
        torch = _torch()
        n, xadj, adjncy, _, _ = self._graph(xadj, adjncy, None, None)
        p = self._dev(part, torch.int32, "part", n)
        out = self._out(n)
        _check(load_library().jet_lip_labels(self._h, n, _ptr(xadj), _ptr(adjncy), int(k), _ptr(p), _ptr(out)),
               "jet_lip_labels")
        return out

    def lip_decode(self, logits, k, cap, vwgt=None):
        """jet_lip_decode of float32 logits (n x k)."""
        torch = _torch()
        lg = self._dev(logits, torch.float32, "logits")
        n = lg.numel() // int(k)
        vw = self._dev(vwgt, torch.int32, "vwgt", n, allow_none=True)
        part = self._out(n)
        _check(load_library().jet_lip_decode(self._h, n, _ptr(lg), _ptr(vw), int(k), int(cap), _ptr(part)),
               "jet_lip_decode")
        return part
