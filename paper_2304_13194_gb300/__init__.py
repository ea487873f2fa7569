"""GB300 (sm_103a) Jet multilevel k-way graph partitioner.

Thin Python binding over the C ABI of ``libjet.so`` (include/jet.h): argument
marshalling only — every step of coarsening, initial partitioning and Jet
refinement runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library cannot be
built or loaded, or no GPU is present, calls raise.

    import torch, paper_2304_13194_gb300 as jet
    ctx = jet.Context()                                  # current device + stream
    part, cut = ctx.partition(xadj, adjncy, vwgt, adjwgt, k=64, eps=0.03, seed=1)

``xadj`` is int64[n+1], ``adjncy``/``adjwgt`` int32[xadj[n]], ``vwgt``
int32[n]; weights may be None (unit).  Tensors must be CUDA tensors on the
context's device (``partition_host`` takes CPU arrays).
"""
from __future__ import annotations

from .binding import (  # noqa: F401
    JET_MAX_K, JetError, Context, Options, Stats, load_library, status_string, kernel_names, JET_K_COUNT,
    FLAG_VALIDATE, FLAG_HOSTLOOP, FLAG_PROFILE, FLAG_NO_LOCKS, FLAG_NO_AFTERBURN, FLAG_WEAK_AFTERBURN, FLAG_BASELINE_LP,
    FLAG_TWO_HOP, FLAG_STRICT_GAIN, FLAG_NO_PDL, FLAG_GRID_LOOP,
    KIND_LP, KIND_RW, KIND_RS, NONE_GAIN, EXPORTED_SYMBOLS,
    LearnedPartitioner, num_lip_params, LIP_FEATURES, LIP_HIDDEN, LIP_MAX_K, LIP_MAX_N,
)

__all__ = ["Context", "Options", "Stats", "JetError", "load_library", "status_string", "kernel_names", "JET_MAX_K",
           "EXPORTED_SYMBOLS", "LearnedPartitioner", "num_lip_params"]
