"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every function include/jet.h declares.  No compute calls."""
import ctypes
import os
import re

import pytest

from paper_2304_13194_gb300 import build as jet_build
from paper_2304_13194_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "jet.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jet_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return jet_build.build()


def test_header_declares_the_binding_symbols():
    assert declared_functions() == sorted(binding.EXPORTED_SYMBOLS)


def test_library_loads_and_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_without_gpu(lib_path):
    L = binding.load_library(lib_path)
    o = binding.Options.default()
    assert (o.c_fine, o.c_coarse, o.phi) == (0.25, 0.75, 0.999)
    assert (o.max_no_improve, o.weak_limit, o.max_levels, o.max_iters_per_level, o.hem_rounds) == (12, 2, 64, 10000, 8)
    assert L.jet_status_string(-6).decode().startswith("weight sums")


def test_library_is_sm103a_only(lib_path):
    # the build passes exactly one -gencode for compute_103a / sm_103a
    assert jet_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(lib_path) > 0


def test_options_struct_layout_matches_header():
    # 3 doubles, 6 int32, 1 uint32, 2 int32 -> 60 bytes, padded to 64
    assert ctypes.sizeof(binding.Options) == 64
    # jet_batch_item: int32, 4 pointers, int32, double, uint64, pointer, int64, int32, float
    assert ctypes.sizeof(binding._BatchItem) == 88
    assert ctypes.sizeof(binding._LearnedInfo) == 48
    assert ctypes.sizeof(binding._TuneReport) == 16 + 4 * 64
    # jet_stats: int32 + 2*64 int64 + 3*64 int32 + 64 int64 + 2 int64 + 5 float + 2 int64
    assert ctypes.sizeof(binding._CStats) % 8 == 0


def test_flag_values_match_header():
    """Every JET_FLAG_* of include/jet.h has the same value in the binding."""
    text = open(os.path.join(ROOT, "include", "jet.h")).read()
    flags = dict(re.findall(r"#define JET_FLAG_([A-Z_]+) (\d+)u", text))
    assert len(flags) >= 11
    for name, value in flags.items():
        assert getattr(binding, "FLAG_" + name) == int(value), name


def test_status_codes_match_header():
    """The binding's status names are the header's codes."""
    text = open(os.path.join(ROOT, "include", "jet.h")).read()
    codes = {name: int(v) for name, v in re.findall(r"#define (JET_(?:OK|E[A-Z]+|W[A-Z]+)) \(?(-?\d+)\)?", text)}
    assert codes["JET_OK"] == 0 and len(codes) == 9
    assert {v: k for k, v in codes.items()} == binding._STATUS
