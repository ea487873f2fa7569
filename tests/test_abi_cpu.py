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


def _c_layout(exprs):
    """sizeof / offsetof values of the header's structs, from gcc."""
    import subprocess
    import tempfile
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"jet.h\"\nint main(void){\n"
    for e in exprs:
        src += f'printf("%zu\\n", (size_t)({e}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    return [int(x) for x in out]


def test_struct_layouts_match_header():
    """Every struct the binding passes across the ABI has the size and field
    offsets the C compiler gives the header's declaration."""
    cases = [("jet_options", binding.Options), ("jet_stats", binding._CStats), ("jet_batch_item", binding._BatchItem),
             ("jet_learned_info", binding._LearnedInfo), ("jet_tune_report", binding._TuneReport)]
    exprs = []
    for cname, py in cases:
        exprs.append(f"sizeof({cname})")
        exprs += [f"offsetof({cname}, {f[0]})" for f in py._fields_]
    vals = iter(_c_layout(exprs))
    for cname, py in cases:
        assert next(vals) == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert next(vals) == getattr(py, f[0]).offset, (cname, f[0])


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
