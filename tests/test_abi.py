"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every function include/pm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("estimate_permanent", "estimate_permanent_batch", "pm_trace", "pm_context_create"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2608_15390_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_debug_library_exports_every_declared_symbol():
    """The PM_DEBUG variant (bounds-checked trajectory kernels) has the same ABI."""
    from paper_2608_15390_b300 import build
    path = build.build(debug=True)
    assert path.endswith("libpm_b300_debug.so")
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_names_match():
    from paper_2608_15390_b300 import binding
    assert set(declared_functions()) <= set(binding.EXPORTED) | {"pm_status_string", "pm_last_error"}
    assert binding.lib().pm_status_string(1) == b"PM_EINVAL"


def test_product_path_has_no_cpu_fallback():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_2608_15390_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
