"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/bgemm.h declares; the binding's signatures match the header."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{]*\)\s*;", text)
    return sorted(set(n for n in names if n not in ("sizeof",)))


def test_header_declares_the_paths_entry_points():
    names = declared_functions()
    for n in ("batched_gemm_fixed", "batched_gemm_plan", "batched_gemm_grouped", "chain_plan",
              "chain_step", "bg_plan_destroy", "bg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(bglib):
    import paper_2203_09353_gb300 as bg
    names = declared_functions()
    missing = [n for n in names if not hasattr(bglib, n)]
    assert not missing, missing
    assert sorted(bg.EXPORTS) == names


def test_status_strings_and_version(bglib):
    import paper_2203_09353_gb300 as bg
    assert bg.version().startswith("bgemm-gb300")
    for code, name in bg.STATUS.items():
        assert bglib.bg_status_string(code).decode() == name


def test_structs_match_header_sizes():
    import ctypes
    import paper_2203_09353_gb300 as bg
    assert ctypes.sizeof(bg.Precision) == 16
    assert ctypes.sizeof(bg.Instance) == 72
    assert ctypes.sizeof(bg.PlanInfo) == 40


def test_build_targets_sm103a_only():
    """One -gencode for sm_103a; no other architecture is compiled."""
    from paper_2203_09353_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
