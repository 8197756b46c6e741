"""The C-ABI library builds, loads and exports every function include/svt.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "svt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(svt_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_stage_entry_points():
    names = declared_functions()
    for stage in ("svt_unpack", "svt_combine", "svt_fit", "svt_select", "svt_format", "svt_run"):
        assert stage in names


def test_library_exports_every_declared_symbol():
    from paper_1311_0380_gb300 import build, _native
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding describes every declared function
    assert set(declared_functions()) <= set(_native.SIGNATURES)


def test_version_and_workspace_sizes_need_no_gpu():
    from paper_1311_0380_gb300 import _native
    L = _native.load()
    assert L.svt_version() >= 10000
    assert L.svt_unpack_workspace_size(0) > 0
    assert L.svt_run_workspace_size(1 << 20, 1000, 50000, None) > 50000 * 20


def test_autotune_cache_key_separates_flushed_and_back_to_back_timing():
    """The schedule cache keys on the GPU, the workload shape and whether the
    tuner timed every run after an L2 flush (host logic only)."""
    from paper_1311_0380_gb300 import api, autotune
    cfg = api.config(15, 15, 100, 4096, 5, 512)
    a = autotune.signature(1 << 20, 3000, 191300, cfg)
    b = autotune.signature(1 << 20, 3000, 191300, cfg, flushed=True)
    assert a != b and a.endswith("|l0") and b.endswith("|l1")
    assert autotune.signature((1 << 20) + 5, 3000, 191300, cfg) == a   # same powers of two
    assert autotune.signature(1 << 21, 3000, 191300, cfg) != a
