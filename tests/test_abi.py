"""The C ABI library loads without a GPU and exports every function that
include/rtsdf.h declares (no compute call is made here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rtsdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtsdf_[a-z_]+)\s*\(", src)))


def _lib():
    from paper_2210_04449_gb300 import _abi, build
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi.lib()


def test_header_declares_the_pipeline():
    names = _declared()
    for n in ("rtsdf_create", "rtsdf_upload_mesh", "rtsdf_build_bvh", "rtsdf_voxelize", "rtsdf_jfa",
              "rtsdf_trace", "rtsdf_shadow", "rtsdf_shadow_backward"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2210_04449_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == _declared()


def test_host_only_calls():
    lib = _lib()
    assert lib.rtsdf_version().decode().count(".") == 2
    for code in range(8):
        assert lib.rtsdf_status_str(code)
    # argument errors are reported before any device work
    from paper_2210_04449_gb300 import _abi
    assert lib.rtsdf_create(None, None) == 1
    assert lib.rtsdf_destroy(None) == 1
    assert lib.rtsdf_sync(None) == 1
    assert lib.rtsdf_set_bvh_builder(None, 1) == 1
    assert lib.rtsdf_get_bvh_builder(None, None) == 1
    assert lib.rtsdf_get_bvh_topology(None, None, None, None) == 1
    from paper_2210_04449_gb300._abi import F3
    assert lib.rtsdf_shadow_fallback(None, None, None, 0, F3(0.0, 1.0, 0.0), 1.0, None, None) == 1
    cfg = _abi.Config()
    cfg.extent = 1.0
    cfg.coarse_n = 300          # above the 256 limit
    import ctypes
    h = ctypes.c_void_p()
    assert lib.rtsdf_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.coarse_n = 16
    cfg.alpha = 2.0             # outside [0, 1]
    assert lib.rtsdf_create(ctypes.byref(cfg), ctypes.byref(h)) == 1


def test_product_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2210_04449_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
