"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ace.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:int|void)\s+(\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2110_07670_gb300 import build
    build.build_library()
    import paper_2110_07670_gb300 as ace
    return ace.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("ace_plan_create", "ace_build", "ace_apply", "hfx_apply_exact", "ace_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    import paper_2110_07670_gb300 as ace
    assert set(_declared()) <= set(ace.SYMBOLS) | {"ace_plan_destroy"}


def test_last_error_without_gpu_work(lib):
    import ctypes
    buf = ctypes.create_string_buffer(64)
    n = lib.ace_last_error(buf, 64)
    assert n >= 0


def test_package_has_no_cpu_fallback():
    """The product path never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2110_07670_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "ace_oracle" not in txt, f
