"""The C-ABI library loads and exports every entry point include/icarus.h declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(icarus_\w+)\s*\(", src)) - {"icarus_alloc_fn", "icarus_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_2501_15923_gb300 import build
    build.build()
    from paper_2501_15923_gb300 import icarus as ic
    return ic.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared("icarus.h")
    assert "icarus_init" in names and "icarus_step" in names and "icarus_sample" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2501_15923_gb300 import icarus as ic
    names = declared("icarus.h")
    assert set(names) <= set(ic.SIGNATURES), set(names) - set(ic.SIGNATURES)


def test_last_error_is_callable_without_gpu(lib):
    assert isinstance(lib.icarus_last_error(), bytes)
