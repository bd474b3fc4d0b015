"""CPU checks of the boundary: the C-ABI library builds, loads and exports
every entry point declared in include/gbp.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2308_08410_gb300 import build, gbp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "gbp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(gbp_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(gbp.exported_symbols()) == set(names)


def test_status_strings_without_gpu():
    lib = gbp.load()
    for s in range(10):
        assert lib.gbp_status_string(s)


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        gbp.Context(0)
