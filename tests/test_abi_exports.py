"""The C-ABI library loads and exports every entry point include/pbdr.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:int|const char \*)\s*(pbdr_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pbdr_ctx_create", "pbdr_create_scene", "pbdr_step", "pbdr_read_state"):
        assert required in names


def test_library_exports_every_declared_symbol(pbdr_lib):
    from paper_2603_14634_gb300.build import LIB
    lib = ctypes.CDLL(LIB)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pbdr_\w+)$", out, re.M))
    assert set(_declared()) <= exported
    # the binding wraps exactly the declared set
    assert set(pbdr_lib.EXPORTS) == set(_declared())


def test_library_built_for_sm_103a():
    from paper_2603_14634_gb300 import build as B
    assert "arch=compute_103a,code=sm_103a" in B.ARCH


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2603_14634_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved
