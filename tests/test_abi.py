"""The C-ABI library loads and exports every entry point include/md.h
declares; the product package does not reach the oracle.  No GPU needed."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2505_08491_gb300 import build
    return build.build()


def test_library_exports_declared_symbols(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (md_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert len(declared_symbols()) >= 20


def test_binding_declares_every_symbol(lib_path):
    from paper_2505_08491_gb300 import _lib
    lib = _lib.load(lib_path)
    for s in declared_symbols():
        assert s in _lib.SIGNATURES, s
        assert getattr(lib, s) is not None
    assert lib.md_version().decode().startswith("md-gb300")


def test_library_targets_sm103a(lib_path):
    """The shared library carries sm_103a device code only (checked from the
    build command, not from the binary)."""
    from paper_2505_08491_gb300 import build
    assert build.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2505_08491_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), f
                assert "oracle/" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2505_08491_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved
