"""The C ABI library builds, loads, and exports every entry point that
include/bem.h declares (no compute calls: these run without a GPU)."""
import os
import re

import pytest

import paper_1510_07244_gb300 as pkg
from paper_1510_07244_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return pkg.load()


def declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("bem_mesh_upload", "bem_near_field", "bem_pivot_entries", "bem_coupling_blocks",
              "bem_assemble_dense"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared():
        assert hasattr(lib, n), n
    assert sorted(declared()) == sorted(pkg.EXPORTS)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1510_07244_gb300 import _binding
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _binding.load()


def test_package_never_imports_the_oracle():
    pkgdir = os.path.join(ROOT, "paper_1510_07244_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "bem_oracle" not in text, f


def test_create_without_gpu_is_an_error(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.bem_create(ctypes.byref(h), 0, None) != 0
