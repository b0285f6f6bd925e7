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
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", src)))


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


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Every struct the binding passes through the C ABI has the size and field
    offsets that the C compiler gives the declarations in include/bem.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_1510_07244_gb300 import _binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"bem_kernel_desc": b.bem_kernel_desc, "bem_quad_desc": b.bem_quad_desc,
               "bem_block_job": b.bem_block_job, "bem_green_job": b.bem_green_job,
               "bem_mesh_stats": b.bem_mesh_stats, "bem_kernel_time": b.bem_kernel_time}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "bem.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field_name, _ in cls._fields_:
            lines.append(f'printf("{name} {field_name} %zu\\n", offsetof({name}, {field_name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field_name, _ in cls._fields_:
            assert got[(name, field_name)] == getattr(cls, field_name).offset, (name, field_name)
