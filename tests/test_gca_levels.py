"""The level-by-level GCA driver behind bem_gca_pivots_device, on the host:
with every level's Green matrices written in the device call's block layout
(from the host's own integrals), it gives the pivots of bem_gca_pivots bit for
bit (tests/gca_levels_check.cpp, built here with the host compiler).  The
device run of the same driver is compared in tests/test_gpu_representation.py."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from synth import meshes, structure

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_07244_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("gca") / "gca_levels_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", cuda_inc, os.path.join(ROOT, "tests", "gca_levels_check.cpp"),
                    os.path.join(CSRC, "bem_rules.cpp"), "-o", exe, "-lpthread"], check=True)
    return exe


def _write(path, mesh, basis, kappa, g, part):
    ptr, idx = part.cluster_csr()
    son = part.son_array()
    with open(path, "wb") as f:
        np.array([mesh.nv, mesh.nt, 0 if basis == "p0" else 1], np.int64).tofile(f)
        np.array([kappa], np.float64).tofile(f)
        np.array([g, len(ptr) - 1], np.int64).tofile(f)
        np.ascontiguousarray(mesh.verts, np.float64).tofile(f)
        np.ascontiguousarray(mesh.tris, np.int32).tofile(f)
        np.ascontiguousarray(ptr, np.int32).tofile(f)
        np.ascontiguousarray(idx, np.int32).tofile(f)
        np.ascontiguousarray(son, np.int32).tofile(f)


@pytest.mark.parametrize("basis,kappa,g", [("p0", 0.0, 3), ("p1", 0.0, 4), ("p0", 4.0, 2),
                                           ("p1", 2.5, 3)])
def test_level_driver_reproduces_host_pivots(checker, tmp_path, basis, kappa, g):
    mesh = meshes.jitter(meshes.icosphere(3), 0.1, 11)
    part = structure.build_block_partition(mesh, basis, 16, 2.0)
    path = str(tmp_path / "tree.bin")
    _write(path, mesh, basis, kappa, g, part)
    r = subprocess.run([checker, path], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "same 1" in r.stdout
