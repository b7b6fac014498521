"""The C-ABI library builds for sm_103a and exports every function declared in
include/bcmg.h (no GPU needed: nothing is called)."""

import ctypes
import shutil

import pytest


def test_library_exports_every_declared_symbol():
    from paper_2207_14208_gb300 import bcmg, build
    if shutil.which("nvcc") is None and not build.os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = build.build()
    lib = ctypes.CDLL(path)
    names = bcmg.declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_declares_the_boundary_calls():
    from paper_2207_14208_gb300 import bcmg
    names = set(bcmg.declared_functions())
    for n in ["bcmg_create_grid_hierarchy", "bcmg_vcycle", "bcmg_solve", "bcmg_residual_norm",
              "bcmg_destroy", "bcmg_last_error"]:
        assert n in names


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2207_14208_gb300 import bcmg
    monkeypatch.setattr(bcmg, "_lib", None)
    monkeypatch.setattr(bcmg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="library missing"):
        bcmg.load()
