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


def test_dtau_opt_host_matches_oracle():
    # the library's Delta tau_OPT (a host function: no GPU needed) against
    # the oracle's, for both boundary conditions, both G0 forms, 2D and 3D
    import numpy as np
    from oracle import oracle as O
    from paper_2207_14208_gb300 import bcmg, build
    build.build()
    for d in (2, 3):
        for bc in (0, 1):
            for mode in (bcmg.DTAU_EXP, bcmg.DTAU_POLY):
                for th in np.linspace(0.0, 1.0, 11):
                    a = bcmg.dtau_opt(d, th, mode, bc=bc)
                    b = O.dtau(d, th, mode, bc=bc)
                    assert abs(a - b) <= 1e-14 * abs(b), (d, bc, mode, th, a, b)
    # the Neumann 2D values of eq. dtauoptLFA_Neumann at theta = 0, 1/2, 1
    for th, want in [(0.0, 0.92099), (0.5, 1.28166), (1.0, 2.10663)]:
        assert abs(bcmg.dtau_opt(2, th, bcmg.DTAU_POLY, bc=1) - want) < 1e-5


def test_footprint_per_axis_matches_estimate():
    # bcmg_footprint (grid size per axis) is the estimate of
    # bcmg_footprint_estimate; a host function, no GPU needed
    from paper_2207_14208_gb300 import bcmg, build
    if shutil.which("nvcc") is None and not build.os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    build.build()
    for d, N in ((2, 128), (3, 64), (2, 1024)):
        for prec in (bcmg.PREC_FP64, bcmg.PREC_MIXED):
            assert bcmg.footprint(d, [N] * d, precision=prec) == bcmg.footprint_estimate(d, N, precision=prec) > 0
    with pytest.raises(bcmg.BcmgError) as e:
        bcmg.footprint(3, [64, 64, 32])
    assert e.value.code == bcmg.EINVAL
