"""Pins of the oracle's discrete problem and multigrid cycle (CPU only).

The oracle is checked against: numpy/LAPACK solves of its assembled system,
second-order convergence to manufactured solutions, the BLFA amplification
factor of eq. LFA2Dampl / LFA3Dampl measured on an actual grid, and the
convergence factors the paper prints (tests/golden/paper_values.txt).
"""

import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_value(key):
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        if parts[0] == key:
            return float(parts[1]), float(parts[2])
    raise KeyError(key)


def rho_of(d, N, phi, **kw):
    orc = O.Oracle(d, N, phi, **kw)
    nn = orc.nn(0)
    orc.set_rhs(np.zeros(nn), np.zeros(orc.info(0)["n_ghost"]))
    r, _ = orc.rho(W.random_u0(nn, 3), 16)
    return r


# ------------------------------------------------------------ direct solve

@pytest.mark.parametrize("d,N,mk", [(2, 12, W.phi_disk), (2, 16, W.phi_flower_paper),
                                    (3, 12, W.phi_ellipsoid)])
def test_dense_solve_matches_lapack(oracle_mod, d, N, mk):
    orc = O.Oracle(d, N, mk(N))
    f, us = W.manufactured(d, N)
    g = orc.ghosts(0)
    orc.set_rhs(f, W.g_at(d, g["Q"]))
    u0 = np.zeros(orc.nn(0))
    act, A, rhs = orc.assemble(0, u0, orc.F(0))
    x_np = np.linalg.solve(A, rhs)
    u = orc.direct_solve(0, u0, orc.F(0))
    np.testing.assert_allclose(u[act], x_np, rtol=1e-11, atol=1e-12)
    # the assembled rows are the residual operator: r = F - A u
    rng = np.random.default_rng(1)
    v = np.zeros(orc.nn(0))
    v[act] = rng.uniform(-1, 1, act.size)
    r = orc.residual(0, v, orc.F(0))
    np.testing.assert_allclose(r[act], rhs - A @ v[act], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("d,N,mk", [(2, 16, W.phi_disk), (2, 32, W.phi_flower_paper),
                                    (3, 16, W.phi_ellipsoid)])
def test_multigrid_fixed_point_is_the_discrete_solution(oracle_mod, d, N, mk):
    orc = O.Oracle(d, N, mk(N))
    assert orc.L >= 2
    f, us = W.manufactured(d, N)
    orc.set_rhs(f, W.g_at(d, orc.ghosts(0)["Q"]))
    u_mg, cycles, hist = orc.solve(np.zeros(orc.nn(0)), 1e-14, 200)
    assert cycles < 200
    u_dir = orc.direct_solve(0, np.zeros(orc.nn(0)), orc.F(0))
    act = np.isin(orc.cls(0), [O.INTERIOR, O.GHOST])
    scale = np.abs(u_dir[act]).max()
    assert np.abs(u_mg[act] - u_dir[act]).max() <= 1e-11 * scale


# ----------------------------------------------------- discretisation order

@pytest.mark.parametrize("d,Ns,mk", [(2, [32, 64, 128, 256], W.phi_disk),
                                     (2, [64, 128, 256], W.phi_flower_paper),
                                     (3, [32, 64, 128], W.phi_ellipsoid)])
def test_second_order_accuracy(oracle_mod, d, Ns, mk):
    # Sec. 3.3: the ghost-point discretisation with the 3^d stencil is second
    # order accurate: the max error drops by ~4 per halving of h
    errs = []
    for N in Ns:
        orc = O.Oracle(d, N, mk(N))
        f, us = W.manufactured(d, N)
        orc.set_rhs(f, W.g_at(d, orc.ghosts(0)["Q"]))
        u, c, _ = orc.solve(np.zeros(orc.nn(0)), 1e-11, 100)
        act = orc.cls(0) == O.INTERIOR
        errs.append(np.abs(u - us)[act].max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios[-2:] > 3.3) and np.all(ratios[-2:] < 5.0), ratios


# ------------------------------------------------------- BLFA on a grid

@pytest.mark.parametrize("theta", [0.3, 0.8])
@pytest.mark.parametrize("k_frac", [0.55, 0.8, 0.95])
def test_blfa_amplification_2d_grid(oracle_mod, theta, k_frac):
    # eq. LFA2Dampl: with the interior solved exactly (REL-BC) and ghost values
    # set to the tangential mode sin(alpha j), one ghost relaxation multiplies
    # the mode by 1 - dtau (c_-2 e^{-2p} + c_-1 e^{-p} + c_0) up to O(e^{-2 p N})
    N = 64
    h = 2.0 / N
    iG = N - 2
    xV = (-1 + iG * h) - theta * h
    orc = O.Oracle(2, N, W.phi_halfspace(2, N, xV), max_levels=1, dtau_mode=O.DT_POLY)
    g = orc.ghosts(0)
    n = N + 1
    k = int(round(k_frac * N))
    alpha = k * math.pi / N
    u = np.zeros(orc.nn(0))
    u[g["idx"]] = np.sin(alpha * (g["idx"] // n))
    F = np.zeros(orc.nn(0))
    u = orc.interior_block(0, u, F)
    u2 = orc.ghost_relax(0, u, F)
    m = np.abs(u[g["idx"]]) > 1e-2
    ratio = u2[g["idx"]][m] / u[g["idx"]][m]
    p = math.acosh(2 - math.cos(alpha))
    c2, c1, c0 = theta * (theta - 1) / 2, theta * (2 - theta), (1 - theta) * (2 - theta) / 2
    G = 1 - g["dtau"][0] * (c2 * math.exp(-2 * p) + c1 * math.exp(-p) + c0)
    np.testing.assert_allclose(ratio, G, rtol=0, atol=1e-10)


def test_blfa_amplification_3d_grid(oracle_mod):
    # eq. LFA3Dampl with p(alpha_1, alpha_2) of eq. alphaNalpha3D
    N = 16
    h = 2.0 / N
    iG = N - 2
    theta = 0.6
    xV = (-1 + iG * h) - theta * h
    orc = O.Oracle(3, N, W.phi_halfspace(3, N, xV), max_levels=1, dtau_mode=O.DT_POLY)
    g = orc.ghosts(0)
    n = N + 1
    k1, k2 = 11, 6
    a1, a2 = k1 * math.pi / N, k2 * math.pi / N
    j = (g["idx"] // n) % n
    kk = g["idx"] // (n * n)
    u = np.zeros(orc.nn(0))
    u[g["idx"]] = np.sin(a1 * j) * np.sin(a2 * kk)
    F = np.zeros(orc.nn(0))
    u = orc.interior_block(0, u, F)
    u2 = orc.ghost_relax(0, u, F)
    m = np.abs(u[g["idx"]]) > 1e-2
    ratio = u2[g["idx"]][m] / u[g["idx"]][m]
    p = math.acosh(3 - math.cos(a1) - math.cos(a2))
    c2, c1, c0 = theta * (theta - 1) / 2, theta * (2 - theta), (1 - theta) * (2 - theta) / 2
    G = 1 - g["dtau"][0] * (c2 * math.exp(-2 * p) + c1 * math.exp(-p) + c0)
    np.testing.assert_allclose(ratio, G, rtol=0, atol=1e-9)


def test_ghost_relaxation_with_inverse_c0_is_gauss_seidel(oracle_mod):
    # after eq. relghostdt: dtau = 1/c_0 solves the ghost's own equation
    N = 32
    h = 2.0 / N
    theta = 0.35
    xV = (-1 + N * h) - theta * h
    c0 = (1 - theta) * (2 - theta) / 2
    orc = O.Oracle(1, N, W.phi_halfspace(1, N, xV), max_levels=1, dtau_mode=O.DT_CONST,
                   dtau_const=1.0 / c0)
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, orc.nn(0))
    F = np.zeros(orc.nn(0))
    F[orc.ghosts(0)["idx"]] = 0.37
    u2 = orc.ghost_relax(0, u, F)
    r = orc.residual(0, u2, F)
    assert abs(r[orc.ghosts(0)["idx"][0]]) < 1e-14


# -------------------------------------------------- convergence factors

def test_rho_box_2d_gslex_tgcs(oracle_mod):
    want, tol = paper_value("rho_opt_2d_box")
    r = rho_of(2, 64, W.phi_box(2, 64), ordering=O.LEX, cycle=O.CYC_TGCS)
    assert abs(r - want) <= tol, r


def test_rho_box_3d_gslex_tgcs(oracle_mod):
    want, tol = paper_value("rho_opt_3d_box")
    r = rho_of(3, 32, W.phi_box(3, 32), ordering=O.LEX, cycle=O.CYC_TGCS)
    assert abs(r - want) <= tol, r


@pytest.mark.parametrize("theta", [0.1, 0.5, 0.9])
def test_rho_1d_tgcs_small_dtau(oracle_mod, theta):
    # Sec. 2.2: in 1D rho stays at the interior value for small Delta tau
    want, tol = paper_value("rho_opt_1d_tgcs")
    N = 512
    h = 2.0 / N
    xV = (-1 + N * h) - theta * h
    r = rho_of(1, N, W.phi_halfspace(1, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS,
               dtau_mode=O.DT_CONST, dtau_const=0.2, max_levels=2)
    assert abs(r - want) <= tol, r


def test_rho_1d_diverges_for_large_dtau(oracle_mod):
    # Sec. 2.2: the cycle stops converging when Delta tau is too large
    N = 512
    h = 2.0 / N
    xV = (-1 + N * h) - 0.5 * h
    r = rho_of(1, N, W.phi_halfspace(1, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS,
               dtau_mode=O.DT_CONST, dtau_const=4.0, max_levels=2)
    assert not (r < 1.0)


@pytest.mark.parametrize("theta", [0.2, 0.5])
@pytest.mark.parametrize("shift", [4, 3])
def test_rectangle_optimal_dtau_keeps_interior_factor(oracle_mod, theta, shift):
    # eq. rhomax: with Delta tau_OPT(theta) REL-ALL matches rho_OPT
    want, tol = paper_value("rho_opt_2d_box")
    N = 64
    h = 2.0 / N
    xV = (-1 + (N - shift) * h) - theta * h
    r = rho_of(2, N, W.phi_halfspace(2, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS,
               dtau_mode=O.DT_POLY)
    r_box = rho_of(2, N, W.phi_box(2, N), ordering=O.LEX, cycle=O.CYC_TGCS)
    assert r <= r_box + 0.01 and abs(r - want) <= tol, (r, r_box)


def test_curved_optimal_beats_constant_2d(oracle_mod):
    # Sec. 3.3.3 (Circle): constant Delta tau = 1.75 gives rho about 0.3, the
    # theta-dependent Delta tau_OPT does better
    want, tol = paper_value("rho_const_1p75_2d")
    N = 128
    ph = W.phi_circle_paper(N)
    r_opt = rho_of(2, N, ph, ordering=O.LEX, cycle=O.CYC_TGCS)
    r_c = rho_of(2, N, ph, ordering=O.LEX, cycle=O.CYC_TGCS, dtau_mode=O.DT_CONST, dtau_const=1.75)
    assert abs(r_c - want) <= tol, r_c
    assert r_opt < r_c - 0.05, (r_opt, r_c)


def test_curved_optimal_beats_constant_3d(oracle_mod):
    # Sec. 4.2 (ellipsoid): constant Delta tau = 1.75 gives rho about 0.5
    want, tol = paper_value("rho_const_1p75_3d")
    N = 32
    ph = W.phi_ellipsoid(N)
    r_opt = rho_of(3, N, ph, ordering=O.LEX, cycle=O.CYC_TGCS)
    r_c = rho_of(3, N, ph, ordering=O.LEX, cycle=O.CYC_TGCS, dtau_mode=O.DT_CONST, dtau_const=1.75)
    assert abs(r_c - want) <= tol, r_c
    assert r_opt < r_c - 0.1, (r_opt, r_c)


def test_red_black_vcycle_box_factor(oracle_mod):
    # red-black GS with FW and bilinear interpolation smooths better than
    # GS-LEX; its V(2,1) factor on the box stays well below the GS-LEX value
    r_rb = rho_of(2, 64, W.phi_box(2, 64))
    r_lex = rho_of(2, 64, W.phi_box(2, 64), ordering=O.LEX)
    assert r_rb < 0.09 and r_rb < r_lex
