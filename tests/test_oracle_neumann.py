"""Oracle pins for Neumann boundary rows and the reaction term (CPU only).

Neumann ghost rows (Sec. 3.2.2 in 1D/2D, Sec. 4.1 in 3D) are the normal
derivative at Q of the ghost's quadratic interpolant.  They are pinned by
what fixes them independently of the oracle's code: exactness on quadratic
functions (the gradient of any quadratic is reproduced), the 1D coefficients
(c_0, c_-1, c_-2)/h = ((3/2 - theta), 2(theta - 1), (1/2 - theta))/h of eq.
coeffN on a straight boundary, second-order accuracy on manufactured
solutions, and convergence of the cycle on the paper's Test1N (mixed
Dirichlet/Neumann) and Test2N (u - Lap u = f with Neumann) problems.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W


def _quad2(X, Y):
    return 1 + 2 * X - Y + 3 * X * X - X * Y + 0.5 * Y * Y


def _grad_quad2(P):
    x, y = P[:, 0], P[:, 1]
    return np.stack([2 + 6 * x - y, -1 - x + y], 1)


def _quad3(X, Y, Z):
    return 0.5 - X + 2 * Y + Z + X * X - 2 * Y * Z + 0.7 * Z * Z + X * Y


def _grad_quad3(P):
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    return np.stack([-1 + 2 * x + y, 2 - 2 * z + x, 1 - 2 * y + 1.4 * z], 1)


def _ghost_rows(o, u):
    act, A, _ = o.assemble(0, u, np.zeros(o.nn(0)))
    pos = {a: i for i, a in enumerate(act)}
    gh = o.ghosts(0)
    return np.array([A[pos[X]] @ u[act] for X in gh["idx"]]), gh


@pytest.mark.parametrize("d,N,mk", [(2, 32, W.phi_disk), (2, 48, W.phi_flower_paper), (3, 20, W.phi_ellipsoid)])
def test_neumann_rows_exact_on_quadratics(oracle_mod, d, N, mk):
    o = O.Oracle(d, N, mk(N), bc=O.NEUMANN, reaction=1.0)
    C = [c.reshape(-1) for c in W.coords(d, N)]
    u = _quad2(*C) if d == 2 else _quad3(*C)
    Bu, gh = _ghost_rows(o, u)
    grad = _grad_quad2(gh["Q"]) if d == 2 else _grad_quad3(gh["Q"])
    want = (grad * gh["n"][:, :d]).sum(1)
    full = (gh["q"][:, :d] == 2).all(1)
    assert full.sum() > 10
    np.testing.assert_allclose(Bu[full], want[full], rtol=0, atol=1e-10 * np.abs(want).max())


def test_neumann_row_on_straight_boundary_is_eq_coeffN(oracle_mod):
    # domain x < xV: ghosts on the column x = 0.25, theta = (0.25 - xV)/h,
    # n = (1, 0); the row is (1/h)((3/2-theta) u_G + 2(theta-1) u_-1 + (1/2-theta) u_-2)
    N, xV = 16, 0.2
    h = 2.0 / N
    theta = (0.25 - xV) / h
    o = O.Oracle(2, N, W.phi_halfspace(2, N, xV), bc=O.NEUMANN)
    act, A, _ = o.assemble(0, np.zeros(o.nn(0)), np.zeros(o.nn(0)))
    pos = {a: i for i, a in enumerate(act)}
    n = N + 1
    checked = 0
    for X in o.ghosts(0)["idx"]:
        i, j = X % n, X // n
        assert i == 10
        row = A[pos[X]]
        nz = {act[k]: row[k] for k in np.nonzero(row)[0]}
        want = {X: (1.5 - theta) / h, X - 1: 2 * (theta - 1) / h, X - 2: (0.5 - theta) / h}
        assert set(nz) == set(want)
        for k, v in want.items():
            assert nz[k] == pytest.approx(v, rel=1e-13)
        checked += 1
    assert checked > 5


def test_reaction_term_on_the_diagonal(oracle_mod):
    N, c = 24, 2.5
    o0 = O.Oracle(2, N, W.phi_disk(N))
    o1 = O.Oracle(2, N, W.phi_disk(N), reaction=c)
    z = np.zeros(o0.nn(0))
    act, A0, _ = o0.assemble(0, z, z)
    _, A1, _ = o1.assemble(0, z, z)
    interior = o0.cls(0)[act] == O.INTERIOR
    D = A1 - A0
    np.testing.assert_allclose(np.diag(D)[interior], c, rtol=1e-12)
    D[np.diag_indices_from(D)] = 0.0
    assert not D.any() and not np.diag(A1 - A0)[~interior].any()


def _man2_reaction(N):
    X, Y = [c.reshape(-1) for c in W.coords(2, N)]
    us = np.sin(np.pi * X) * np.cos(np.pi * Y) * np.exp(X)
    f, _ = W.manufactured(2, N)  # -Lap u*
    return us, f + us              # u* - Lap u*


def _grad_u2(P):
    x, y = P[:, 0], P[:, 1]
    ux = (np.pi * np.cos(np.pi * x) + np.sin(np.pi * x)) * np.cos(np.pi * y) * np.exp(x)
    uy = -np.pi * np.sin(np.pi * x) * np.sin(np.pi * y) * np.exp(x)
    return np.stack([ux, uy], 1)


def _solve_test2n(N, mk, mode=O.DT_EXP, const=1.75):
    o = O.Oracle(2, N, mk(N), bc=O.NEUMANN, reaction=1.0, dtau_mode=mode, dtau_const=const)
    us, f = _man2_reaction(N)
    gh = o.ghosts(0)
    o.set_rhs(f, (_grad_u2(gh["Q"]) * gh["n"][:, :2]).sum(1))
    u, c, hist = o.solve(np.zeros(o.nn(0)), 1e-10, 120)
    interior = o.cls(0) == O.INTERIOR
    rates = hist[1:] / hist[:-1]
    return np.abs(u - us)[interior].max(), c, float(np.mean(rates[-5:]))


def test_test2n_second_order_and_convergence(oracle_mod):
    # Test2N (Sec. 4.2): u - Lap u = f on the disk, Neumann data from u*
    errs = []
    for N in (32, 64, 128):
        e, c, rho = _solve_test2n(N, W.phi_disk)
        assert c <= 40 and rho < 0.45
        errs.append(e)
    assert errs[1] <= errs[0] / 3 and errs[2] <= errs[1] / 3
    # the flower converges too, more slowly (the paper notes the same)
    e, c, rho = _solve_test2n(64, W.phi_flower_paper)
    assert c <= 60 and rho < 0.65


def test_test2n_optimal_dtau_not_worse_than_constant(oracle_mod):
    # constant Delta tau / h = 1 against Delta tau_OPT(theta) (Sec. 4.2: the
    # choice matters less for Neumann than for Dirichlet)
    _, c_opt, rho_opt = _solve_test2n(64, W.phi_disk)
    _, c_cst, rho_cst = _solve_test2n(64, W.phi_disk, O.DT_CONST, 1.0)
    assert rho_opt <= 1.1 * rho_cst


def _phi_line(N, beta=0.35, c=0.1):
    X, Y = W.coords(2, N)
    return (X * math.cos(beta) + Y * math.sin(beta) - c).reshape(-1)


def test_test1n_mixed_dirichlet_neumann(oracle_mod):
    # Test1N (Sec. 4.2): Dirichlet on the box sides inside the domain (the
    # eliminated nodes hold u*), Neumann on the oblique line phi = 0; Poisson
    errs = []
    for N in (32, 64, 128):
        o = O.Oracle(2, N, _phi_line(N), bc=O.NEUMANN)
        X, Y = [c.reshape(-1) for c in W.coords(2, N)]
        us = np.sin(np.pi * X) * np.cos(np.pi * Y) * np.exp(X)
        f, _ = W.manufactured(2, N)
        gh = o.ghosts(0)
        o.set_rhs(f, (_grad_u2(gh["Q"]) * gh["n"][:, :2]).sum(1))
        u0 = np.zeros(o.nn(0))
        box = o.cls(0) == O.BOXDIR
        assert box.any()
        u0[box] = us[box]
        u, c, hist = o.solve(u0, 1e-10, 120)
        assert c <= 40
        errs.append(np.abs(u - us)[o.cls(0) == O.INTERIOR].max())
    assert errs[1] <= errs[0] / 3 and errs[2] <= errs[1] / 3
