"""Pins of the oracle's geometry (Sec. 3.3): node partition, projection point Q,
upwind 3^d stencil and its interpolation weights, band (CPU only)."""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W


def _nbrs(d, N, lin):
    n = N + 1
    ix = [(lin // n ** a) % n for a in range(d)]
    out = []
    for a in range(d):
        for s in (-1, 1):
            iy = list(ix)
            iy[a] += s
            if 0 <= iy[a] <= N:
                out.append(sum(iy[b] * n ** b for b in range(d)))
    return ix, out


@pytest.mark.parametrize("d,N,mk", [(2, 24, lambda N: W.phi_disk(N)),
                                    (2, 30, lambda N: W.phi_flower_paper(N)),
                                    (3, 16, lambda N: W.phi_ellipsoid(N)),
                                    (2, 16, lambda N: W.phi_halfspace(2, N, 0.41))])
def test_partition_matches_definition(oracle_mod, d, N, mk):
    # Omega_h / Gamma_h / I_h of Sec. 3.3 checked by brute force in Python
    phi = mk(N)
    orc = O.Oracle(d, N, phi, max_levels=1)
    cls = orc.cls(0)
    for lin in range(phi.size):
        ix, nb = _nbrs(d, N, lin)
        edge = any(v in (0, N) for v in ix)
        if phi[lin] < 0:
            want = O.BOXDIR if edge else O.INTERIOR
        else:
            inner = [y for y in nb if phi[y] < 0 and not any(
                ((y // (N + 1) ** a) % (N + 1)) in (0, N) for a in range(d))]
            want = O.GHOST if inner else O.INACTIVE
        assert cls[lin] == want, (lin, ix)


def test_projection_point_on_circle(oracle_mod):
    # Q = G - eta h n lies on the zero set: for the disk the distance of Q to
    # the circle is O(h^2) (multilinear interpolation of a quadratic phi);
    # |G - Q| = eta h; and eta = theta~ in [0, 1]
    for N in (64, 128, 256):
        h = 2.0 / N
        orc = O.Oracle(2, N, W.phi_disk(N), max_levels=1)
        g = orc.ghosts(0)
        n = N + 1
        G = np.stack([-1 + (g["idx"] % n) * h, -1 + (g["idx"] // n) * h], axis=1)
        Q = g["Q"]
        assert np.all((g["eta"] >= 0) & (g["eta"] <= 1))
        np.testing.assert_allclose(np.linalg.norm(G - Q, axis=1), g["eta"] * h, rtol=1e-12, atol=1e-15)
        dist = np.abs(np.linalg.norm(Q, axis=1) - 0.7)
        assert dist.max() < 0.5 * h * h
        # the normal is the outward normal of the circle, up to O(h^2)
        nrm = G / np.linalg.norm(G, axis=1)[:, None]
        assert np.max(np.linalg.norm(g["n"] - nrm, axis=1)) < 2 * h * h


def _poly(X, deg_mask):
    # a tensor-product polynomial of degree <= 2 per axis
    out = np.ones(X.shape[0])
    for a in range(X.shape[1]):
        x = X[:, a]
        out = out * (0.3 + (0.7 * x if deg_mask[a] >= 1 else 0) + (-1.1 * x * x if deg_mask[a] >= 2 else 0))
    return out


@pytest.mark.parametrize("d,N,mk", [(2, 64, lambda N: W.phi_flower_paper(N)),
                                    (3, 24, lambda N: W.phi_ellipsoid(N)),
                                    (3, 128, lambda N: W.phi_spheres(N))])
def test_ghost_interpolation_exact_on_polynomials(oracle_mod, d, N, mk):
    # eq. BCh: B u~ at Q is the (bi/tri)quadratic interpolant on ST_G, so it
    # reproduces any tensor polynomial of degree <= q_a per axis exactly.
    orc = O.Oracle(d, N, mk(N), max_levels=1)
    g = orc.ghosts(0)
    C = W.coords(d, N)
    X = np.stack([c.reshape(-1) for c in C], axis=1)
    full = np.all(g["q"] == 2, axis=1)
    assert full.mean() > 0.8
    u = _poly(X, [2] * d)
    got = orc.ghost_apply(0, u)
    want = _poly(g["Q"], [2] * d)
    np.testing.assert_allclose(got[full], want[full], rtol=1e-11, atol=1e-12)
    # every ghost (also the fall-backs) reproduces constants
    np.testing.assert_allclose(orc.ghost_apply(0, np.ones(X.shape[0])), 1.0, rtol=1e-13)
    # stencil geometry: upwind corners, xi = eta |n_a| in [0, 1] unless flipped
    s, xi, n, eta = g["s"], g["xi"], g["n"], g["eta"]
    np.testing.assert_allclose(xi, s * eta[:, None] * n, rtol=1e-13, atol=1e-15)
    up = (np.sign(n) == s) | (n == 0)
    assert np.all(xi[up] >= -1e-15) and np.all(xi[up] <= 1 + 1e-15)


def test_no_inactive_node_in_any_stencil(oracle_mod):
    # Sec. 3.3: ST_G has no inactive node (the fall-back lowers the degree on
    # coarse grids where it would)
    orc = O.Oracle(3, 64, W.phi_spheres(64))
    for l in range(orc.L):
        info = orc.info(l)
        cls = orc.cls(l)
        g = orc.ghosts(l)
        n = info["N"] + 1
        st = [1, n, n * n]
        for k in range(len(g["idx"])):
            X = g["idx"][k]
            for o0 in range(g["q"][k, 0] + 1):
                for o1 in range(g["q"][k, 1] + 1):
                    for o2 in range(g["q"][k, 2] + 1):
                        Y = X - g["s"][k, 0] * o0 * st[0] - g["s"][k, 1] * o1 * st[1] - g["s"][k, 2] * o2 * st[2]
                        assert cls[Y] != O.INACTIVE


def test_theta_distribution_remark(oracle_mod):
    # Remark thetaxy: theta~ covers [0,1), almost uniformly away from 1 and
    # thinning towards 1 (Circle and Flower, N = 2048)
    for fn in (W.phi_circle_paper, W.phi_flower_paper):
        N = 2048
        orc = O.Oracle(2, N, fn(N), max_levels=1)
        eta = orc.ghosts(0)["eta"]
        hst, _ = np.histogram(eta, bins=10, range=(0.0, 1.0))
        frac = hst / hst.sum()
        assert np.all(frac[:7] > 0.07) and np.all(frac[:7] < 0.15)
        assert frac[9] < frac[:7].mean() / 2
        assert eta.min() < 0.01 and eta.max() > 0.95


def test_band_is_inactive_near_ghosts(oracle_mod):
    d, N = 2, 48
    orc = O.Oracle(d, N, W.phi_flower_paper(N), max_levels=1)
    cls = orc.cls(0)
    band = orc.band(0)
    gh = orc.ghosts(0)["idx"]
    n = N + 1
    gi, gj = gh % n, gh // n
    want = set()
    for i, j in zip(gi, gj):
        for a in range(-2, 3):
            for b in range(-2, 3):
                if 0 <= i + a <= N and 0 <= j + b <= N and cls[(j + b) * n + i + a] == O.INACTIVE:
                    want.add((j + b) * n + i + a)
    assert set(band.tolist()) == want
    assert np.all(np.diff(band) > 0)


def test_extension_is_constant_along_normals_halfspace(oracle_mod):
    # dr/dn = 0 in the band: for a plane boundary x = xV the upwind extension
    # copies the ghost value along +x
    N = 32
    orc = O.Oracle(2, N, W.phi_halfspace(2, N, 0.33), max_levels=1)
    g = orc.ghosts(0)
    a = np.zeros(orc.nn(0))
    rng = np.random.default_rng(0)
    a[g["idx"]] = rng.uniform(-1, 1, g["idx"].size)
    e = orc.extend(0, a)
    n = N + 1
    for b in orc.band(0):
        i, j = b % n, b // n
        # the ghost of the same row
        same = [k for k in g["idx"] if k // n == j]
        if same:
            assert e[b] == pytest.approx(a[same[0]], abs=1e-15)
