"""Pins of the oracle's transfer operators and convergence on curved domains.

* The restriction of Sec. 3.3.2 (FW where the 3^d fine neighbours all lie in
  the coarse node's class family, else the FW-weighted mean over the family)
  is recomputed here, independently, with numpy array slicing on a small disk
  and flower grid, and compared element by element.
* The extension into the inactive band is a weighted average of upwind
  values: it reproduces a constant exactly wherever it reaches.
* Rectangle of Sec. 3.2: where the boundary's ghost column is not a coarse
  grid column, the two-grid factor at Delta tau_OPT(theta) stays at the box
  value for every theta (the paper's conclusion: the BLFA prediction is
  excellent for rectangles whose boundary does not pass through grid points),
  and the numerically best constant Delta tau is close to Delta tau_OPT
  (Fig. dtau_opt).  Where the ghost column is a coarse column the factor
  degrades for theta > 0.5 (a finding, pinned as such).
* The convergence factors of the paper's Circle, Flower and ellipsoid under
  the adopted readings are pinned against ``tests/golden/rho_study.txt``
  (written by ``tests/golden/make_rho_study.py`` from the oracle alone).
"""

import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W

STUDY = os.path.join(os.path.dirname(__file__), "golden", "rho_study.txt")


def study_value(domain, reading, N):
    for line in open(STUDY):
        if line.startswith("#"):
            continue
        p = line.split()
        if p[0] == domain and p[1] == reading and int(p[2]) == N:
            return float(p[3])
    raise KeyError((domain, reading, N))


def rho_of(d, N, phi, **kw):
    orc = O.Oracle(d, N, phi, **kw)
    nn = orc.nn(0)
    orc.set_rhs(np.zeros(nn), np.zeros(orc.info(0)["n_ghost"]))
    r, _ = orc.rho(W.random_u0(nn, 3), 16)
    return r


# -------------------------------------------------- restriction, numpy check

def _restrict_numpy(cls_f, r_f, cls_c, n_f, n_c):
    """FW / family mean written with array slicing (2D), independent of the
    oracle's loops: coarse node (I, J) reads fine (2I+a, 2J+b), a, b in
    {-1, 0, 1}, with FW weight (2 - |a|)(2 - |b|) / 16."""
    cf = cls_f.reshape(n_f, n_f)
    rf = r_f.reshape(n_f, n_f)
    cc = cls_c.reshape(n_c, n_c)
    pad_c = np.pad(cf, 1, constant_values=255)  # outside the grid: no family
    pad_r = np.pad(rf, 1)
    J, I = np.meshgrid(np.arange(n_c), np.arange(n_c), indexing="ij")
    num = np.zeros((n_c, n_c))
    den = np.zeros((n_c, n_c))
    alln = np.ones((n_c, n_c), dtype=bool)
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            w = (2 - abs(a)) * (2 - abs(b)) / 16.0
            cy = pad_c[2 * J + b + 1, 2 * I + a + 1]
            ry = pad_r[2 * J + b + 1, 2 * I + a + 1]
            fam_int = cy == O.INTERIOR
            fam_gh = (cy == O.GHOST) | (cy == O.INACTIVE)
            fam = np.where(cc == O.INTERIOR, fam_int, fam_gh)
            alln &= fam
            num += np.where(fam, w * ry, 0.0)
            den += np.where(fam, w, 0.0)
    act = (cc == O.INTERIOR) | (cc == O.GHOST)
    avg = np.where(den > 0, num / np.where(den > 0, den, 1), 0.0)
    out = np.where(alln, num, avg)
    return np.where(act, out, 0.0).reshape(-1)


@pytest.mark.parametrize("N,mk", [(32, W.phi_disk), (32, W.phi_flower_paper), (48, W.phi_circle_paper)])
def test_restriction_family_average_matches_numpy(oracle_mod, N, mk):
    orc = O.Oracle(2, N, mk(N))
    assert orc.L >= 2
    rng = np.random.default_rng(11)
    cf = orc.cls(0)
    r = np.where((cf == O.INTERIOR) | (cf == O.GHOST), rng.uniform(-1, 1, cf.size), 0.0)
    r = orc.extend(0, r)  # band values as the cycle restricts them
    Fc = orc.restrict(0, r)
    ref = _restrict_numpy(cf, r, orc.cls(1), N + 1, N // 2 + 1)
    np.testing.assert_allclose(Fc, ref, rtol=1e-14, atol=1e-15)
    # the check itself is sensitive: dropping the renormalisation breaks it
    cc = orc.cls(1)
    mixed = 0
    cfm = cf.reshape(N + 1, N + 1)
    for c in np.where(cc == O.GHOST)[0]:
        J, I = divmod(c, N // 2 + 1)
        blk = cfm[max(2 * J - 1, 0):2 * J + 2, max(2 * I - 1, 0):2 * I + 2]
        mixed += int((blk == O.INTERIOR).any())
    assert mixed > 0


@pytest.mark.parametrize("mk,N", [(W.phi_disk, 64), (W.phi_flower_paper, 64)])
def test_extension_reproduces_constants(oracle_mod, mk, N):
    # each sweep is a convex combination of upwind values (band starting
    # from zero): with enough sweeps every reached band node carries the
    # constant (a concave stretch can make two band nodes each other's
    # upwind source, so the limit is geometric, not reached in K steps);
    # with the default K = 4 values stay within [0, c] and grow
    # with K
    c = 0.731
    vals = {}
    for K in (4, 64):
        orc = O.Oracle(2, N, mk(N), ext_sweeps=K)
        a = np.zeros(orc.nn(0))
        a[orc.ghosts(0)["idx"]] = c
        vals[K] = orc.extend(0, a)[orc.band(0)]
    reached = vals[64] != 0.0
    assert reached.mean() > 0.9
    np.testing.assert_allclose(vals[64][reached], c, rtol=1e-14)
    assert np.all(vals[4] >= 0.0) and np.all(vals[4] <= c * (1 + 1e-15))
    assert np.all(vals[4] <= vals[64] * (1 + 1e-15))
    assert (vals[4][reached] == vals[64][reached]).mean() > 0.4


# ----------------------------------------------------------- rectangle

@pytest.mark.parametrize("theta", [0.6, 0.7, 0.8, 0.9])
def test_rectangle_off_coarse_column_keeps_box_factor(oracle_mod, theta):
    # boundary between grid lines, ghost column at an odd index: the BLFA
    # prediction holds for every theta (Sec. 3.2 Fig. 2D_rhoD, Sec. 5)
    N = 64
    h = 2.0 / N
    xV = (-1 + (N - 3) * h) - theta * h
    r = rho_of(2, N, W.phi_halfspace(2, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS, dtau_mode=O.DT_POLY)
    r_box = rho_of(2, N, W.phi_box(2, N), ordering=O.LEX, cycle=O.CYC_TGCS)
    assert r <= r_box + 0.012, (r, r_box)


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_rectangle_numerical_optimum_near_blfa(oracle_mod, theta):
    # Fig. dtau_opt: the constant Delta tau that minimises the measured factor
    # agrees with Delta tau_OPT(theta) of eq. dtauoptLFA
    N = 64
    h = 2.0 / N
    xV = (-1 + (N - 3) * h) - theta * h
    opt = O.dtau(2, theta, O.DT_POLY)
    grid = opt * np.array([0.4, 0.6, 0.8, 0.9, 1.0, 1.1, 1.2, 1.4])
    rs = [rho_of(2, N, W.phi_halfspace(2, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS,
                 dtau_mode=O.DT_CONST, dtau_const=float(c)) for c in grid]
    best = min(rs)
    # Delta tau_OPT is within the near-optimal range, the far ends are not
    assert rs[4] <= best + 0.01, rs
    assert rs[0] > best + 0.05, rs


def test_rectangle_on_coarse_column_degrades_above_half(oracle_mod):
    # finding: with the ghost column on the coarse grid, Delta tau_OPT > 2
    # (theta > 0.6) leaves a tangentially smooth ghost-flip mode the coarse
    # correction does not remove; the factor grows with theta
    N = 64
    h = 2.0 / N
    rs = []
    for theta in (0.5, 0.7, 0.9):
        xV = (-1 + (N - 4) * h) - theta * h
        rs.append(rho_of(2, N, W.phi_halfspace(2, N, xV), ordering=O.LEX, cycle=O.CYC_TGCS,
                         dtau_mode=O.DT_POLY))
    for theta, r in zip((0.5, 0.7, 0.9), rs):
        np.testing.assert_allclose(r, study_value("rect4", str(theta), 64), atol=0.01)
    assert rs[0] < 0.12 and rs[1] > 0.15 and rs[2] > rs[1] + 0.1, rs


# --------------------------------------------- curved domains (regression)

@pytest.mark.parametrize("domain,mk,Ns", [("circle", W.phi_circle_paper, [64, 128, 256]),
                                          ("flower", W.phi_flower_paper, [64, 128, 256])])
def test_curved_factor_curve_pinned(oracle_mod, domain, mk, Ns):
    # the adopted readings' two-grid factor on the paper's domains (TGCS,
    # GS-LEX, V(2,1), Delta tau_OPT exp): no reading of the study reaches
    # the box value 0.119 here; the curve is pinned to 0.01
    for N in Ns:
        r = rho_of(2, N, mk(N), ordering=O.LEX, cycle=O.CYC_TGCS)
        np.testing.assert_allclose(r, study_value(domain, "default", N), atol=0.01)
        r_c = study_value(domain, "const1.75", N)
        assert r < r_c, (N, r, r_c)


def test_curved_factor_ellipsoid_pinned(oracle_mod):
    N = 32
    r = rho_of(3, N, W.phi_ellipsoid_paper(N), ordering=O.LEX, cycle=O.CYC_TGCS)
    np.testing.assert_allclose(r, study_value("ellipsoid", "default", N), atol=0.01)
    assert r < study_value("ellipsoid", "const1.75", N) - 0.1
