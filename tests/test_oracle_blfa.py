"""Pins of the oracle's Boundary Local Fourier Analysis pieces (CPU only).

Each test checks the oracle against something other than its own formula:
brute-force minimax searches over the frequency ranges of the paper's
definitions (eqs. def_dtau_opt, def_dtau_opt3D), polynomial interpolation
done independently with numpy, and the GS limit stated after eq. relghostdt.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O


def _lagrange_interp_at(theta, values):
    """Quadratic through (0, v0), (1, v1), (2, v2) evaluated at theta (numpy)."""
    coef = np.polyfit([0.0, 1.0, 2.0], values, 2)
    return float(np.polyval(coef, theta))


@pytest.mark.parametrize("theta", [0.0, 0.13, 0.5, 0.77, 0.99])
@pytest.mark.parametrize("p", [0.3, math.acosh(2.0), math.acosh(3.0), math.acosh(5.0)])
def test_poly_G0_is_quadratic_interpolant_of_exponential(oracle_mod, theta, p):
    # Remark exptheta2D: eq. G is the quadratic interpolation of exp(-p x) on
    # the nodes 0, 1, 2 evaluated at theta (coefficients eq. coeff are the
    # Lagrange basis).  Check against numpy's own interpolation.
    t = math.exp(-p)
    want = _lagrange_interp_at(theta, [1.0, t, t * t])
    assert O.blfa_G0(0, 1, p, theta) == pytest.approx(want, rel=1e-12, abs=1e-14)
    # Neumann eq. GN: derivative of the same interpolant of exp(p x) at the
    # boundary, i.e. a quadratic in theta.  Derivative of the interpolant of
    # v_k = exp(-p k) taken in the direction away from the domain.
    coef = np.polyfit([0.0, 1.0, 2.0], [1.0, t, t * t], 2)
    d = -float(np.polyval(np.polyder(coef), theta))
    assert O.blfa_G0(1, 1, p, theta) == pytest.approx(d, rel=1e-12, abs=1e-13)


def test_exp_G0_agrees_with_poly_at_nodes(oracle_mod):
    # the exp form (Remark exptheta2D) coincides with eq. G at theta = 0 and 1
    for p in [0.5, 1.3, 2.2]:
        for th in [0.0, 1.0]:
            assert O.blfa_G0(0, 0, p, th) == pytest.approx(O.blfa_G0(0, 1, p, th), rel=1e-13)


def _brute_dtau(G0_of_alpha, thetas, dts):
    out = []
    for th in thetas:
        g0 = np.array([G0_of_alpha(a, th) for a in G0_of_alpha.alphas])
        worst = np.max(np.abs(1.0 - np.outer(dts, g0)), axis=1)
        out.append(dts[np.argmin(worst)])
    return np.array(out)


@pytest.mark.parametrize("form", [0, 1])
def test_dtau_opt_2d_equals_bruteforce_minimax(oracle_mod, form):
    # eq. def_dtau_opt: argmin over dtau of sup_{pi/2<alpha<pi} |1 - dtau G0|
    alphas = np.linspace(math.pi / 2, math.pi, 1201)
    dts = np.linspace(0.5, 6.0, 55001)
    thetas = [0.0, 0.2, 0.45, 0.7, 0.95]

    def g0(alpha, th):
        return O.blfa_G0(0, form, O.blfa_p(2, [alpha]), th)

    g0.alphas = alphas
    brute = _brute_dtau(g0, thetas, dts)
    mode = O.DT_EXP if form == 0 else O.DT_POLY
    formula = np.array([O.dtau(2, th, mode) for th in thetas])
    np.testing.assert_allclose(formula, brute, rtol=2e-4, atol=2e-4)


@pytest.mark.parametrize("form", [0, 1])
def test_dtau_opt_3d_equals_bruteforce_minimax(oracle_mod, form):
    # eq. def_dtau_opt3D: sup over HIGH = [0,pi]^2 minus [0,pi/2]^2
    a = np.linspace(0.0, math.pi, 81)
    A1, A2 = np.meshgrid(a, a)
    high = np.maximum(A1, A2) >= math.pi / 2
    pts = np.stack([A1[high], A2[high]], axis=1)
    dts = np.linspace(0.5, 7.0, 6501)
    for th in [0.0, 0.3, 0.6, 0.9]:
        g0 = np.array([O.blfa_G0(0, form, O.blfa_p(3, pt), th) for pt in pts])
        worst = np.max(np.abs(1.0 - np.outer(dts, g0)), axis=1)
        brute = dts[np.argmin(worst)]
        mode = O.DT_EXP if form == 0 else O.DT_POLY
        assert O.dtau(3, th, mode) == pytest.approx(brute, rel=1.5e-3, abs=1.5e-3)


def test_dtau_opt_neumann_2d_bruteforce(oracle_mod):
    # Prop. 2 (eq. dtauoptLFA_Neumann): Dtau/h from the same minimax with eq. GN
    alphas = np.linspace(math.pi / 2, math.pi, 1201)
    dts = np.linspace(0.2, 4.0, 38001)
    for th in [0.0, 0.5, 0.9]:
        g0 = np.array([O.blfa_G0(1, 1, O.blfa_p(2, [al]), th) for al in alphas])
        worst = np.max(np.abs(1.0 - np.outer(dts, g0)), axis=1)
        assert O.dtau(2, th, O.DT_POLY, bc=1) == pytest.approx(dts[np.argmin(worst)], rel=3e-4, abs=3e-4)


@pytest.mark.parametrize("d", [2, 3])
def test_dtau_zero_distance_is_gauss_seidel(oracle_mod, d):
    # after eq. relghostdt: dtau = 1/c_0 reverts to Gauss-Seidel; at theta = 0
    # c_0 = 1 and Delta tau_OPT(0) must be 1 in both forms.
    for mode in (O.DT_EXP, O.DT_POLY):
        assert O.dtau(d, 0.0, mode) == pytest.approx(1.0, rel=1e-14)


def test_G0_positive_and_monotone_in_alpha(oracle_mod):
    # Lemmas fnostat / G0pos (and their 3D versions): G0 > 0 for theta in [0,1)
    # and no stationary point in alpha on (pi/2, pi) -> monotone there.
    alphas = np.linspace(math.pi / 2 + 1e-3, math.pi - 1e-3, 400)
    # theta = 0 gives G0 = c_0 = 1 for every alpha (constant), so the open
    # interval (0, 1) is checked
    for th in np.linspace(0.01, 0.999, 41):
        g = np.array([O.blfa_G0(0, 1, O.blfa_p(2, [a]), th) for a in alphas])
        assert np.all(g > 0)
        dg = np.diff(g)
        assert np.all(dg < 0) or np.all(dg > 0)


def test_continuous_p_gives_wrong_dtau(oracle_mod):
    # Remark solnum2D: using p(alpha) = alpha (continuous solution) changes the
    # optimum by O(1); negative control on the discrete p of eq. alphaNalpha.
    th = 0.6
    disc = O.dtau(2, th, O.DT_POLY)
    cont = 2.0 / (O.blfa_G0(0, 1, math.pi / 2, th) + O.blfa_G0(0, 1, math.pi, th))
    assert abs(disc - cont) / disc > 0.1


def test_discrete_p_closed_form(oracle_mod):
    # eq. alphaNalpha at the corner frequencies: e^{-p} = a - sqrt(a^2-1)
    for d, al, a in [(2, [math.pi / 2], 2.0), (2, [math.pi], 3.0),
                     (3, [math.pi / 2, 0.0], 2.0), (3, [math.pi / 2, math.pi / 2], 3.0),
                     (3, [math.pi, math.pi], 5.0)]:
        assert math.exp(-O.blfa_p(d, al)) == pytest.approx(a - math.sqrt(a * a - 1), rel=1e-13)
