"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Discrete set-up data (classes, ghost and band lists, stencil directions and
degrees) must match exactly; floating-point results per stage and per
V-cycle within 1e-12 relative (the FP64 tolerance of the method's parity
requirement; both sides differ only in summation order and FMA rounding).
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def bcmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14208_gb300 import bcmg as B
    from paper_2207_14208_gb300 import build
    build.build()
    O.build()
    return B


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pair(B, d, N, phi, f=None, **kw):
    s = B.Solver(d, N, dev(phi), dev(f) if f is not None else None, **kw)
    okw = {}
    if "dtau_mode" in kw:
        okw["dtau_mode"] = kw["dtau_mode"]
    if "dtau_const" in kw:
        okw["dtau_const"] = kw["dtau_const"]
    o = O.Oracle(d, N, phi, **okw)
    return s, o


CASES = [
    ("disk128", 2, 128, lambda N: W.phi_disk(N)),
    ("disk144", 2, 144, lambda N: W.phi_disk(N)),
    ("flower96", 2, 96, lambda N: W.phi_flower_paper(N)),
    ("star90", 2, 90, lambda N: W.phi_star(N, 0.15, 5, 0.3)),
    ("ellipsoid72", 3, 72, lambda N: W.phi_ellipsoid(N)),
    ("spheres64", 3, 64, lambda N: W.phi_spheres(N)),
    ("halfspace_box40", 2, 40, lambda N: W.phi_halfspace(2, N, 0.37)),
    ("halfspace3d_box24", 3, 24, lambda N: W.phi_halfspace(3, N, 0.2)),
]


@pytest.mark.parametrize("name,d,N,mk", CASES, ids=[c[0] for c in CASES])
def test_setup_matches_oracle(bcmg, name, d, N, mk):
    phi = mk(N)
    s, o = pair(bcmg, d, N, phi)
    assert s.levels == o.L
    for l in range(o.L):
        gi, oi = s.info(l), o.info(l)
        for k in ["N", "nn", "n_interior", "n_ghost", "n_band", "n_boxdir", "n_clamped", "n_fallback"]:
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        np.testing.assert_array_equal(s.cls(l), o.cls(l))
        gg, og = s.ghosts(l), o.ghosts(l)
        np.testing.assert_array_equal(gg["idx"], og["idx"])
        np.testing.assert_array_equal(gg["s"], og["s"])
        np.testing.assert_array_equal(gg["q"], og["q"])
        for k in ["eta", "n", "xi", "Q"]:
            np.testing.assert_allclose(gg[k], og[k], rtol=0, atol=1e-14)
        np.testing.assert_allclose(gg["dtau"], og["dtau"], rtol=1e-13)
        np.testing.assert_array_equal(s.band(l), o.band(l))


def _rand_level(o, l, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    nn = o.info(l)["nn"]
    cls = o.cls(l)
    u = np.where(cls != O.INACTIVE, rng.uniform(-1, 1, nn), 0.0) * scale
    F = np.where((cls == O.INTERIOR) | (cls == O.GHOST), rng.uniform(-1, 1, nn), 0.0)
    return u, F, cls


@pytest.mark.parametrize("name,d,N,mk", CASES, ids=[c[0] for c in CASES])
def test_stage_operators_match_oracle(bcmg, name, d, N, mk):
    phi = mk(N)
    s, o = pair(bcmg, d, N, phi)
    for l in range(o.L):
        u, F, cls = _rand_level(o, l, 10 + l)
        act = (cls == O.INTERIOR) | (cls == O.GHOST)
        # one smoothing step
        ug = dev(u)
        s.smooth(l, ug, dev(F), 1)
        uo = o.smooth(l, u, F, 1)
        scale = np.abs(uo).max()
        assert np.abs(host(ug) - uo).max() <= REL * scale
        # residual (scale: the largest term of the rows)
        rg = torch.zeros(o.info(l)["nn"], dtype=torch.float64, device="cuda")
        s.residual(l, dev(uo), dev(F), rg)
        ro = o.residual(l, uo, F)
        h = 2.0 / o.info(l)["N"]
        rscale = np.abs(F).max() + 2 * d * np.abs(uo).max() / (h * h)
        np.testing.assert_allclose(host(rg)[act], ro[act], rtol=0, atol=REL * rscale)
        # extension of the ghost residual into the band
        ag = dev(ro)
        s.extend(l, ag)
        ao = o.extend(l, ro)
        band = o.band(l)
        np.testing.assert_allclose(host(ag)[band], ao[band], rtol=0, atol=REL * np.abs(ro).max())
        if l + 1 < o.L:
            # restriction from the same extended residual
            Fc = torch.zeros(o.info(l + 1)["nn"], dtype=torch.float64, device="cuda")
            s.restrict(l, dev(ao), Fc)
            Fo = o.restrict(l, ao)
            ca = np.isin(o.cls(l + 1), [O.INTERIOR, O.GHOST])
            np.testing.assert_allclose(host(Fc)[ca], Fo[ca], rtol=0, atol=REL * np.abs(ao).max())
            # prolongation of a coarse field onto u
            ec, _, _ = _rand_level(o, l + 1, 99 + l)
            ug2 = dev(uo)
            s.prolong(l, dev(ec), ug2)
            po = o.prolong(l, ec, uo)
            np.testing.assert_allclose(host(ug2)[act], po[act], rtol=0, atol=REL * np.abs(po).max())
        else:
            ug3 = dev(u)
            s.coarsest_solve(ug3, dev(F))
            co = o.coarsest_solve(u, F)
            np.testing.assert_allclose(host(ug3)[act], co[act], rtol=0, atol=REL * np.abs(co).max())


VCASES = [c for c in CASES if c[0] in ("disk128", "flower96", "ellipsoid72", "spheres64", "halfspace_box40")]


@pytest.mark.parametrize("name,d,N,mk", VCASES, ids=[c[0] for c in VCASES])
def test_vcycle_matches_oracle(bcmg, name, d, N, mk):
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s, o = pair(bcmg, d, N, phi, f)
    Q = o.ghosts(0)["Q"]
    g = W.g_at(d, Q)
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    np.testing.assert_allclose(host(s.ghost_points()), Q, rtol=0, atol=1e-14)
    cls = o.cls(0)
    act = (cls == O.INTERIOR) | (cls == O.GHOST)
    rng = np.random.default_rng(7)
    for u0 in [np.zeros(o.nn(0)), np.where(cls == O.BOXDIR, us, rng.uniform(-1, 1, o.nn(0)))]:
        uo = u0.copy()
        ug = dev(u0)
        for cyc in range(3):
            uo = o.vcycle(uo, 1)
            s.vcycle(ug, 1)
            got = host(ug)
            assert np.abs(got[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), cyc
            # nodes outside interior and ghosts are left untouched
            np.testing.assert_array_equal(got[~act], u0[~act])


def test_solve_and_norms_match_oracle(bcmg):
    d, N = 2, 128
    phi = W.phi_disk(N)
    f, us = W.manufactured(d, N)
    s, o = pair(bcmg, d, N, phi, f)
    g = W.g_at(d, o.ghosts(0)["Q"])
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    u0 = np.zeros(o.nn(0))
    np.testing.assert_allclose(s.residual_norm(dev(u0)), o.norms(u0), rtol=1e-13)
    ug = dev(u0)
    cyc, rel = s.solve(ug, 1e-10, 100)
    uo, co, hist = o.solve(u0, 1e-10, 100)
    assert abs(cyc - co) <= 1 and rel <= 1e-10
    act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
    if cyc == co:
        assert np.abs(host(ug)[act] - uo[act]).max() <= 1e-11 * np.abs(uo[act]).max()
    # the final residual sits near rounding level: agree to a few digits
    np.testing.assert_allclose(s.residual_norm(ug), o.norms(uo), rtol=5e-2)


def test_edge_cases(bcmg):
    B = bcmg
    # single level (N too small to coarsen): the cycle is the exact solve
    for d, N, mk in [(2, 12, W.phi_disk), (2, 75, W.phi_disk), (3, 10, W.phi_ellipsoid)]:
        phi = mk(N)
        f, us = W.manufactured(d, N)
        s, o = pair(B, d, N, phi, f)
        g = W.g_at(d, o.ghosts(0)["Q"])
        o.set_rhs(f, g)
        s.set_boundary_values(dev(g))
        assert s.levels == o.L
        ug = dev(np.zeros(o.nn(0)))
        s.vcycle(ug, 1)
        uo = o.vcycle(np.zeros(o.nn(0)), 1)
        act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
        # with a single level the cycle is a direct solve of the whole system:
        # two backward-stable solves agree to about cond(A) * eps only
        _, A, _ = o.assemble(0, np.zeros(o.nn(0)), o.F(0))
        tol = max(REL, 8 * np.linalg.cond(A) * np.finfo(float).eps)
        assert np.abs(host(ug)[act] - uo[act]).max() <= tol * np.abs(uo[act]).max()
    # no interior node -> EGEOM; bad arguments -> EINVAL
    with pytest.raises(B.BcmgError) as e:
        B.Solver(2, 16, dev(np.ones(17 * 17)))
    assert e.value.code == B.EGEOM
    with pytest.raises(B.BcmgError) as e:
        B.Solver(4, 16, dev(np.ones(17 ** 4)))
    assert e.value.code == B.EINVAL
    with pytest.raises(B.BcmgError) as e:
        B.Solver(2, 2, dev(-np.ones(9)))
    assert e.value.code == B.EINVAL
    # constant and polynomial Delta tau options reach the ghosts
    phi = W.phi_disk(64)
    for kw in [dict(dtau_mode=B.DTAU_CONST, dtau_const=1.75), dict(dtau_mode=B.DTAU_POLY)]:
        s = B.Solver(2, 64, dev(phi), **kw)
        o = O.Oracle(2, 64, phi, **kw)
        np.testing.assert_allclose(s.ghosts(0)["dtau"], o.ghosts(0)["dtau"], rtol=1e-13)


def test_nonconvergence_reported(bcmg):
    B = bcmg
    d, N = 2, 64
    phi = W.phi_disk(N)
    f, _ = W.manufactured(d, N)
    s = B.Solver(d, N, dev(phi), dev(f))
    g = W.g_at(d, host(s.ghost_points()))
    s.set_boundary_values(dev(g))
    u = dev(np.zeros((N + 1) ** 2))
    with pytest.raises(B.BcmgError) as e:
        s.solve(u, 1e-14, 2)
    assert e.value.code == B.ENOCONV
    c, rel = s.solve(u, 1e-14, 2, raise_noconv=False)
    assert c == 2 and rel > 1e-14
    # a NaN in the boundary data is reported, not propagated silently
    g[3] = np.nan
    s.set_boundary_values(dev(g))
    with pytest.raises(B.BcmgError) as e:
        s.solve(dev(np.zeros((N + 1) ** 2)), 1e-10, 5)
    assert e.value.code == B.ENONFINITE


@pytest.mark.parametrize("d,N", [(2, 32), (2, 64), (3, 16)])
def test_box_domain_without_ghosts(bcmg, d, N):
    # phi < 0 everywhere: no ghost on any level, the box edge is the
    # Dirichlet boundary (its values are taken from u); the cycle, the solve
    # (whose norms then have no ghost rows) and the box values left untouched
    B = bcmg
    phi = -np.ones((N + 1) ** d)
    f, us = W.manufactured(d, N)
    s, o = pair(B, d, N, phi, f)
    assert s.ghost_count() == 0 and o.ghosts(0)["idx"].size == 0
    o.set_rhs(f, np.zeros(0))
    cls = o.cls(0)
    box, act = cls == O.BOXDIR, cls == O.INTERIOR
    u0 = np.where(box, us, 0.0)
    ug = dev(u0)
    s.vcycle(ug, 1)
    uo = o.vcycle(u0, 1)
    assert np.abs(host(ug)[act] - uo[act]).max() <= REL * np.abs(uo[act]).max()
    np.testing.assert_array_equal(host(ug)[~act], u0[~act])
    ug = dev(u0)
    cyc, rel = s.solve(ug, 1e-10, 100)
    uo, co, _ = o.solve(u0, 1e-10, 100)
    assert abs(cyc - co) <= 1 and rel <= 1e-10
    err = np.abs(host(ug)[act] - us[act]).max()
    # second order (Sec. 4): the error against u* shrinks about fourfold per
    # halving of h; checked between the two 2D sizes
    _box_err[(d, N)] = err
    if d == 2 and (2, 32) in _box_err and (2, 64) in _box_err:
        ratio = _box_err[(2, 32)] / _box_err[(2, 64)]
        assert 3.0 < ratio < 5.0, ratio


_box_err = {}


# mid-size 3D cases (more than 2^18 interior nodes on the finest level), two
# V-cycles from a random start
MCASES = [("ellipsoid176", 3, 176, W.phi_ellipsoid), ("spheres192", 3, 192, W.phi_spheres)]


@pytest.mark.parametrize("name,d,N,mk", MCASES, ids=[c[0] for c in MCASES])
def test_midsize_vcycles_match_oracle(bcmg, name, d, N, mk):
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s, o = pair(bcmg, d, N, phi, f)
    assert s.info(0)["n_interior"] >= 1 << 18
    Q = o.ghosts(0)["Q"]
    g = W.g_at(d, Q)
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    cls = o.cls(0)
    act = (cls == O.INTERIOR) | (cls == O.GHOST)
    rng = np.random.default_rng(11)
    u0 = np.where(cls == O.BOXDIR, us, rng.uniform(-1, 1, o.nn(0)))
    uo = u0.copy()
    ug = dev(u0)
    for cyc in range(2):
        uo = o.vcycle(uo, 1)
        s.vcycle(ug, 1)
        got = host(ug)
        assert np.abs(got[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), cyc
        np.testing.assert_array_equal(got[~act], u0[~act])


@pytest.mark.slow
def test_full_size_ellipsoid_256(bcmg):
    """The benchmark workload (3D ellipsoid, N = 256, V(2,1), FP64): set-up
    identical to the oracle's, one V-cycle within 1e-12 of the oracle's, and
    the solve reaches 1e-10 with the discretisation error of the oracle."""
    d, N = 3, 256
    phi = W.phi_ellipsoid(N)
    f, us = W.manufactured(d, N)
    s, o = pair(bcmg, d, N, phi, f)
    for l in range(o.L):
        np.testing.assert_array_equal(s.cls(l), o.cls(l))
        np.testing.assert_array_equal(s.ghosts(l)["idx"], o.ghosts(l)["idx"])
    Q = o.ghosts(0)["Q"]
    g = W.g_at(d, Q)
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
    ug = dev(np.zeros(o.nn(0)))
    s.vcycle(ug, 1)
    uo = o.vcycle(np.zeros(o.nn(0)), 1)
    assert np.abs(host(ug)[act] - uo[act]).max() <= REL * np.abs(uo[act]).max()
    ug = dev(np.zeros(o.nn(0)))
    cyc, rel = s.solve(ug, 1e-10, 60)
    assert rel <= 1e-10 and cyc <= 30
    interior = o.cls(0) == O.INTERIOR
    err = np.abs(host(ug) - us)[interior].max()
    assert err < 5e-5


@pytest.mark.parametrize("name,d,N,mk", [("disk128", 2, 128, W.phi_disk), ("ellipsoid48", 3, 48, W.phi_ellipsoid),
                                         ("flower96", 2, 96, W.phi_flower_paper)],
                         ids=["disk128", "ellipsoid48", "flower96"])
def test_wcycle_matches_oracle(bcmg, name, d, N, mk):
    # W-cycle (gamma = 2, Sec. 2.1): every coarse level visited twice per
    # visit of the level above (the grid path and the cluster tail alike)
    B = bcmg
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s = B.Solver(d, N, dev(phi), dev(f), cycle=B.CYCLE_W)
    o = O.Oracle(d, N, phi, cycle=O.CYC_W)
    g = W.g_at(d, o.ghosts(0)["Q"])
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
    uo = np.zeros(o.nn(0))
    ug = dev(uo)
    for cyc in range(3):
        uo = o.vcycle(uo, 1)
        s.vcycle(ug, 1)
        assert np.abs(host(ug)[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), cyc
    c, rel = s.solve(dev(np.zeros(o.nn(0))), 1e-10, 60)
    assert rel <= 1e-10


@pytest.mark.parametrize("name,d,N,mk", [("disk128", 2, 128, W.phi_disk), ("ellipsoid48", 3, 48, W.phi_ellipsoid),
                                         ("flower96", 2, 96, W.phi_flower_paper)],
                         ids=["disk128", "ellipsoid48", "flower96"])
def test_tgcs_matches_oracle(bcmg, name, d, N, mk):
    # two-grid correction scheme (Sec. 2.1): the level-1 problem solved by K
    # V-cycles from zero (the grid path and the cluster tail below level 1);
    # the oracle's TGCS with tolerance 0 runs exactly K
    B = bcmg
    K = 12
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s = B.Solver(d, N, dev(phi), dev(f), cycle=B.CYCLE_TG, tg_inner=K)
    o = O.Oracle(d, N, phi, cycle=O.CYC_TGCS, tgcs_tol=0.0, tgcs_maxit=K)
    assert s.levels == o.L > 2
    g = W.g_at(d, o.ghosts(0)["Q"])
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
    uo = np.zeros(o.nn(0))
    ug = dev(uo)
    for cyc in range(3):
        uo = o.vcycle(uo, 1)
        s.vcycle(ug, 1)
        assert np.abs(host(ug)[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), cyc
    c, rel = s.solve(dev(np.zeros(o.nn(0))), 1e-10, 60)
    assert rel <= 1e-10
    cv, _ = B.Solver(d, N, dev(phi), dev(f)).solve(dev(np.zeros(o.nn(0))), 1e-10, 60)
    assert c <= cv  # an exact coarse solve needs no more cycles than the V-cycle


def test_tgcs_rho_harness_matches_oracle(bcmg):
    from paper_2207_14208_gb300 import repro
    N = 64
    phi = W.phi_circle_paper(N)
    r_gpu = repro.rho(2, N, phi, cycle=bcmg.CYCLE_TG, tg_inner=30)
    o = O.Oracle(2, N, phi, cycle=O.CYC_TGCS, tgcs_tol=0.0, tgcs_maxit=30)
    r_orc, _ = o.rho(np.random.Generator(np.random.PCG64(3)).uniform(-1.0, 1.0, (N + 1) ** 2))
    assert r_gpu == pytest.approx(r_orc, rel=1e-6)


def test_rho_harness_matches_oracle(bcmg):
    # the reproduction harness's rho (Sec. 2.2 protocol) against the oracle's
    from paper_2207_14208_gb300 import repro
    N = 64
    phi = W.phi_circle_paper(N)
    r_gpu = repro.rho(2, N, phi)
    r_orc, _ = O.Oracle(2, N, phi).rho(np.random.Generator(np.random.PCG64(3)).uniform(-1.0, 1.0, (N + 1) ** 2))
    assert r_gpu == pytest.approx(r_orc, rel=1e-6)


@pytest.mark.parametrize("name,d,N,mk", [("disk64", 2, 64, W.phi_disk), ("flower48", 2, 48, W.phi_flower_paper),
                                         ("ellipsoid24", 3, 24, W.phi_ellipsoid)],
                         ids=["disk64", "flower48", "ellipsoid24"])
def test_gslex_matches_oracle(bcmg, name, d, N, mk):
    # the paper's GS-LEX interior order (eq. GSLEX_2D), run on the GPU as a
    # sweep over the hyperplanes i + j (+ k) = p, against the oracle's
    # lexicographic loop
    B = bcmg
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s = B.Solver(d, N, dev(phi), dev(f), ordering=B.ORDER_LEX)
    o = O.Oracle(d, N, phi, ordering=O.LEX)
    g = W.g_at(d, o.ghosts(0)["Q"])
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
    uo = np.where(o.cls(0) == O.BOXDIR, us, 0.0)
    ug = dev(uo)
    for cyc in range(3):
        uo = o.vcycle(uo, 1)
        s.vcycle(ug, 1)
        assert np.abs(host(ug)[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), cyc
