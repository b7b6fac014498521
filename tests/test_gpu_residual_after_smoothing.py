"""The cycle's residual right after a red-black smoothing step.

After the black sweep every black interior row holds its own equation
solved from the red values (eq. GSLEX_2D in red-black order), and the ghost
relaxation that ends the smoothing step (eq. rel) changes only ghost
values.  So a black row whose neighbours are all interior has a zero
residual up to the sweep's rounding, and the cycle's residual (before the restriction) and
the solve's per-cycle norm store zero there without computing it.  These
tests check that the norm a solve reports equals the full residual norm of
the u it returns, to rounding, on domains whose black rows do and do not
touch the box edge and for the smoothing counts that decide whether the
shortcut applies; the V-cycle parity tests cover the restriction."""

import numpy as np
import pytest

from paper_2207_14208_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bcmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14208_gb300 import bcmg as B
    from paper_2207_14208_gb300 import build
    build.build()
    return B


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _norm(n4):
    return float(np.hypot(n4[0], n4[1]))


CASES = [("ellipsoid64", 3, 64, W.phi_ellipsoid, {}),
         ("flower128", 2, 128, W.phi_flower_paper, {}),
         ("halfspace96", 2, 96, lambda N: W.phi_halfspace(2, N, 0.37), {}),
         ("disk128_v11", 2, 128, W.phi_disk, {"nu1": 1, "nu2": 1}),
         ("disk128_v20", 2, 128, W.phi_disk, {"nu1": 2, "nu2": 0}),
         ("disk128_v02", 2, 128, W.phi_disk, {"nu1": 0, "nu2": 2}),
         ("flower96_neumann", 2, 96, W.phi_flower_paper, {"bc": 1, "reaction": 1.0}),
         ("ellipsoid48_w", 3, 48, W.phi_ellipsoid, {"cycle": 1})]


@pytest.mark.parametrize("name,d,N,mk,kw", CASES, ids=[c[0] for c in CASES])
def test_reported_norm_equals_full_residual(bcmg, name, d, N, mk, kw):
    B = bcmg
    f, _ = W.manufactured(d, N)
    s = B.Solver(d, N, dev(mk(N)), dev(f), **kw)
    Q = s.ghost_points().cpu().numpy()
    s.set_boundary_values(dev(W.g_at(d, Q)))
    u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
    r0 = _norm(s.residual_norm(u))
    assert r0 > 0.0
    for ncyc in (1, 3, 8):
        u.zero_()
        c, rel = s.solve(u, 0.0, ncyc, raise_noconv=False)
        torch.cuda.synchronize()
        assert c == ncyc
        full = _norm(s.residual_norm(u)) / r0
        # the skipped rows' true residual is the sweep's rounding: far below
        # the cycle's residual at these counts
        assert rel == pytest.approx(full, rel=1e-6, abs=1e-15), (ncyc, rel, full)
    s.close()


def _expected_lists(cls, d, n, B):
    c = cls.reshape((n,) * d)
    inter = c == B.INTERIOR
    idx = np.indices(c.shape).sum(axis=0)
    red = inter & (idx % 2 == 0)
    black = inter & (idx % 2 == 1)
    near = np.zeros_like(black)
    for a in range(d):
        for sh in (-1, 1):
            # interior nodes are off the box edge, so no shift wraps for them
            near |= ~np.roll(inter, sh, axis=a)
    return int(red.sum()), int((black & near).sum()), int((black & ~near).sum())


@pytest.mark.parametrize("name,d,N,mk", [("ellipsoid64", 3, 64, W.phi_ellipsoid),
                                          ("spheres64", 3, 64, W.phi_spheres),
                                          ("flower128", 2, 128, W.phi_flower_paper),
                                          ("halfspace96", 2, 96, lambda N: W.phi_halfspace(2, N, 0.37)),
                                          ("box3d", 3, 32, lambda N: -np.ones((N + 1) ** 3))])
def test_list_split_matches_classes(bcmg, name, d, N, mk):
    # red / black next to a ghost or box-edge node / other black, counted
    # from the classes
    B = bcmg
    s = B.Solver(d, N, dev(mk(N)), None)
    for l in range(s._num_levels()):
        n = s.info(l)["n"]
        got = s.lists(l)
        want = _expected_lists(s.cls(l), d, n, B)
        assert (got["red"], got["black_near"], got["black_inner"]) == want, (l, got, want)
        assert sum(want) == s.info(l)["n_interior"]
    with pytest.raises(B.BcmgError) as e:
        s.lists(s._num_levels())
    assert e.value.code == B.EINVAL
    s.close()
