"""GPU parity at the grid sizes the batched and served workloads run.

2D star and disk domains up to N = 2048 (the served stream's largest 2D
request) and N = 960 (a batched-workload size, m 2^k with m = 15, whose
coarsening stops at the odd N = 15), and 3D ellipsoids whose level sizes are
not powers of two (N = 320 down to 10, N = 336 down to the odd 21): set-up
identical to the oracle's on every level, then V-cycles from zero and from a
random start within 1e-12 of the oracle's, and the mixed-precision solve on
the FP64 solution to 1e-10 (both solved to a relative residual of 1e-10).
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


def _star960():
    # the first batched-workload star whose N is 960
    for N, a, k, psi in W.star_params():
        if N == 960:
            return lambda n: W.phi_star(n, a, k, psi)
    return lambda n: W.phi_star(n, 0.12, 7, 1.1)


CASES = [
    ("disk1024", 2, 1024, W.phi_disk),
    ("star2048", 2, 2048, lambda N: W.phi_star(N, 0.15, 5, 0.3)),
    ("star960", 2, 960, _star960()),
    ("ellipsoid320", 3, 320, W.phi_ellipsoid),
    ("ellipsoid336", 3, 336, W.phi_ellipsoid),
]


@pytest.mark.parametrize("name,d,N,mk", CASES, ids=[c[0] for c in CASES])
def test_large_setup_and_vcycles_match_oracle(bcmg, name, d, N, mk):
    B = bcmg
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s = B.Solver(d, N, dev(phi), dev(f))
    o = O.Oracle(d, N, phi)
    assert s.levels == o.L
    for l in range(o.L):
        gi, oi = s.info(l), o.info(l)
        for k in ["N", "n_interior", "n_ghost", "n_band", "n_boxdir", "n_fallback"]:
            assert gi[k] == oi[k], (l, k, gi[k], oi[k])
        np.testing.assert_array_equal(s.cls(l), o.cls(l))
        np.testing.assert_array_equal(s.ghosts(l)["idx"], o.ghosts(l)["idx"])
        np.testing.assert_array_equal(s.band(l), o.band(l))
    Q = o.ghosts(0)["Q"]
    g = W.g_at(d, Q)
    o.set_rhs(f, g)
    s.set_boundary_values(dev(g))
    cls = o.cls(0)
    act = (cls == O.INTERIOR) | (cls == O.GHOST)
    rng = np.random.default_rng(21)
    starts = [np.zeros(o.nn(0)), np.where(cls == O.BOXDIR, us, rng.uniform(-1, 1, o.nn(0)))]
    for u0 in starts:
        uo = u0.copy()
        ug = dev(u0)
        for cyc in range(2):
            uo = o.vcycle(uo, 1)
            s.vcycle(ug, 1)
            got = host(ug)
            assert np.abs(got[act] - uo[act]).max() <= REL * np.abs(uo[act]).max(), (cyc,)
            np.testing.assert_array_equal(got[~act], u0[~act])


@pytest.mark.parametrize("name,d,N,mk", [CASES[1], CASES[3]], ids=["star2048", "ellipsoid320"])
def test_large_mixed_matches_fp64(bcmg, name, d, N, mk):
    B = bcmg
    phi = mk(N)
    f, us = W.manufactured(d, N)
    out = {}
    for prec in (B.PREC_FP64, B.PREC_MIXED):
        s = B.Solver(d, N, dev(phi), dev(f), precision=prec)
        g = W.g_at(d, host(s.ghost_points()))
        s.set_boundary_values(dev(g))
        u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        # 1e-10 is the workloads' tolerance; far below it the FP64 residual of
        # these grids reaches its rounding floor (rows of size 2d |u| / h^2)
        c, rel = s.solve(u, 1e-10, 100)
        assert rel <= 1e-10
        out[prec] = (host(u), c, s.cls(0))
    u64, c64, cls = out[B.PREC_FP64]
    u32, c32, _ = out[B.PREC_MIXED]
    act = np.isin(cls, [B.INTERIOR, B.GHOST])
    assert np.abs(u32[act] - u64[act]).max() <= 1e-10 * np.abs(u64[act]).max()
    assert c32 <= c64 + 3
