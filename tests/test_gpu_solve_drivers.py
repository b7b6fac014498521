"""The three ways bcmg_solve can drive its cycles give the same answer:
the whole solve as one graph (a WHILE conditional node with the
convergence check on the device), a host loop over captured cycle graphs
(used when sweeps are profiled), and plain launches without graphs.  They
run the same kernels in the same order, so u and the cycle count agree
exactly; the stopping rule (stop once ||r|| / ||r0|| <= rtol, Sec. 4) and
the max_cycles limit behave alike."""

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


def _run(B, d, N, mk, rtol, max_cycles, zero_rhs=False, **kw):
    phi = mk(N)
    f, _ = W.manufactured(d, N)
    if zero_rhs:
        f = np.zeros_like(f)
    s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), **kw)
    g = W.g_at(d, s.ghost_points().cpu().numpy())
    if zero_rhs:
        g = np.zeros_like(g)
    s.set_boundary_values(torch.from_numpy(g).cuda())
    u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
    c, rel = s.solve(u, rtol, max_cycles, raise_noconv=False)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    s.close()
    return c, rel, out


DRIVERS = [dict(), dict(profile=1), dict(use_graph=0)]
CASES = [("disk128", 2, 128, W.phi_disk), ("ellipsoid48", 3, 48, W.phi_ellipsoid)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,d,N,mk", CASES, ids=[c[0] for c in CASES])
def test_drivers_agree(bcmg, name, d, N, mk, prec):
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    res = [_run(B, d, N, mk, 1e-10, 100, precision=p, **kw) for kw in DRIVERS]
    c0, r0, u0 = res[0]
    assert r0 <= 1e-10 and c0 > 3
    for c, rel, u in res[1:]:
        assert c == c0 and rel == r0
        np.testing.assert_array_equal(u, u0)


def test_cycle_limit_and_zero_residual(bcmg):
    B = bcmg
    for kw in DRIVERS:
        # the limit stops the loop after exactly max_cycles cycles
        c, rel, _ = _run(B, 2, 64, W.phi_disk, 1e-14, 3, **kw)
        assert c == 3 and 0.0 < rel < 1.0
        c, rel, _ = _run(B, 2, 64, W.phi_disk, 1e-10, 0, **kw)
        assert c == 0 and rel == 1.0
        # zero data: r0 = 0, nothing to do
        c, rel, u = _run(B, 2, 64, W.phi_disk, 1e-10, 50, zero_rhs=True, **kw)
        assert c == 0 and rel == 0.0 and not u.any()
