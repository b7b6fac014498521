"""Mixed precision on the GPU: FP32 V-cycles on the correction inside FP64
iterative refinement (FP64 residual and update).  The refined solution must
match the FP64 solve to 1e-10 and keep the FP64 discretisation error."""

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


def _solve(B, d, N, mk, precision, rtol):
    phi = mk(N)
    f, us = W.manufactured(d, N)
    s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), precision=precision)
    g = W.g_at(d, s.ghost_points().cpu().numpy())
    s.set_boundary_values(torch.from_numpy(g).cuda())
    u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
    cyc, rel = s.solve(u, rtol, 200)
    torch.cuda.synchronize()
    return s, u.cpu().numpy(), us, cyc, rel


CASES = [("disk128", 2, 128, W.phi_disk), ("flower96", 2, 96, W.phi_flower_paper),
         ("ellipsoid64", 3, 64, W.phi_ellipsoid), ("ellipsoid48", 3, 48, W.phi_ellipsoid)]


@pytest.mark.parametrize("name,d,N,mk", CASES, ids=[c[0] for c in CASES])
def test_mixed_matches_fp64_solution(bcmg, name, d, N, mk):
    B = bcmg
    s64, u64, us, c64, r64 = _solve(B, d, N, mk, B.PREC_FP64, 1e-13)
    s32, u32, _, c32, r32 = _solve(B, d, N, mk, B.PREC_MIXED, 1e-13)
    act = np.isin(s64.cls(0), [B.INTERIOR, B.GHOST])
    assert r64 <= 1e-13 and r32 <= 1e-13
    assert np.abs(u32[act] - u64[act]).max() <= 1e-10 * np.abs(u64[act]).max()
    # the refinement converges at the rate of the FP32 cycle (a few more steps at most)
    assert c32 <= c64 + 3


# ellipsoid176: a mid-size 3D case (more than 2^18 interior nodes)
@pytest.mark.parametrize("name,d,N,mk", CASES[:1] + CASES[2:3] + [("ellipsoid176", 3, 176, W.phi_ellipsoid)],
                         ids=["disk128", "ellipsoid64", "ellipsoid176"])
def test_mixed_keeps_discretisation_error(bcmg, name, d, N, mk):
    B = bcmg
    s64, u64, us, c64, _ = _solve(B, d, N, mk, B.PREC_FP64, 1e-10)
    s32, u32, _, c32, _ = _solve(B, d, N, mk, B.PREC_MIXED, 1e-10)
    interior = s64.cls(0) == B.INTERIOR
    e64 = np.abs(u64 - us)[interior].max()
    e32 = np.abs(u32 - us)[interior].max()
    assert abs(e32 - e64) <= 0.01 * e64


def test_mixed_vcycle_tracks_fp64_cycles(bcmg):
    # bcmg_vcycle in mixed precision: each call is one refinement step; after
    # 3 and 8 steps the residual is where 3 and 8 FP64 V-cycles put it
    B = bcmg
    d, N = 2, 64
    phi = W.phi_disk(N)
    f, _ = W.manufactured(d, N)
    res = {}
    for prec in (B.PREC_FP64, B.PREC_MIXED):
        s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), precision=prec)
        g = W.g_at(d, s.ghost_points().cpu().numpy())
        s.set_boundary_values(torch.from_numpy(g).cuda())
        u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        s.vcycle(u, 3)
        r3 = np.hypot(*s.residual_norm(u)[:2])
        s.vcycle(u, 5)
        r8 = np.hypot(*s.residual_norm(u)[:2])
        res[prec] = (r3, r8)
    for k in range(2):
        assert res[B.PREC_MIXED][k] <= 1.5 * res[B.PREC_FP64][k] + 1e-12
