"""Serving loop: requests of different sizes, geometries and precisions
arrive over time, are admitted by estimated footprint and overlap on the
device; each result must be the same as the same request solved alone
(bit for bit: the solves are independent and the kernels deterministic)."""

import math

import numpy as np
import pytest

from paper_2207_14208_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14208_gb300 import bcmg as B
    from paper_2207_14208_gb300 import build, serve
    build.build()
    return B, serve


def g2(Q):
    x, y = Q[:, 0], Q[:, 1]
    return torch.sin(math.pi * x) * torch.cos(math.pi * y) * torch.exp(x)


def g3(Q):
    x, y, z = Q[:, 0], Q[:, 1], Q[:, 2]
    return torch.exp(x + y + z) * torch.sin(math.pi * z)


def _requests(B, S):
    rng = np.random.Generator(np.random.PCG64(2))
    reqs, t = [], 0.0
    stars = [p for p in W.star_params(64, 1) if p[0] <= 256][:6]
    for i, (N, a, k, psi) in enumerate(stars):
        t += rng.exponential(0.002)
        reqs.append(S.Request(len(reqs), 2, N, W.phi_star(N, a, k, psi), W.manufactured(2, N)[0], g2,
                              precision=B.PREC_MIXED if i % 2 else B.PREC_FP64, arrival=t, keep_u=True))
    for i, N in enumerate([32, 48, 64]):
        t += rng.exponential(0.002)
        reqs.append(S.Request(len(reqs), 3, N, W.phi_ellipsoid(N), W.manufactured(3, N)[0], g3,
                              precision=B.PREC_FP64 if i % 2 else B.PREC_MIXED, arrival=t, keep_u=True))
    return reqs


def test_served_results_equal_alone(mods):
    B, S = mods
    reqs = _requests(B, S)
    est = sorted(B.footprint_estimate(r.dim, r.N, precision=r.precision) for r in reqs)
    budget = sum(est[-3:])  # at most a few large requests at once: admission must wait
    res = S.Server(budget, workers=4).run(reqs)
    assert sorted(r.rid for r in res) == [r.rid for r in reqs]
    by = {r.rid: r for r in res}
    for q in reqs:
        r = by[q.rid]
        assert r.status == B.OK and r.rel <= q.rtol and r.done >= r.start >= r.arrival - 1e-6
        c, rel, st, fp, u = S.solve_one(q)
        assert (c, rel, st) == (r.cycles, r.rel, r.status) and fp == r.footprint
        np.testing.assert_array_equal(u, r.u)
    lat = S.percentiles([r.latency for r in res])
    assert 0 < lat[50] <= lat[99]
