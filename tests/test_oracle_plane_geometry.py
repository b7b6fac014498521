"""Pins of the oracle's ghost geometry against a closed form (Sec. 3.3).

For a plane phi = a . x + c the grid values are samples of a linear function,
so the multilinear interpolant the projection searches is phi itself and the
central-difference gradient is exact.  Every ghost G then has (Sec. 3.3):

* outward normal n = a / |a|;
* distance to the boundary along -n, in units of h, eta = phi(G) / (h |a|),
  which lies in [0, 1] because a ghost has an interior axis neighbour;
* projection point Q = G - eta h n on the plane (phi(Q) = 0);
* stencil offsets xi_a = s_a eta n_a with s_a the upwind direction of axis a
  (the sign of n_a, reversed only where the far stencil node would leave the
  grid).

A sign, scaling or bisection-direction mistake in the oracle's ghost set-up
fails one of these; the values are independent of the oracle's code.
"""

import numpy as np
import pytest

from paper_2207_14208_gb300 import workloads as W


def _planes(d, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        a = rng.normal(size=d)
        a /= np.linalg.norm(a)
        a *= rng.uniform(0.5, 2.0)  # |a| != 1: phi is not a distance
        c = rng.uniform(-0.4, 0.4)
        out.append((a, c))
    return out


@pytest.mark.parametrize("d,N", [(2, 32), (2, 48), (3, 16)])
def test_plane_ghost_geometry_closed_form(oracle_mod, d, N):
    O = oracle_mod.oracle
    h = 2.0 / N
    X = W.coords(d, N)
    for a, c in _planes(d, 4, 11 + d + N):
        phi = sum(a[k] * X[k] for k in range(d)).reshape(-1) + c
        o = O.Oracle(d, N, phi)
        gh = o.ghosts(0)
        idx = gh["idx"]
        assert len(idx) > 0
        pts = np.stack([X[k].reshape(-1)[idx] for k in range(d)], axis=1)
        phiG = pts @ a + c
        na = np.linalg.norm(a)
        # normal
        np.testing.assert_allclose(gh["n"], np.tile(a / na, (len(idx), 1)), rtol=0, atol=1e-13)
        # distance along the normal, in units of h
        eta = phiG / (h * na)
        assert np.all(eta >= -1e-14) and np.all(eta <= 1.0 + 1e-14)
        np.testing.assert_allclose(gh["eta"], eta, rtol=0, atol=1e-12)
        # the projection point lies on the plane, eta h from G along -n
        Q = gh["Q"]
        np.testing.assert_allclose(Q @ a + c, 0.0, rtol=0, atol=1e-12)
        np.testing.assert_allclose(Q, pts - (eta * h)[:, None] * (a / na)[None, :], rtol=0, atol=1e-12)
        # stencil offsets from the upwind directions
        s = gh["s"].astype(np.float64)
        np.testing.assert_allclose(gh["xi"], s * eta[:, None] * (a / na)[None, :], rtol=0, atol=1e-12)

