"""Why the V-cycle diverges on the union of 64 seeded spheres at coarse
resolution (the 512^3 sphere-union workload): with the interior held at
zero, one ghost relaxation (eq. rel) maps the ghost values v to
(I - Dtau B_GG) v, B_GG the ghost-to-ghost block of the boundary rows
(eq. BCh).  On the sphere union at N = 64 that block has eigenvalues with
negative real part, so the map grows for every Delta tau > 0 -- small
constant steps as well as Delta tau_OPT(theta~) -- while on the ellipsoid
it contracts.  The iteration is the oracle's own ghost relaxation, repeated.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2207_14208_gb300 import workloads as W


def ghost_block_growth(phi, N, iters=150, **kw):
    o = O.Oracle(3, N, phi, max_levels=1, **kw)
    cls = o.cls(0)
    gi = o.ghosts(0)["idx"]
    F = np.zeros(o.nn(0))
    rng = np.random.default_rng(4)
    u = np.zeros(o.nn(0))
    u[gi] = rng.uniform(-1, 1, gi.size)
    rates = []
    for _ in range(iters):
        u = o.ghost_relax(0, u, F)
        u[cls == O.INTERIOR] = 0.0  # the interior held at zero
        nrm = np.linalg.norm(u[gi])
        rates.append(nrm)
        u[gi] /= nrm
    return float(np.mean(rates[-20:]))


@pytest.mark.slow
def test_sphere_union_ghost_block_unstable_for_any_step(oracle_mod):
    N = 64
    phi = W.phi_spheres(N)
    # Delta tau_OPT(theta~) (exp form), and two small constant steps: all grow
    assert ghost_block_growth(phi, N) > 2.0
    for dt in (0.5, 0.1):
        g = ghost_block_growth(phi, N, dtau_mode=O.DT_CONST, dtau_const=dt, iters=400)
        assert g > 1.0 + 0.2 * dt, (dt, g)  # |1 + dt |Re lambda|| with Re lambda ~ -0.45


def test_ellipsoid_ghost_block_contracts(oracle_mod):
    N = 64
    assert ghost_block_growth(W.phi_ellipsoid(N), N) < 0.95
