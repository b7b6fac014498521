"""Reproduction harness for the paper's convergence study, on the GPU path.

* rho: the asymptotic convergence factor of Sec. 2.2 (homogeneous problem,
  u^(0) ~ U(-1, 1) on every unknown with PCG64 seed 3, eliminated box values
  0; rho = mean of ||r^(m+1)|| / ||r^(m)|| for m = 11..15) for V(2,1) or
  W(2,1) cycles with Delta tau_OPT(theta) (exp or polynomial G0) or a
  constant Delta tau, Dirichlet or Neumann (with the reaction term).
* theta_histogram: the distribution of theta~ = |G - Q| / h over the finest
  ghosts (the histogram the paper shows at N = 2048).

Run as a module to print the tables:

    python -m paper_2207_14208_gb300.repro
"""

from __future__ import annotations

import math

import numpy as np

from . import bcmg
from . import workloads as W


def rho(d: int, N: int, phi: np.ndarray, ncycles: int = 16, **opts) -> float:
    import torch
    s = bcmg.Solver(d, N, torch.from_numpy(phi).cuda(), None, **opts)
    try:
        s.set_boundary_values(torch.zeros(max(s.ghost_count(), 1), dtype=torch.float64, device="cuda")[
            : s.ghost_count()].contiguous())
        cls = s.cls(0)
        rng = np.random.Generator(np.random.PCG64(3))
        u0 = rng.uniform(-1.0, 1.0, s.nn)
        u0[cls == bcmg.BOXDIR] = 0.0
        u = torch.from_numpy(u0).cuda()
        norms = []
        for m in range(ncycles + 1):
            r = s.residual_norm(u)
            norms.append(math.hypot(r[0], r[1]))
            if m < ncycles:
                s.vcycle(u, 1)
        ratios = [norms[m + 1] / norms[m] for m in range(11, min(16, ncycles))]
        return float(np.mean(ratios))
    finally:
        s.close()


def theta_histogram(d: int, N: int, phi: np.ndarray, bins: int = 10):
    import torch
    s = bcmg.Solver(d, N, torch.from_numpy(phi).cuda(), None)
    try:
        eta = s.ghosts(0)["eta"]
    finally:
        s.close()
    h, edges = np.histogram(eta, bins=bins, range=(0.0, 1.0))
    return h / max(1, eta.size), edges


def _table(rows, cols, cell):
    out = ["| | " + " | ".join(str(c) for c in cols) + " |", "|---" * (len(cols) + 1) + "|"]
    for r in rows:
        out.append("| %s | " % r + " | ".join(cell(r, c) for c in cols) + " |")
    return "\n".join(out)


def main():
    doms2 = {"circle": W.phi_circle_paper, "flower": W.phi_flower_paper}
    Ns2 = [64, 128, 256, 512, 1024]
    variants = [("Dtau_OPT exp", dict(dtau_mode=bcmg.DTAU_EXP)), ("Dtau_OPT poly", dict(dtau_mode=bcmg.DTAU_POLY)),
                ("Dtau = 1.75", dict(dtau_mode=bcmg.DTAU_CONST, dtau_const=1.75))]
    for dname, mk in doms2.items():
        print("\n2D %s, Dirichlet, V(2,1): rho" % dname)
        cache = {}
        print(_table([v[0] for v in variants], Ns2,
                     lambda r, N: "%.3f" % cache.setdefault((r, N), rho(2, N, mk(N), **dict(variants)[r]))))
    for dname, mk in doms2.items():
        print("\n2D %s, Neumann, u - Lap u = f, V(2,1): rho" % dname)
        nv = [("Dtau_OPT/h exp", dict(dtau_mode=bcmg.DTAU_EXP)),
              ("Dtau/h = 1", dict(dtau_mode=bcmg.DTAU_CONST, dtau_const=1.0))]
        print(_table([v[0] for v in nv], Ns2,
                     lambda r, N: "%.3f" % rho(2, N, mk(N), bc=bcmg.BC_NEUMANN, reaction=1.0, **dict(nv)[r])))
    print("\n3D ellipsoid, Dirichlet, V(2,1): rho")
    Ns3 = [32, 64, 128, 256]
    print(_table([v[0] for v in variants], Ns3,
                 lambda r, N: "%.3f" % rho(3, N, W.phi_ellipsoid(N), **dict(variants)[r])))
    print("\nW(2,1) against V(2,1), Dtau_OPT exp: rho")
    print(_table(["circle V", "circle W"], Ns2[:4],
                 lambda r, N: "%.3f" % rho(2, N, W.phi_circle_paper(N),
                                          cycle=bcmg.CYCLE_W if r.endswith("W") else bcmg.CYCLE_V)))
    for dname, mk in doms2.items():
        h, edges = theta_histogram(2, 2048, mk(2048))
        print("\ntheta~ histogram, %s N = 2048 (fraction of ghosts per bin of width 0.1):" % dname)
        print(" ".join("%.3f" % v for v in h))


if __name__ == "__main__":
    main()
