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


def rectangle_phi(N: int, theta: float):
    """The rectangle set-up of Sec. 3.2 in [-1, 1]^2: the domain x < xV with
    one column of ghosts at node column 3N/4 + 1 (not a coarse-grid column),
    all at distance theta h from the boundary; box sides inside the domain
    are eliminated Dirichlet nodes."""
    h = 2.0 / N
    xV = (-1.0 + (3 * N // 4 + 1) * h) - theta * h
    return (W.coords(2, N)[0] - xV).reshape(-1)


def ghost_residual_spectrum(N: int, theta: float, dtau: float, nsmooth: int = 10, seed: int = 4):
    """Sec. 3.2.1 smoothing check: from u ~ U(-1, 1) (PCG64 seed), nsmooth
    relaxations of the homogeneous problem on the finest level with a
    constant Delta tau, then the DFT of the ghost residual along the ghost
    column, R_k = mean_j r_j exp(-i alpha_k j), alpha_k = -pi + 2 pi k / M.
    Returns (alpha_k in (0, pi), amplitudes 2 |R_k|)."""
    import torch
    s = bcmg.Solver(2, N, torch.from_numpy(rectangle_phi(N, theta)).cuda(), None,
                    dtau_mode=bcmg.DTAU_CONST, dtau_const=float(dtau))
    try:
        cls = s.cls(0)
        rng = np.random.Generator(np.random.PCG64(seed))
        u0 = rng.uniform(-1.0, 1.0, s.nn)
        u0[cls == bcmg.BOXDIR] = 0.0
        u = torch.from_numpy(u0).cuda()
        F = torch.zeros_like(u)
        s.smooth(0, u, F, nsmooth)
        r = torch.zeros_like(u)
        s.residual(0, u, F, r)
        torch.cuda.synchronize()
        idx = s.ghosts(0)["idx"]
        rr = r.cpu().numpy()
    finally:
        s.close()
    j = idx // (N + 1)
    order = np.argsort(j)
    rb, jj = rr[idx[order]], j[order]
    M = rb.size
    ak = -np.pi + np.arange(1, M + 1) * 2.0 * np.pi / M
    R = np.exp(-1j * np.outer(ak, jj)) @ rb / M
    pos = ak > 0
    return ak[pos], 2.0 * np.abs(R[pos])


def high_low_ratio(alpha, amp):
    """Summed high-frequency (alpha > pi/2) over low-frequency amplitude."""
    return float(amp[alpha > np.pi / 2].sum() / amp[alpha < np.pi / 2].sum())


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
    print("\nGS-LEX (the paper's order) against red-black, V(2,1), Dtau_OPT exp: rho")
    print(_table(["circle RB", "circle LEX", "flower RB", "flower LEX"], [64, 128, 256],
                 lambda r, N: "%.3f" % rho(2, N, (W.phi_circle_paper if r.startswith("circle") else
                                                  W.phi_flower_paper)(N),
                                          ordering=bcmg.ORDER_LEX if r.endswith("LEX") else bcmg.ORDER_RB)))
    print("\nTwo-grid correction scheme (the paper's protocol, Sec. 2.1: the level-1 problem solved by 30 "
          "V-cycles), (2,1) smoothing: rho")
    tg = dict(cycle=bcmg.CYCLE_TG, tg_inner=30)
    print(_table(["circle Dtau_OPT exp", "circle Dtau = 1.75", "flower Dtau_OPT exp", "flower Dtau = 1.75"],
                 Ns2[:4],
                 lambda r, N: "%.3f" % rho(2, N, (W.phi_circle_paper if r.startswith("circle") else
                                                  W.phi_flower_paper)(N),
                                          **tg, **(dict(dtau_mode=bcmg.DTAU_CONST, dtau_const=1.75)
                                                   if r.endswith("1.75") else dict(dtau_mode=bcmg.DTAU_EXP)))))
    print("\nW(2,1) against V(2,1), Dtau_OPT exp: rho")
    print(_table(["circle V", "circle W"], Ns2[:4],
                 lambda r, N: "%.3f" % rho(2, N, W.phi_circle_paper(N),
                                          cycle=bcmg.CYCLE_W if r.endswith("W") else bcmg.CYCLE_V)))
    print("\nRectangle (Sec. 3.2.1), N = 128, 10 relaxations from U(-1, 1): high/low ratio of the "
          "ghost-residual spectrum at (0.5, 1, 1.5) x Delta tau_OPT(theta)")
    for theta in (0.2, 0.5, 0.8):
        opt = bcmg.dtau_opt(2, theta, bcmg.DTAU_POLY)
        ratios = [high_low_ratio(*ghost_residual_spectrum(128, theta, f * opt)) for f in (0.5, 1.0, 1.5)]
        print("theta %.1f: " % theta + " ".join("%.3g" % x for x in ratios))
    for dname, mk in doms2.items():
        h, edges = theta_histogram(2, 2048, mk(2048))
        print("\ntheta~ histogram, %s N = 2048 (fraction of ghosts per bin of width 0.1):" % dname)
        print(" ".join("%.3f" % v for v in h))


if __name__ == "__main__":
    main()
