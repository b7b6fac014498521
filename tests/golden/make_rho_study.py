"""Convergence-factor study of the oracle's readings on curved domains.

Writes ``tests/golden/rho_study.txt``: the asymptotic convergence factor rho
of Sec. 2.2 (homogeneous problem, u^(0) ~ U(-1, 1) with PCG64 seed 3, mean of
||r^(m+1)|| / ||r^(m)|| for m = 11..15) in the paper's set-up of Sec. 3.1
(two-grid correction scheme, GS-LEX, nu1 = 2, nu2 = 1, Delta tau_OPT(theta~)
of eq. DtauOptTheta with the exp form of Remark exptheta2D) for each reading
of the places where the paper leaves the transfer operators open:

  default    FW weights restricted to the class family and renormalised, the
             coarse-ghost family = ghost + inactive points, upwind extension
             with K = 4 sweeps over a band of Chebyshev radius 2
  rmode0     unweighted mean of the family members (interior and ghost rows)
  rmode1     weighted mean on interior rows, unweighted on ghost rows
  rmode2     unweighted mean on interior rows, weighted on ghost rows
  gfam1      coarse-ghost family = ghost points only (no extended points)
  K2, K8     2 or 8 extension sweeps
  central    the paper's central-difference extension (explicit Euler, 0.5)
  band3      extension band of Chebyshev radius 3
  inject     coarse-ghost right-hand side injected from the coincident node
  const1.75  constant Delta tau = 1.75 (Remark dtau), default transfers

on the paper's Circle and Flower (Sec. 3.3.3, N = 64..512) and off-centre
ellipsoid (Sec. 4.2, N = 32..128), plus the rectangle of Sec. 3.2 (N = 64)
with the ghost column on and off the coarse grid.

Only the oracle is called.  Run:  python tests/golden/make_rho_study.py
"""

from __future__ import annotations

import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, _ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2207_14208_gb300 import workloads as W  # noqa: E402

READINGS = [
    ("default", {}),
    ("rmode0", dict(rmode=0)),
    ("rmode1", dict(rmode=1)),
    ("rmode2", dict(rmode=2)),
    ("gfam1", dict(gfam=1)),
    ("K2", dict(ext_sweeps=2)),
    ("K8", dict(ext_sweeps=8)),
    ("central", dict(ext_mode=1)),
    ("band3", dict(band_width=3)),
    ("inject", dict(cg_rhs=1)),
    ("const1.75", dict(dtau_mode=O.DT_CONST, dtau_const=1.75)),
]

DOMAINS = [
    ("circle", 2, W.phi_circle_paper, [64, 128, 256, 512]),
    ("flower", 2, W.phi_flower_paper, [64, 128, 256, 512]),
    ("ellipsoid", 3, W.phi_ellipsoid_paper, [32, 64, 128]),
]


def rho(d, N, phi, **kw):
    orc = O.Oracle(d, N, phi, ordering=O.LEX, cycle=O.CYC_TGCS, **kw)
    nn = orc.nn(0)
    orc.set_rhs(np.zeros(nn), np.zeros(orc.info(0)["n_ghost"]))
    r, _ = orc.rho(W.random_u0(nn, 3), 16)
    return r


def rectangle_rows(N=64):
    """rho on the half-plane x < x_V (Sec. 3.2) at Delta tau_OPT (poly form)
    with the ghost column at index N - shift: shift 4 puts it on the coarse
    grid, shift 3 off it."""
    h = 2.0 / N
    out = []
    for shift in (4, 3):
        for th in (0.2, 0.5, 0.6, 0.7, 0.8, 0.9):
            xV = (-1 + (N - shift) * h) - th * h
            out.append((shift, th, rho(2, N, W.phi_halfspace(2, N, xV), dtau_mode=O.DT_POLY)))
    return out


def main(path=None):
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "rho_study.txt")
    lines = ["# rho of the oracle (TGCS, GS-LEX, V(2,1), Delta tau_OPT exp) per reading;",
             "# written by tests/golden/make_rho_study.py (oracle only)",
             "# domain reading N rho"]
    for name, d, mk, Ns in DOMAINS:
        for rname, kw in READINGS:
            for N in Ns:
                r = rho(d, N, mk(N), **kw)
                lines.append(f"{name} {rname} {N} {r:.4f}")
                print(lines[-1], flush=True)
    lines.append("# rectangle x < x_V, N = 64, Delta tau_OPT poly: rect<shift> theta rho")
    for shift, th, r in rectangle_rows():
        lines.append(f"rect{shift} {th} 64 {r:.4f}")
        print(lines[-1], flush=True)
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
