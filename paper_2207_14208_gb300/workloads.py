"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This module only produces problem data (level-set values on the grid,
manufactured solutions and their right-hand sides, random initial guesses);
it contains none of the multigrid method's arithmetic.  Grid convention of the
paper (Sec. 3 and Sec. 4 set-up): D = [-1,1]^d, N cells per axis,
x_i = -1 + i h, h = 2/N, arrays x-fastest with (N+1)^d entries.

Domains, all analytic and synthetic:
  * disk       phi = x^2 + y^2 - 0.49                 (centred stand-in for the
               paper's Circle test, Sec. 3.3.3)
  * ellipsoid  phi = x^2/0.36 + y^2/0.25 + z^2/0.16 - 1 (centred stand-in for
               the paper's 3D ellipsoid, Sec. 4.2)
  * spheres    phi = min_i(|X - c_i| - r_i), 64 seeded spheres
  * star       phi = r - 0.5 - a sin(k atan2(y, x) + psi), seeded a, k, psi
  * box        phi = -1 (no curved boundary; every box node is eliminated)
  * halfspace  phi = x_0 - x_V (the paper's rectangle tests, Sec. 3.2 / 4.1)
  * circle / flower: the paper's own off-centre Circle and Flower level sets
  * ellipsoid_paper: the paper's own off-centre ellipsoid (Sec. 4.2)
"""

from __future__ import annotations

import math

import numpy as np


def coords(d: int, N: int):
    """Meshgrid of node coordinates, each of shape (N+1,)*d in x-fastest
    (C order reversed) layout so that ``arr.reshape(-1)`` is x-fastest."""
    x = -1.0 + (2.0 / N) * np.arange(N + 1, dtype=np.float64)
    if d == 1:
        return (x.copy(),)
    if d == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")  # arr[j, i]
        return X, Y
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")  # arr[k, j, i]
    return X, Y, Z


# ---------------------------------------------------------------- domains

def phi_disk(N: int, R2: float = 0.49) -> np.ndarray:
    X, Y = coords(2, N)
    return (X * X + Y * Y - R2).reshape(-1)


def phi_ellipsoid(N: int, a=0.6, b=0.5, c=0.4) -> np.ndarray:
    X, Y, Z = coords(3, N)
    return (X * X / (a * a) + Y * Y / (b * b) + Z * Z / (c * c) - 1.0).reshape(-1)


def sphere_params(count: int = 64, seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-0.8, 0.8, size=(count, 3))
    radii = rng.uniform(0.05, 0.15, size=count)
    return centres, radii


def phi_spheres(N: int, count: int = 64, seed: int = 0) -> np.ndarray:
    X, Y, Z = coords(3, N)
    centres, radii = sphere_params(count, seed)
    phi = np.full(X.shape, np.inf)
    for (cx, cy, cz), r in zip(centres, radii):
        np.minimum(phi, np.sqrt((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) - r, out=phi)
    return phi.reshape(-1)


def star_params(count: int = 256, seed: int = 1):
    """(N, a, k, psi) per star domain: N log-uniform in [64, 1024] rounded to
    the nearest m 2^k with 8 <= m <= 15."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    cands = sorted({m << k for m in range(8, 16) for k in range(0, 12)})
    cands = np.array([c for c in cands if 32 <= c <= 2048])
    for _ in range(count):
        Nf = math.exp(rng.uniform(math.log(64.0), math.log(1024.0)))
        N = int(cands[np.argmin(np.abs(cands - Nf))])
        a = rng.uniform(0.05, 0.2)
        k = int(rng.integers(3, 9))
        psi = rng.uniform(0.0, 2.0 * math.pi)
        out.append((N, a, k, psi))
    return out


def phi_star(N: int, a: float, k: int, psi: float) -> np.ndarray:
    X, Y = coords(2, N)
    r = np.sqrt(X * X + Y * Y)
    return (r - 0.5 - a * np.sin(k * np.arctan2(Y, X) + psi)).reshape(-1)


def phi_box(d: int, N: int) -> np.ndarray:
    return -np.ones((N + 1) ** d)


def phi_halfspace(d: int, N: int, xV: float) -> np.ndarray:
    """phi = x - xV: domain {x < xV} of the rectangle tests."""
    C = coords(d, N)
    return (C[0] - xV).reshape(-1)


def phi_circle_paper(N: int) -> np.ndarray:
    """The paper's off-centre Circle (eq. dom2D:circle)."""
    X, Y = coords(2, N)
    x0, y0, R = math.sqrt(3.0) / 40.0, -math.sqrt(4.0) / 40.0, math.sqrt(2.0) / 2.0
    return ((X - x0) ** 2 + (Y - y0) ** 2 - R * R).reshape(-1)


def phi_flower_paper(N: int) -> np.ndarray:
    """The paper's Flower level set (eq. dom2D:flower), centred (x0 = y0 = 0):
    r - r1 - r2 (y^5 + 5 x^4 y - 10 x^2 y^3) / r^5 with r1 = 0.5, r2 = 0.2."""
    X, Y = coords(2, N)
    r = np.sqrt(X * X + Y * Y)
    safe = np.where(r == 0, 1.0, r)
    c = np.where(r == 0, 1.0, X / safe)
    s = np.where(r == 0, 0.0, Y / safe)
    r1, r2 = 0.5, 0.2
    return (r - r1 - r2 * (s ** 5 + 5 * c ** 4 * s - 10 * c ** 2 * s ** 3)).reshape(-1)


def phi_ellipsoid_paper(N: int) -> np.ndarray:
    """The paper's off-centre ellipsoid of Sec. 4.2: centre
    (sqrt(2)/20, sqrt(3)/40, -sqrt(2)/50), semi-axes 0.686, 0.386, 0.586."""
    X, Y, Z = coords(3, N)
    cx, cy, cz = math.sqrt(2.0) / 20.0, math.sqrt(3.0) / 40.0, -math.sqrt(2.0) / 50.0
    return (((X - cx) / 0.686) ** 2 + ((Y - cy) / 0.386) ** 2
            + ((Z - cz) / 0.586) ** 2 - 1.0).reshape(-1)


# ---------------------------------------------------- manufactured solutions

def u_exact_2d(x, y):
    """u* = sin(pi x) cos(pi y) e^x."""
    return np.sin(np.pi * x) * np.cos(np.pi * y) * np.exp(x)


def f_exact_2d(x, y):
    """f = -Lap u* for u_exact_2d."""
    pi = np.pi
    return -np.exp(x) * np.cos(pi * y) * ((1 - 2 * pi * pi) * np.sin(pi * x) + 2 * pi * np.cos(pi * x))


def u_exact_3d(x, y, z):
    """u* = exp(x + y + z) sin(pi z)."""
    return np.exp(x + y + z) * np.sin(np.pi * z)


def f_exact_3d(x, y, z):
    pi = np.pi
    return -np.exp(x + y + z) * ((3 - pi * pi) * np.sin(pi * z) + 2 * pi * np.cos(pi * z))


def u_exact(d: int, *X):
    return u_exact_2d(*X) if d == 2 else u_exact_3d(*X)


def f_exact(d: int, *X):
    return f_exact_2d(*X) if d == 2 else f_exact_3d(*X)


def manufactured(d: int, N: int):
    """(f on the grid, u* on the grid) for the manufactured solution of
    dimension d."""
    C = coords(d, N)
    return f_exact(d, *C).reshape(-1), u_exact(d, *C).reshape(-1)


def g_at(d: int, Q: np.ndarray) -> np.ndarray:
    """Dirichlet data g = u* evaluated at projection points Q (n x d)."""
    Q = np.asarray(Q, dtype=np.float64).reshape(-1, d)
    return u_exact(d, *[Q[:, a] for a in range(d)])


def random_u0(nn: int, seed: int = 3) -> np.ndarray:
    """u^(0) ~ U(-1, 1) (the convergence-factor protocol of Sec. 2.2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=nn)
