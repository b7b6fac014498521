"""Rectangle validation on the GPU path (Sec. 3.2.1): after 10 relaxations
from a random guess, the DFT of the residual along the ghost column has the
smallest high- to low-frequency ratio at Delta tau_OPT(theta) — the
smoothing property the paper shows for theta = 0.2, 0.5, 0.8 at N = 128.
The GPU spectrum is also checked against one computed from the oracle's
relaxation (with this file's own DFT)."""

import numpy as np
import pytest

from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def repro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14208_gb300 import build, repro
    build.build()
    O.build()
    return repro


def _oracle_ratio(N, theta, dtau):
    h = 2.0 / N
    xV = (-1.0 + (3 * N // 4 + 1) * h) - theta * h
    x = -1.0 + h * np.arange(N + 1)
    phi = np.tile(x - xV, N + 1)
    o = O.Oracle(2, N, phi, dtau_mode=O.DT_CONST, dtau_const=dtau)
    u = np.random.Generator(np.random.PCG64(4)).uniform(-1.0, 1.0, o.nn(0))
    u[o.cls(0) == O.BOXDIR] = 0.0
    F = np.zeros(o.nn(0))
    r = o.residual(0, o.smooth(0, u, F, 10), F)
    idx = np.sort(o.ghosts(0)["idx"])
    rows = idx // (N + 1)
    M = idx.size
    lo = hi = 0.0
    for k in range(1, M + 1):
        a = -np.pi + 2.0 * np.pi * k / M
        if a <= 0:
            continue
        amp = 2.0 * abs(np.sum(r[idx] * np.exp(-1j * a * rows)) / M)
        if a > np.pi / 2:
            hi += amp
        elif a < np.pi / 2:
            lo += amp
    return hi / lo


@pytest.mark.parametrize("theta", [0.2, 0.5, 0.8])
def test_optimal_dtau_smooths_the_boundary_best(repro, theta):
    from paper_2207_14208_gb300 import bcmg
    N = 128
    opt = bcmg.dtau_opt(2, theta, bcmg.DTAU_POLY)
    ratios = [repro.high_low_ratio(*repro.ghost_residual_spectrum(N, theta, f * opt)) for f in (0.5, 1.0, 1.5)]
    assert ratios[1] < ratios[0] and ratios[1] < ratios[2], ratios
    assert ratios[1] == pytest.approx(_oracle_ratio(N, theta, opt), rel=1e-8)
