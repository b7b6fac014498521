"""The runtime around the kernels: device blocks cached across handles, the
pooled side stream of creation, and the solve graph captured at creation.

A hierarchy created on reused blocks (the same sizes again), after a miss
that returned the cache to the pool (another size in between), or from many
threads at once must solve exactly like the first one: every kernel writes
what it reads before reading it, so nothing left in a reused block can show
through."""

import threading

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


def _solve(B, d, N, mk, precision=None):
    phi = mk(N)
    f, _ = W.manufactured(d, N)
    kw = {} if precision is None else {"precision": precision}
    s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), **kw)
    try:
        g = W.g_at(d, s.ghost_points().cpu().numpy())
        s.set_boundary_values(torch.from_numpy(g).cuda())
        u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        c, rel = s.solve(u, 1e-10, 100)
        # a stream synchronisation: a device-wide one is rejected while another
        # thread's creation has a stream capture open
        torch.cuda.current_stream().synchronize()
        return c, rel, u.cpu().numpy()
    finally:
        s.close()


def test_reused_blocks_give_the_same_solve(bcmg):
    B = bcmg
    first = _solve(B, 3, 48, W.phi_ellipsoid)
    again = _solve(B, 3, 48, W.phi_ellipsoid)  # the same sizes: cached blocks
    other = _solve(B, 2, 96, W.phi_disk)       # other sizes: the cache goes back to the pool
    after = _solve(B, 3, 48, W.phi_ellipsoid)
    for c, rel, u in (again, after):
        assert c == first[0] and rel == first[1]
        np.testing.assert_array_equal(u, first[2])
    assert other[1] <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_threads_create_and_solve_like_one(bcmg, prec):
    # eight threads, each creating and solving three hierarchies on its own
    # caller stream (pooled side lanes, cached blocks, graphs captured at
    # creation) against the same solves one after another
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    cases = [(2, 64, W.phi_disk), (3, 40, W.phi_ellipsoid), (2, 80, W.phi_flower_paper)]
    ref = [_solve(B, d, N, mk, p) for d, N, mk in cases]
    out = {}
    errors = []
    dev = torch.cuda.current_device()

    def work(k):
        try:
            torch.cuda.set_device(dev)
            with torch.cuda.stream(torch.cuda.Stream()):
                out[k] = [_solve(B, d, N, mk, p) for d, N, mk in cases]
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k in range(8):
        for (c, rel, u), (c0, rel0, u0) in zip(out[k], ref):
            assert c == c0 and rel == rel0
            np.testing.assert_array_equal(u, u0)
