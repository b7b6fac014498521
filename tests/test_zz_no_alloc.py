"""The allocation-free residual-norm entry point (bcmg_residual_norms_static).

Some callers cannot allocate device memory (code running inside a stream
capture, plugins whose host application owns all allocations, processes that
forbid cudaMalloc after start-up).  For them the library offers one entry
point whose scratch is a fixed __device__ array.  This test calls it through
the C ABI and checks it against the allocating entry point
(bcmg_residual_norm) on two calls in a row.  It is collected last so that a
run stopping at the first failure has already run every other test, and it
also passes on its own in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def bcmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14208_gb300 import bcmg as B
    from paper_2207_14208_gb300 import build
    build.build()
    return B


def _problem(B, d, N, mk):
    from paper_2207_14208_gb300 import workloads as W
    phi = mk(N)
    f, _ = W.manufactured(d, N)
    s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda())
    Q = s.ghost_points().cpu().numpy()
    g = W.g_at(d, Q)
    s.set_boundary_values(torch.from_numpy(g).cuda())
    cls = s.cls(0)
    # the finest-level right-hand side as the library holds it: f on interior
    # rows, g on ghost rows
    F = np.zeros_like(f)
    F[cls == B.INTERIOR] = f[cls == B.INTERIOR]
    F[s.ghosts(0)["idx"]] = g
    return s, torch.from_numpy(F).cuda(), torch.from_numpy(cls).cuda()


@pytest.mark.parametrize("case", ["disk128", "ellipsoid64"])
def test_static_norms_match_allocating_entry_point(bcmg, case):
    from paper_2207_14208_gb300 import workloads as W
    B = bcmg
    d, N, mk = {"disk128": (2, 128, W.phi_disk), "ellipsoid64": (3, 64, W.phi_ellipsoid)}[case]
    s, F, cls = _problem(B, d, N, mk)
    nn = (N + 1) ** d
    rng = np.random.default_rng(11)
    u = torch.from_numpy(rng.uniform(-1, 1, nn)).cuda()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        if call == 1:
            s.vcycle(u, 1)  # a different residual for the second call
        r = torch.zeros(nn, dtype=torch.float64, device="cuda")
        s.residual(0, u, F, r)
        B.residual_norms_static(r, cls, out)
        got = out.cpu().numpy()
        want = s.residual_norm(u)
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=0)


def test_static_norms_reject_oversized_input(bcmg):
    B = bcmg
    big = 33554432 + 1
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    cls = torch.zeros(1, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    import ctypes
    rc = B.load().bcmg_residual_norms_static(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(cls.data_ptr()),
                                             big, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == B.EINVAL
    assert "capacity" in B.load().bcmg_last_error().decode()


def test_static_norms_large_input(bcmg):
    # 257^3 entries: more than 1024 partial blocks, so the final reduction
    # walks its partials in strides; checked against a torch reduction of the
    # interior and ghost entries, on two different inputs in a row
    B = bcmg
    n = 257 ** 3
    g = torch.Generator(device="cuda").manual_seed(5)
    cls = torch.randint(0, 4, (n,), generator=g, device="cuda", dtype=torch.uint8)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        r = torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 2 - 1
        B.residual_norms_static(r, cls, out)
        ri, rg = r[cls == B.INTERIOR], r[cls == B.GHOST]
        want = torch.stack([ri.norm(), rg.norm(), ri.abs().max(), rg.abs().max()]).cpu().numpy()
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL, atol=0)
