"""Batched solves (bcmg_solve_batch) and device-memory footprints.

Many hierarchies of uneven size and shape are solved in one call.  A batch
of one dimension and precision runs through the batched kernels (one launch
per stage of the cycle for all hierarchies): one batched cycle must match
the oracle's cycle, whole solves must match the same solves alone to
rounding, and the result must not depend on the launch shape (block size,
items per thread, block tail).  A mixed batch (2D and 3D) runs each solve on
its own stream and must be bit-identical to the same solve alone.  The
footprint estimate used for admission must cover what a hierarchy actually
holds."""

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


def _problems():
    """Seeded star domains of the batched workload (sizes 64..1024 drawn
    log-uniformly; the small ones kept so the test stays quick) plus a 3D
    ellipsoid."""
    out = []
    for N, a, k, psi in W.star_params(256, 1):
        if N <= 320 and len(out) < 6:
            out.append((2, N, W.phi_star(N, a, k, psi)))
    out.append((3, 40, W.phi_ellipsoid(40)))
    return out


def _make(B, d, N, phi, precision):
    f, _ = W.manufactured(d, N)
    s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), precision=precision)
    g = W.g_at(d, s.ghost_points().cpu().numpy())
    s.set_boundary_values(torch.from_numpy(g).cuda())
    return s, torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_alone(bcmg, prec):
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    probs = _problems()
    alone = []
    for d, N, phi in probs:
        s, u = _make(B, d, N, phi, p)
        c, rel = s.solve(u, 1e-10, 100)
        torch.cuda.synchronize()
        alone.append((c, rel, u.cpu().numpy()))
        s.close()
    pairs = [_make(B, d, N, phi, p) for d, N, phi in probs]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 100)
    torch.cuda.synchronize()
    assert st == [B.OK] * len(probs)
    for i, (s, u) in enumerate(pairs):
        assert cyc[i] == alone[i][0] and rel[i] == alone[i][1]
        np.testing.assert_array_equal(u.cpu().numpy(), alone[i][2])
        s.close()


def test_batch_rejects_duplicates_and_reports_limits(bcmg):
    B = bcmg
    s, u = _make(B, 2, 64, W.phi_disk(64), B.PREC_FP64)
    with pytest.raises(B.BcmgError):
        B.solve_batch([s, s], [u, u.clone()])
    cyc, rel, st = B.solve_batch([s], [u], 1e-14, 2)
    assert cyc == [2] and st == [B.ENOCONV]
    s.close()


@pytest.mark.parametrize("d,N,mk,prec", [(2, 128, W.phi_disk, "fp64"), (2, 512, W.phi_disk, "mixed"),
                                         (3, 96, W.phi_ellipsoid, "fp64"), (3, 256, W.phi_ellipsoid, "mixed")])
def test_footprint_estimate_covers_actual(bcmg, d, N, mk, prec):
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    s, _ = _make(B, d, N, mk(N), p)
    actual = s.memory_footprint()
    est = B.footprint_estimate(d, N, precision=p)
    assert 0 < actual <= est <= 4 * actual + (16 << 20)
    s.close()


# ------------------------------------------------ batched kernels (one launch
# per stage for every hierarchy of a batch of one dimension and precision)

def _star_set(n, nmax):
    out = []
    for N, a, k, psi in W.star_params(256, 1):
        if N <= nmax and len(out) < n:
            out.append((2, N, W.phi_star(N, a, k, psi)))
    return out


def _ellipsoid_set():
    return [(3, N, W.phi_ellipsoid(N)) for N in (40, 48, 64, 96)]


# launch shapes of the batched kernels: (block, items per thread, tail rows);
# None = the autotuner's choice
SHAPES = [None, (128, 1, 0), (64, 4, 0), (128, 4, 512), (256, 4, 2048)]


@pytest.fixture
def shape(bcmg, request):
    s = request.param
    if s is not None:
        bcmg.debug_batch_shape(*s)
    yield s
    bcmg.debug_batch_shape(0)


@pytest.mark.parametrize("shape", SHAPES, indirect=True, ids=lambda s: "tuned" if s is None else "%d-%d-%d" % s)
@pytest.mark.parametrize("which", ["stars", "ellipsoids"])
def test_batched_cycle_matches_oracle(bcmg, which, shape):
    # one batched V-cycle per hierarchy (max_cycles = 1) against the oracle's
    # V-cycle from the same start: the batched stages (and the block tail,
    # where the shape has one) run the same per-node steps, the coarse levels
    # included
    from oracle import oracle as O
    O.build()
    B = bcmg
    probs = _star_set(8, 400) if which == "stars" else _ellipsoid_set()
    pairs = [_make(B, d, N, phi, B.PREC_FP64) for d, N, phi in probs]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 0.0, 1)
    torch.cuda.synchronize()
    assert cyc == [1] * len(probs)
    for (d, N, phi), (s, u) in zip(probs, pairs):
        o = O.Oracle(d, N, phi)
        f, _ = W.manufactured(d, N)
        o.set_rhs(f, W.g_at(d, o.ghosts(0)["Q"]))
        uo = o.vcycle(np.zeros(o.nn(0)), 1)
        act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
        got = u.cpu().numpy()
        assert np.abs(got[act] - uo[act]).max() <= 1e-12 * np.abs(uo[act]).max(), (d, N)
        s.close()


@pytest.mark.parametrize("shape", [None, (128, 4, 2048)], indirect=True,
                         ids=lambda s: "tuned" if s is None else "%d-%d-%d" % s)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solves_match_alone(bcmg, prec, shape):
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    probs = _star_set(12, 640)
    alone = []
    for d, N, phi in probs:
        s, u = _make(B, d, N, phi, B.PREC_FP64)
        c, rel = s.solve(u, 1e-10, 100, raise_noconv=False)
        torch.cuda.synchronize()
        alone.append((c, rel, u.cpu().numpy(), s.cls(0)))
        s.close()
    pairs = [_make(B, d, N, phi, p) for d, N, phi in probs]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 100)
    torch.cuda.synchronize()
    for i, (s, u) in enumerate(pairs):
        c0, r0, u0, cls = alone[i]
        if r0 > 1e-10:  # a star the method does not converge on
            assert st[i] == B.ENOCONV
            continue
        assert st[i] == B.OK and rel[i] <= 1e-10
        assert abs(cyc[i] - c0) <= (1 if prec == "fp64" else 3)
        act = np.isin(cls, [B.INTERIOR, B.GHOST])
        got = u.cpu().numpy()
        assert np.abs(got[act] - u0[act]).max() <= 1e-9 * np.abs(u0[act]).max()
        s.close()


def test_batched_limits_and_mixed_convergence(bcmg):
    B = bcmg
    probs = _star_set(5, 400)
    pairs = [_make(B, d, N, phi, B.PREC_FP64) for d, N, phi in probs]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-14, 2)
    assert cyc == [2] * len(probs) and st == [B.ENOCONV] * len(probs)
    # a second call on the same hierarchies continues from the caller's u
    cyc2, rel2, st2 = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-6, 60)
    assert all(c < 60 for c in cyc2) and st2 == [B.OK] * len(probs)
    for s, _ in pairs:
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_tail_is_shape_independent(bcmg, prec):
    # the same batched cycles with and without the block tail: identical u
    # (the tail runs the stages' per-node steps in the stages' order), and
    # the tail takes stage launches off every cycle
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    probs = _star_set(10, 640)
    res = {}
    try:
        for shp in ((128, 4, 0), (128, 4, 2048), (64, 1, 512)):
            B.debug_batch_shape(*shp)
            pairs = [_make(B, d, N, phi, p) for d, N, phi in probs]
            k0 = B.kernel_launches()
            cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 0.0, 3)
            torch.cuda.synchronize()
            res[shp] = (B.kernel_launches() - k0, [u.cpu().numpy() for _, u in pairs])
            for s, _ in pairs:
                s.close()
    finally:
        B.debug_batch_shape(0)
    base = res[(128, 4, 0)][1]
    for shp in ((128, 4, 2048), (64, 1, 512)):
        for a, b in zip(base, res[shp][1]):
            np.testing.assert_array_equal(a, b)
    assert res[(128, 4, 2048)][0] < res[(128, 4, 0)][0]


def test_last_shape_reports_the_fixed_shape(bcmg):
    B = bcmg
    probs = _star_set(3, 200)
    try:
        B.debug_batch_shape(64, 4, 512)
        pairs = [_make(B, d, N, phi, B.PREC_FP64) for d, N, phi in probs]
        B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 5)
        assert B.batch_last_shape() == (64, 4, 512)
        for s, _ in pairs:
            s.close()
    finally:
        B.debug_batch_shape(0)


def test_batch_shape_rejects_bad_values(bcmg):
    B = bcmg
    for bad in ((100, 1, 0), (128, 3, 0), (128, 1, -1)):
        with pytest.raises(B.BcmgError) as e:
            B.debug_batch_shape(*bad)
        assert e.value.code == B.EINVAL
    B.debug_batch_shape(0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_degenerate_hierarchies(bcmg, prec):
    # one level only (odd N: the finest level is the coarsest, solved
    # directly), two levels, a zero problem (r0 = 0: done before any cycle)
    # and an ordinary star in one batch; every result as alone
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    probs = [(2, 15, W.phi_disk(15)), (2, 30, W.phi_disk(30)), (2, 64, W.phi_star(64, 0.12, 5, 0.4)),
             (2, 48, W.phi_disk(48))]

    def build(i, d, N, phi):
        if i == 3:  # zero data
            s = B.Solver(d, N, torch.from_numpy(phi).cuda(), None, precision=p)
            s.set_boundary_values(torch.zeros(s.ghost_count(), dtype=torch.float64, device="cuda"))
            return s, torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        return _make(B, d, N, phi, p)

    alone = []
    for i, (d, N, phi) in enumerate(probs):
        s, u = build(i, d, N, phi)
        c, rel, st = B.solve_batch([s], [u], 1e-10, 60)
        torch.cuda.synchronize()
        alone.append((c[0], rel[0], st[0], u.cpu().numpy(), s.levels))
        s.close()
    assert alone[0][4] == 1 and alone[1][4] == 2
    assert alone[3][0] == 0 and alone[3][2] == B.OK
    pairs = [build(i, d, N, phi) for i, (d, N, phi) in enumerate(probs)]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 60)
    torch.cuda.synchronize()
    for i, (s, u) in enumerate(pairs):
        c0, r0, s0, u0, _ = alone[i]
        assert st[i] == s0
        assert abs(cyc[i] - c0) <= (1 if prec == "fp64" else 3)
        got = u.cpu().numpy()
        scale = max(np.abs(u0).max(), 1e-300)
        assert np.abs(got - u0).max() <= 1e-9 * scale, i
        s.close()
    # no cycle allowed: every non-trivial solve ends unconverged, the zero
    # problem converged, in the batch as alone
    pairs = [build(i, d, N, phi) for i, (d, N, phi) in enumerate(probs)]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 0)
    assert cyc == [0, 0, 0, 0]
    assert st == [B.ENOCONV, B.ENOCONV, B.ENOCONV, B.OK]
    for s, _ in pairs:
        s.close()


def test_vcycle_batch_matches_oracle_and_alone(bcmg):
    # batched V-cycles (bcmg_vcycle_batch): on an eligible batch exactly
    # ncycles cycles per hierarchy, each within 1e-12 of the oracle's cycles
    # (also a zero problem, whose cycles keep u at zero); on a mixed 2D / 3D
    # batch identical to bcmg_vcycle on each handle
    from oracle import oracle as O
    O.build()
    B = bcmg
    probs = _star_set(5, 300)
    pairs = [_make(B, d, N, phi, B.PREC_FP64) for d, N, phi in probs]
    B.vcycle_batch([s for s, _ in pairs], [u for _, u in pairs], 2)
    torch.cuda.synchronize()
    for (d, N, phi), (s, u) in zip(probs, pairs):
        o = O.Oracle(d, N, phi)
        f, _ = W.manufactured(d, N)
        o.set_rhs(f, W.g_at(d, o.ghosts(0)["Q"]))
        uo = o.vcycle(np.zeros(o.nn(0)), 2)
        act = np.isin(o.cls(0), [O.INTERIOR, O.GHOST])
        assert np.abs(u.cpu().numpy()[act] - uo[act]).max() <= 1e-12 * np.abs(uo[act]).max(), N
        s.close()
    zs = B.Solver(2, 64, torch.from_numpy(W.phi_disk(64)).cuda(), None)
    zs.set_boundary_values(torch.zeros(zs.ghost_count(), dtype=torch.float64, device="cuda"))
    zu = torch.zeros(65 * 65, dtype=torch.float64, device="cuda")
    s2, u2 = _make(B, 2, 96, W.phi_disk(96), B.PREC_FP64)
    B.vcycle_batch([zs, s2], [zu, u2], 3)
    assert float(zu.abs().max()) == 0.0 and float(u2.abs().max()) > 0.0
    zs.close()
    s2.close()
    mixed = [(2, 64, W.phi_disk(64)), (3, 24, W.phi_ellipsoid(24)), (2, 80, W.phi_flower_paper(80))]
    alone = []
    for d, N, phi in mixed:
        s, u = _make(B, d, N, phi, B.PREC_FP64)
        s.vcycle(u, 2)
        torch.cuda.synchronize()
        alone.append(u.cpu().numpy())
        s.close()
    pairs = [_make(B, d, N, phi, B.PREC_FP64) for d, N, phi in mixed]
    B.vcycle_batch([s for s, _ in pairs], [u for _, u in pairs], 2)
    torch.cuda.synchronize()
    with pytest.raises(B.BcmgError) as e:
        B.vcycle_batch([pairs[0][0]], [pairs[0][1]], -1)
    assert e.value.code == B.EINVAL
    for a, (s, u) in zip(alone, pairs):
        np.testing.assert_array_equal(u.cpu().numpy(), a)
        s.close()


def test_host_boundary_data_equals_device(bcmg):
    # bcmg_ghost_points into host memory and bcmg_set_boundary_values from
    # host memory give what the device buffers give
    B = bcmg
    d, N = 2, 96
    phi = torch.from_numpy(W.phi_flower_paper(N)).cuda()
    f = torch.from_numpy(W.manufactured(d, N)[0]).cuda()
    out = []
    for host in (False, True):
        s = B.Solver(d, N, phi, f)
        if host:
            Q = s.ghost_points(out=np.empty((s.ghost_count(), d)))
            s.set_boundary_values(W.g_at(d, Q))
        else:
            Q = s.ghost_points().cpu().numpy()
            s.set_boundary_values(torch.from_numpy(W.g_at(d, Q)).cuda())
        u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        c, rel = s.solve(u, 1e-10, 60)
        out.append((Q.copy(), c, u.cpu().numpy()))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_neumann_with_reaction_matches_alone(bcmg, prec):
    # Neumann rows and the reaction term (c u - Lap u = f, Sec. 4.2 Test2N)
    # through the batched kernels: the same results as each solve alone
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    probs = [(2, N, W.phi_star(N, 0.1, k, 0.3)) for N, k in ((64, 5), (96, 4), (128, 6))]

    def make(d, N, phi):
        f, _ = W.manufactured(d, N)
        s = B.Solver(d, N, torch.from_numpy(phi).cuda(), torch.from_numpy(f).cuda(), precision=p,
                     bc=B.BC_NEUMANN, reaction=1.0)
        Q = s.ghost_points()
        s.set_boundary_values((torch.sin(3.0 * Q[:, 0]) * torch.cos(2.0 * Q[:, 1])).contiguous())
        return s, torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")

    alone = []
    for d, N, phi in probs:
        s, u = make(d, N, phi)
        c, rel = s.solve(u, 1e-10, 80)
        torch.cuda.synchronize()
        alone.append((c, u.cpu().numpy(), s.cls(0)))
        s.close()
    pairs = [make(d, N, phi) for d, N, phi in probs]
    cyc, rel, st = B.solve_batch([s for s, _ in pairs], [u for _, u in pairs], 1e-10, 80)
    torch.cuda.synchronize()
    for (c0, u0, cls), (s, u), c, r, status in zip(alone, pairs, cyc, rel, st):
        assert status == B.OK and r <= 1e-10
        assert abs(c - c0) <= (1 if prec == "fp64" else 3)
        act = np.isin(cls, [B.INTERIOR, B.GHOST])
        assert np.abs(u.cpu().numpy()[act] - u0[act]).max() <= 1e-9 * np.abs(u0[act]).max()
        s.close()
