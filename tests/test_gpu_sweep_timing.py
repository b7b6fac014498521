"""The sweep timing entry points (bcmg_time_sweeps, bcmg_time_sweeps_bf16).

They run finest-level colour sweeps back to back for the bench's roofline and
must leave the hierarchy as it was: the next V-cycle from the caller's u is
the same as on a hierarchy that was never timed.  The bfloat16 variant works
on temporary 16-bit copies (FP32 arithmetic) and rejects a finest level that
is not split by parity (odd N)."""

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_timed_sweeps_leave_the_hierarchy_unchanged(bcmg, prec):
    B = bcmg
    p = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    d, N = 3, 64
    phi, f = dev(W.phi_ellipsoid(N)), dev(W.manufactured(d, N)[0])
    out = []
    for timed in (False, True):
        s = B.Solver(d, N, phi, f, precision=p)
        s.set_boundary_values(dev(W.g_at(d, s.ghost_points().cpu().numpy())))
        if timed:
            assert s.time_sweeps(20) > 0.0
            assert s.time_sweeps_bf16(20) > 0.0
        u = torch.zeros((N + 1) ** d, dtype=torch.float64, device="cuda")
        s.vcycle(u, 2)
        torch.cuda.synchronize()
        out.append(u.cpu().numpy())
        s.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_bf16_sweeps_need_a_parity_split_level(bcmg):
    B = bcmg
    N = 63  # odd N: one level, dense layout
    s = B.Solver(2, N, dev(W.phi_disk(N)), None)
    with pytest.raises(B.BcmgError) as e:
        s.time_sweeps_bf16(2)
    assert e.value.code == B.EINVAL
    s.close()
