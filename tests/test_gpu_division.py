"""The restriction's family mean divides by the family's FW weight sum
w in 1..64 with a table reciprocal and one FMA correction (Markstein's
method).  The result must equal the correctly rounded quotient a / w, in FP64
and in FP32, for values across many binades."""

import numpy as np
import pytest

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


def _inputs(n, lo_exp, hi_exp, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(-2.0, 2.0, n)
    return mant * np.exp2(rng.integers(lo_exp, hi_exp, n).astype(np.float64))


def test_div_wsum_fp64_correctly_rounded(bcmg):
    a = _inputs(64 * 4096, -60, 60, 1)
    a[:64] = 1.0  # 1/w itself
    w = 1.0 + np.arange(a.size) % 64
    got = bcmg.selftest_div_wsum(a, fp32=False)
    np.testing.assert_array_equal(got, a / w)


def test_div_wsum_fp32_correctly_rounded(bcmg):
    a = _inputs(64 * 4096, -30, 30, 2).astype(np.float32).astype(np.float64)
    a[:64] = 1.0
    w = (1 + np.arange(a.size) % 64).astype(np.float32)
    got = bcmg.selftest_div_wsum(a, fp32=True)
    np.testing.assert_array_equal(got, (a.astype(np.float32) / w).astype(np.float64))
