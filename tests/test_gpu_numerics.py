"""GPU checks of the numerical building blocks the kernels use in place of
CUDA's own routines, against their error bounds.

* The solve's reciprocal (an FP32 seed from the SFU refined by two
  Newton-Raphson steps, used instead of FP64 divisions in the statistical
  equilibrium and the line parameters): within one FP64 ulp of the correctly
  rounded 1 / d over the whole normal range, exact IEEE results for the
  special inputs it hands to the division.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def loc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_12609_gb300 import build, loc as L
    build.build()
    L.load()
    return L


def test_solve_reciprocal_within_one_ulp(loc):
    rng = np.random.default_rng(20091260)
    n = 1 << 18
    mant = rng.uniform(1.0, 2.0, n)
    mant[:64] = 1.0 + np.arange(64) * 2.0 ** -52          # mantissas next to 1
    mant[64:128] = 2.0 - (np.arange(64) + 1) * 2.0 ** -52  # and next to 2
    e = rng.integers(-1020, 1021, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    d = sign * np.ldexp(mant, e)
    d[-4:] = [1.0, -1.0, 2.0 ** -1021, 2.0 ** 1021]
    r = loc.loc_check_recip(d)
    ref = 1.0 / d
    ulps = np.abs(r - ref) / np.spacing(np.abs(ref))
    assert np.all(np.sign(r) == np.sign(ref))
    assert ulps.max() <= 1.0, ulps.max()
    assert np.mean(r == ref) > 0.5          # mostly the correctly rounded value


def test_solve_reciprocal_special_inputs(loc):
    d = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -2.5e-310, 1e308, -1.7e308,
                  2.0 ** -1022, 2.0 ** 1023])
    r = loc.loc_check_recip(d)
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / d
    np.testing.assert_array_equal(r, ref)
    assert loc.loc_check_recip(np.zeros(0)).size == 0
