"""Pins of the oracle's channel-integrated line profile (Sect. 2: phi is the
fraction of emitted photons per channel; Sect. 3.1: Doppler shift of the
local profile).

Pinned against numerical quadrature of the Gaussian density (scipy.quad, not
the error function the oracle uses), the moments of a discretised Gaussian,
and the sign convention (approaching gas is blue-shifted).
"""
import numpy as np
import pytest
from scipy import integrate


def _gauss(v, mu, sigma):
    return np.exp(-0.5 * ((v - mu) / sigma) ** 2) / (np.sqrt(2 * np.pi) * sigma)


@pytest.mark.parametrize("v_los,sigma", [(0.0, 2.0e4), (3.1e4, 1.5e4), (-2.2e5, 4.0e4), (1.7e5, 0.9e4)])
def test_channel_fractions_match_quadrature(oracle, v_los, sigma):
    n_ch, v_min, dv = 40, -2.0e5, 1.0e4
    phi = oracle.profile(n_ch, v_min, dv, v_los, sigma)
    for k in range(n_ch):
        lo, hi = v_min + k * dv, v_min + (k + 1) * dv
        # local line centre at channel velocity -v_los
        ref = integrate.quad(_gauss, lo, hi, args=(-v_los, sigma), epsabs=0, epsrel=1e-13,
                             limit=200)[0]
        assert phi[k] == pytest.approx(ref, rel=1e-9, abs=1e-300)


def test_band_sum_and_moments(oracle):
    sigma, dv = 2.0e4, 4.0e3
    n_ch = 200
    v_min = -0.5 * n_ch * dv
    v_los = 1.3e4
    phi = oracle.profile(n_ch, v_min, dv, v_los, sigma)
    assert phi.sum() == pytest.approx(1.0, abs=1e-14)          # band >> 6 sigma
    vc = v_min + (np.arange(n_ch) + 0.5) * dv
    mean = (vc * phi).sum()
    var = ((vc - mean) ** 2 * phi).sum()
    assert mean == pytest.approx(-v_los, abs=1e-6 * sigma)
    # Sheppard's correction: binned variance = sigma^2 + dv^2 / 12
    assert var == pytest.approx(sigma ** 2 + dv ** 2 / 12.0, rel=1e-6)


def test_approaching_gas_is_blue_shifted(oracle):
    phi = oracle.profile(64, -2.0e5, 6.25e3, +1.0e5, 2.0e4)
    vc = -2.0e5 + (np.arange(64) + 0.5) * 6.25e3
    assert vc[np.argmax(phi)] < 0.0
    # mirror symmetry of a symmetric band
    phim = oracle.profile(64, -2.0e5, 6.25e3, -1.0e5, 2.0e4)
    np.testing.assert_allclose(phi, phim[::-1], rtol=1e-12, atol=1e-300)


def test_far_wing_relative_accuracy(oracle):
    # channels 6..9 sigma away: the wing must keep relative accuracy
    sigma = 1.0e4
    phi = oracle.profile(4, 6.0 * sigma, sigma, 0.0, sigma)
    for k in range(4):
        lo, hi = (6 + k) * sigma, (7 + k) * sigma
        ref = integrate.quad(_gauss, lo, hi, args=(0.0, sigma), epsabs=0, epsrel=1e-13)[0]
        assert phi[k] == pytest.approx(ref, rel=1e-8)
