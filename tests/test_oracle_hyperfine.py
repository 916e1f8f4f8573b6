"""Pins of the oracle's hyperfine lines (Sect. 2.1: lines with hyperfine
structure and LTE between the components; the profile reading is ours: with
the components' relative populations fixed, the line is one transition
whose channel profile is the strength-weighted sum of the component
profiles, each shifted by its velocity offset).

What fixes it:
  * one component at offset 0 with strength 1 is the plain line, bit for
    bit (march, iterations, spectra);
  * a uniform static sphere with fixed populations has the closed-form
    spectrum I(p) = n_bg e^-tau + S (1 - e^-tau) with tau_k = K s(p) times
    the sum over components of w_c times the Gaussian's channel fraction
    shifted by v_c -- written here from scipy's erf, independently of the
    oracle's profile routine (a wrong sign of the offset or a dropped
    weight breaks it);
  * in the optically thin limit the spectrum of the multiplet is the
    strength-weighted sum of the spectra of single shifted components;
  * the strengths sum to one, so a static cloud's NORM and the LTE fixed
    point do not depend on the hyperfine structure.
"""
import numpy as np
from scipy.special import erf

import loc_inputs as LI

H = 6.62607015e-27
KB = 1.380649e-16
AMU = 1.66053906660e-24


def test_single_unshifted_component_is_the_plain_line(oracle):
    mol = LI.rotor_molecule(n_levels=6)
    hf = LI.with_hyperfine(mol, line=1, offsets_kms=(0.0,), strengths=(1.0,))
    model = LI.cloud1d_rotor(K=24, n_ch=64)
    x0, d0 = oracle.iterate_1d(mol, model, 4)
    x1, d1 = oracle.iterate_1d(hf, model, 4)
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(d0, d1)
    p = [0.0, 0.3 * model["radius"][-1]]
    np.testing.assert_array_equal(oracle.spectra_1d(mol, model, x0, 1, p),
                                  oracle.spectra_1d(hf, model, x1, 1, p))


def test_uniform_sphere_multiplet_closed_form(oracle):
    mol = LI.with_hyperfine(LI.two_level_molecule(), offsets_kms=(-1.1, 0.0, 0.7),
                            strengths=(0.2, 0.5, 0.3))
    m = LI.uniform_sphere(K=7, n_ch=48, abundance=2e-8, half_width_kms=3.0)
    x = np.tile(np.array([0.4, 0.6]), (7, 1))
    R = m["radius"][-1]
    p = np.array([0.0, 0.2 * R, 0.55 * R, 0.93 * R, 1.01 * R])
    T = oracle.spectra_1d(mol, m, x, 0, p)
    Kp, S = oracle.line_params(mol, m, x)
    sig = np.sqrt(m["sigma_turb"][0] ** 2 + KB * m["t_kin"][0] / (mol["mass_amu"] * AMU))
    edges = m["v_min"] + m["dv"] * np.arange(m["n_ch"] + 1)
    phi = np.zeros(m["n_ch"])
    for vc, wc in zip(mol["hf_v"], mol["hf_w"]):
        # component at velocity vc: the Gaussian centred at vc, channel fractions
        cdf = 0.5 * (1.0 + erf((edges - vc) / (np.sqrt(2.0) * sig)))
        phi += wc * np.diff(cdf)
    nu = mol["line_nu"][0]
    nbg = 1.0 / np.expm1(H * nu / (KB * m["t_bg"]))
    for ip, pp in enumerate(p):
        L = 2.0 * np.sqrt(max(R * R - pp * pp, 0.0))
        tau = Kp[0, 0] * phi * L
        n = nbg * np.exp(-tau) - S[0, 0] * np.expm1(-tau)
        np.testing.assert_allclose(T[ip], H * nu / KB * (n - nbg), rtol=1e-9, atol=1e-12)
    # the three components are resolved: the spectrum peaks at the strongest
    assert abs(m["v_min"] + (np.argmax(T[0]) + 0.5) * m["dv"]) < 2 * m["dv"]


def test_thin_multiplet_is_the_weighted_sum_of_components(oracle):
    base = LI.two_level_molecule()
    offs, ws = (-1.1, 0.0, 0.7), (0.2, 0.5, 0.3)
    mol = LI.with_hyperfine(base, offsets_kms=offs, strengths=ws)
    m = LI.cloud1d_two_level(K=16, abundance=1e-16, half_width_kms=3.0)
    x = oracle.lte_populations(base, m["t_kin"])
    p = [0.0, 0.4 * m["radius"][-1]]
    T = oracle.spectra_1d(mol, m, x, 0, p)
    ref = np.zeros_like(T)
    for vc, wc in zip(offs, ws):
        one = LI.with_hyperfine(base, offsets_kms=(vc,), strengths=(1.0,))
        ref += wc * oracle.spectra_1d(one, m, x, 0, p)
    # thin limit: linear in the profile up to O(tau) relative
    np.testing.assert_allclose(T, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_static_norm_and_lte_fixed_point(oracle):
    base = LI.two_level_molecule()
    mol = LI.with_hyperfine(base)
    m = LI.uniform_sphere(K=8, n_ch=64, abundance=1e-9, half_width_kms=3.0, n_h2=1e9)
    x = oracle.lte_populations(base, m["t_kin"])
    Kp, S = oracle.line_params(base, m, x)
    _, _, n0 = oracle.march_1d(base, m, Kp, S)
    _, _, n1 = oracle.march_1d(mol, m, Kp, S)
    np.testing.assert_array_equal(n0, n1)
    # thermalised by collisions: LTE populations whatever the profile
    xh, _ = oracle.iterate_1d(mol, m, 5)
    np.testing.assert_allclose(xh, x, rtol=2e-5)
