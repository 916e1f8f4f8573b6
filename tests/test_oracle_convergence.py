"""Pins of the oracle's convergence metric (Sect. 3.3.2 follows the change
of the excitation temperatures between iterations; the metric is the
largest relative change of T_ex over cells and over lines whose upper level
holds at least 1e-6 of the molecules).

What fixes it: populations are built from chosen excitation temperatures by
the Boltzmann ratio of each line, x_u / x_l = (g_u / g_l) exp(-h nu / (k T)),
level by level up the rotor ladder.  So the T_ex of every line is known by
construction, and the metric must return the largest |T_new - T_old| /
|T_old| of the chosen numbers.  A swapped weight ratio, a sign slip in the
exponent, a mask taken on the wrong level or population set, or a relative
change divided by the new T_ex instead of the old one each moves a value
below by more than the tolerance.
"""
import numpy as np

import loc_inputs as LI

H = 6.62607015e-27
KB = 1.380649e-16


def _pops(mol, tex_per_line):
    """Populations of one cell whose line t (J = t+1 -> t) has excitation
    temperature tex_per_line[t]; None marks an empty upper level (and every
    level above it)."""
    L = len(mol["g"])
    x = np.zeros(L)
    x[0] = 1.0
    for t, T in enumerate(tex_per_line):
        u, l = mol["line_u"][t], mol["line_l"][t]
        if T is None or x[l] == 0.0:
            x[u] = 0.0
            continue
        x[u] = x[l] * mol["g"][u] / mol["g"][l] * np.exp(-H * mol["line_nu"][t] / (KB * T))
    return x / x.sum()


def test_tex_recovers_the_chosen_temperatures(oracle):
    mol = LI.rotor_molecule(n_levels=4)
    chosen = [[12.0, 9.0, 7.5], [30.0, -40.0, 25.0]]   # cell 1, line 1: inverted levels
    x = np.array([_pops(mol, c) for c in chosen])
    tex = oracle.tex(mol, x)                              # [line][cell]
    np.testing.assert_allclose(tex.T, np.array(chosen), rtol=1e-12)


def test_metric_is_the_largest_relative_change(oracle):
    mol = LI.rotor_molecule(n_levels=4)
    old = [[10.0, 10.0, 10.0], [20.0, 20.0, 20.0], [-50.0, 15.0, 15.0]]
    new = [[10.5, 10.2, 9.9], [20.0, 19.4, 20.0], [-45.0, 15.0, 15.3]]
    # relative changes by construction: 0.05, 0.02, 0.01 / 0, 0.03, 0 / 0.1, 0, 0.02
    xo = np.array([_pops(mol, c) for c in old])
    xn = np.array([_pops(mol, c) for c in new])
    assert (xn[:, 1:] >= 1e-6).all()                      # every line monitored
    d = oracle.max_rel_dtex(mol, xo, xn)
    assert abs(d - 0.1) < 1e-12                           # the maser line, |dT| / |T_old|
    # without the inverted cell the largest change is cell 0, line 0
    d2 = oracle.max_rel_dtex(mol, xo[:2], xn[:2])
    assert abs(d2 - 0.05) < 1e-12
    # relative to the old value, not the new one: 0.5 / 10 (not 0.5 / 10.5)
    d3 = oracle.max_rel_dtex(mol, xo[:1], xn[:1])
    assert abs(d3 - 0.05) < 1e-12
    # no change at all
    assert oracle.max_rel_dtex(mol, xo, xo) == 0.0


def test_metric_skips_lines_with_an_almost_empty_upper_level(oracle):
    mol = LI.rotor_molecule(n_levels=4)
    # line 2 (J = 3 -> 2, h nu / k = 16.6 K) at T_ex ~ 1 K leaves x_3 < 1e-6:
    # its 20 % change must not count; the monitored lines change by 1 %
    old = [[10.0, 8.0, 1.00]]
    new = [[10.1, 8.0, 1.20]]
    xo = np.array([_pops(mol, c) for c in old])
    xn = np.array([_pops(mol, c) for c in new])
    assert xn[0, 3] < 1e-6 and xn[0, 2] >= 1e-6
    d = oracle.max_rel_dtex(mol, xo, xn)
    assert abs(d - 0.01) < 1e-12
    # the mask looks at the new populations: the same pair in reverse order
    # (upper level of the "new" set above 1e-6) does count
    hi_old = [[10.0, 8.0, 6.0]]
    hi_new = [[10.1, 8.0, 4.8]]
    xo2 = np.array([_pops(mol, c) for c in hi_old])
    xn2 = np.array([_pops(mol, c) for c in hi_new])
    assert xn2[0, 3] >= 1e-6
    assert abs(oracle.max_rel_dtex(mol, xo2, xn2) - 0.2) < 1e-12


def test_metric_skips_lines_without_an_old_temperature(oracle):
    mol = LI.rotor_molecule(n_levels=4)
    # old populations have an empty J = 3 level (T_ex of line 2 undefined,
    # reported as 0): the line is skipped although it is populated now
    xo = np.array([_pops(mol, [10.0, 10.0, None])])
    xn = np.array([_pops(mol, [10.3, 10.0, 30.0])])
    assert xo[0, 3] == 0.0 and xn[0, 3] >= 1e-6
    assert oracle.tex(mol, xo)[2, 0] == 0.0
    d = oracle.max_rel_dtex(mol, xo, xn)
    assert abs(d - 0.03) < 1e-12
