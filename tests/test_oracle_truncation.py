"""Pins of the oracle's per-cell line truncation (Sect. 4 proposes computing,
cell by cell, only the transitions whose levels are populated; the rule --
a line is off in a cell when both of its levels hold less than the cutoff,
and an off line has no opacity there and takes the background field,
J = n_bg with beta = 1 -- is our reading).

What fixes it:
  * a cutoff below every population switches nothing off: bit-identical to
    the untruncated iteration;
  * two-level molecule with every line off: the level ratio is the
    closed-form solution of the two-level balance under the CMB alone,
    x_u / x_l = ((g_u/g_l) A n_bg + C_lu) / (A (1 + n_bg) + C_ul), whatever
    the optical depth (the untruncated thick cloud traps radiation and
    differs, so the pin separates the two branches);
  * multi-level rotor: truncating levels below 1e-8 leaves the excitation of
    every monitored line (x_u >= 1e-6) unchanged to 1e-9 and switches a
    sizeable share of (line, cell) pairs off.
"""
import numpy as np

import loc_inputs as LI

H = 6.62607015e-27
KB = 1.380649e-16


def test_cutoff_below_every_population_changes_nothing(oracle):
    mol = LI.rotor_molecule(n_levels=12)
    model = LI.cloud1d_rotor(K=24, n_ch=48)
    x0, d0 = oracle.iterate_1d(mol, model, 4)
    x1, d1 = oracle.iterate_1d(mol, model, 4, level_cutoff=1e-300)
    assert oracle.line_off(mol, x1, 1e-300).sum() == 0
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(d0, d1)


def test_two_level_all_lines_off_closed_form(oracle):
    mol = LI.two_level_molecule()
    model = LI.cloud1d_two_level(K=16, density_scale=30.0)   # optically thick core
    # both populations are below 1 in every cell: the line is off everywhere
    x, _ = oracle.iterate_1d(mol, model, 1, level_cutoff=1.0)
    nu, A = mol["line_nu"][0], mol["line_A"][0]
    gl, gu = mol["g"]
    n_bg = 1.0 / np.expm1(H * nu / (KB * model["t_bg"]))
    c_ul = model["n_h2"] * mol["coll_k"][0]
    c_lu = c_ul * (gu / gl) * np.exp(-(mol["energy_K"][1] - mol["energy_K"][0]) / model["t_kin"])
    ratio = ((gu / gl) * A * n_bg + c_lu) / (A * (1.0 + n_bg) + c_ul)
    np.testing.assert_allclose(x[:, 1] / x[:, 0], ratio, rtol=1e-12)
    np.testing.assert_allclose(x.sum(axis=1), 1.0, rtol=1e-14)
    # untruncated, the trapped line radiation raises the upper level
    y, _ = oracle.iterate_1d(mol, model, 1)
    assert np.max(y[:, 1] / y[:, 0] / ratio) > 1.01


def test_truncating_empty_levels_keeps_populated_lines(oracle):
    mol = LI.rotor_molecule(n_levels=20)
    model = LI.cloud1d_rotor(K=32, n_ch=64)
    x0, _ = oracle.iterate_1d(mol, model, 10)
    x1, _ = oracle.iterate_1d(mol, model, 10, level_cutoff=1e-8)
    off = oracle.line_off(mol, x1, 1e-8)
    assert 0.2 < off.mean() < 0.9
    # the mask is the rule itself: both levels below the cutoff
    lo = x1[:, mol["line_l"]].T < 1e-8
    up = x1[:, mol["line_u"]].T < 1e-8
    np.testing.assert_array_equal(off.astype(bool), lo & up)
    t0, t1 = oracle.tex(mol, x0), oracle.tex(mol, x1)
    sel = x0[:, mol["line_u"]].T >= 1e-6
    assert np.max(np.abs(t1[sel] / t0[sel] - 1.0)) < 1e-9
    np.testing.assert_allclose(x1.sum(axis=1), 1.0, rtol=1e-12)


def test_grid_and_octree_truncated_loops_reduce_to_the_plain_ones(oracle):
    """The truncated 3D iterations (composed from the same steps as the plain
    loops) are bit-identical to them when nothing is below the cutoff, and
    a 1e-8 cutoff switches lines off in the 14-level rotor's cold cells."""
    mol = LI.rotor_molecule(n_levels=14)
    g = LI.small_grid3d(N=4, n_ch=16, nside=1, abundance=3e-4)
    x0, d0 = oracle.iterate_grid3d(mol, g, 2)
    x1, d1 = oracle.iterate_grid3d(mol, g, 2, level_cutoff=1e-300)
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(d0, d1)
    o = LI.small_octree(N=4, levels=2, refine_frac=0.3, nside=1, n_ch=16, abundance=1e-4)
    y0, e0 = oracle.iterate_octree(mol, o, 2)
    y1, e1 = oracle.iterate_octree(mol, o, 2, level_cutoff=1e-300)
    np.testing.assert_array_equal(y0, y1)
    np.testing.assert_array_equal(e0, e1)
    y2, _ = oracle.iterate_octree(mol, o, 2, level_cutoff=1e-8)
    assert oracle.line_off(mol, y2, 1e-8).mean() > 0.1
