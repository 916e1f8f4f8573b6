"""Pins of the oracle's sub-iterations (Sect. 4 suggests updating the
populations of optically thick regions more often than the rest; the scheme
is our reading: after each full ALI iteration, n_sub sub-iterations of the
k_sub innermost shells -- line parameters, a ray simulation of the rays that
cross those shells over their steps inside them, each starting from the
intensity it carried into the region in the full iteration, the
equilibrium of those shells only -- with the populations outside and the
radiation entering the region held).

What fixes it:
  * the rays that cross a shell are exactly those whose tangent shell is at
    or inside it, and with unchanged line parameters their steps inside the
    region, started from the held intensities, give the region a full ray
    simulation's sums (the other rays never reach the region);
  * a region of every shell makes each sub-iteration a full iteration:
    n iterations with n_sub sub-iterations are (1 + n_sub) n plain ones,
    bit for bit;
  * the shells outside the region keep the populations of the full
    iteration, bit for bit;
  * no sub-iterations is the plain iteration, bit for bit;
  * the fixed point does not move: converged with and without
    sub-iterations, the populations agree to rounding;
  * on a cloud with an optically thick core in a thin envelope,
    sub-iterating the core reaches 1e-4 in T_ex in fewer full iterations
    (the speed-up the paper anticipates).
"""
import numpy as np

import loc_inputs as LI


def _thick_core(K=64, core=16, core_ab=1e-7, env_ab=1e-10):
    model = LI.cloud1d_two_level(K=K)
    ab = np.full(K, env_ab)
    ab[:core] = core_ab
    model["abundance"] = ab
    return model


def _iters_to(d, tol):
    k = int(np.argmax(d < tol))
    assert d[k] < tol
    return k + 1


def test_sub_rays_are_those_reaching_the_region(oracle):
    for model in (LI.cloud1d_rotor(K=40, n_ch=32), LI.cloud1d_rotor(K=40, n_ch=32, n_rays=57),
                  dict(LI.cloud1d_rotor(K=40, n_ch=32, n_rays=30), ray_power=2.0)):
        for k_sub in (1, 7, 23, 40):
            j_end = oracle.sub_rays_1d(model, k_sub)
            for j in range(model["n_rays"]):
                cells = oracle.paths_1d(model, j)[0]
                reaches = len(cells) > 0 and cells.min() < k_sub
                assert reaches == (j < j_end), (k_sub, j)


def test_region_sums_equal_the_full_simulation(oracle):
    """With unchanged line parameters, the region's steps started from the
    held intensities give the region the full simulation's sums."""
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.cloud1d_rotor(K=48, n_ch=40, n_rays=61)
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    full = oracle.march_1d(mol, model, Kp, S)
    k_sub = 13
    *stored, Ib = oracle.march_1d_sub(mol, model, Kp, S, k_sub, 0)
    for a, b in zip(stored, full):                  # storing changes nothing
        np.testing.assert_array_equal(a, b)
    part = oracle.march_1d_sub(mol, model, Kp, S, k_sub, 1, Ib)
    for a, b in zip(part, full):
        np.testing.assert_allclose(a[..., :k_sub], b[..., :k_sub], rtol=1e-12, atol=0)
    # outside the region nothing is accumulated
    assert np.all(part[2][k_sub:] == 0.0)


def test_whole_cloud_region_is_plain_iteration(oracle):
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.cloud1d_rotor(K=24, n_ch=48)
    x1, _ = oracle.iterate_1d(mol, model, 6)
    x2, _ = oracle.iterate_1d_sub(mol, model, 2, 2, 24)
    np.testing.assert_array_equal(x1, x2)
    x3, d3 = oracle.iterate_1d_sub(mol, model, 5, 0, 7)
    x4, d4 = oracle.iterate_1d(mol, model, 5)
    np.testing.assert_array_equal(x3, x4)
    np.testing.assert_array_equal(d3, d4)


def test_outside_the_region_keeps_the_full_iteration(oracle):
    mol = LI.two_level_molecule()
    model = _thick_core()
    x0 = oracle.lte_populations(mol, model["t_kin"])
    x_full, _ = oracle.iterate_1d(mol, model, 1, x0=x0)
    x_sub, _ = oracle.iterate_1d_sub(mol, model, 1, 3, 16, x0=x0)
    np.testing.assert_array_equal(x_sub[16:], x_full[16:])
    assert np.max(np.abs(x_sub[:16] - x_full[:16])) > 1e-6      # the region moved on


def test_same_fixed_point_and_fewer_full_iterations(oracle):
    mol = LI.two_level_molecule()
    model = _thick_core()
    x_p, d_p = oracle.iterate_1d(mol, model, 200)
    x_s, d_s = oracle.iterate_1d_sub(mol, model, 80, 4, 16)
    assert d_p[-1] < 1e-12 and d_s[-1] < 1e-12
    np.testing.assert_allclose(x_s, x_p, rtol=1e-9, atol=1e-15)
    n_plain, n_sub = _iters_to(d_p, 1e-4), _iters_to(d_s, 1e-4)
    assert n_sub * 2 < n_plain, (n_plain, n_sub)
