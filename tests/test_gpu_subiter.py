"""Sub-iterations of an inner region on the device against the oracle's
(Sect. 4: populations of optically thick regions updated more often; after
each full ALI iteration, sub-iterations of the k_sub innermost shells --
line parameters, the region's steps of the rays that reach it started from
the intensities those rays carried into it in the full iteration, the
region's equilibrium -- with the populations outside and the radiation
entering the region held).

Tolerances as for the plain iteration: T_ex within 1e-4 of the oracle after
a fixed number of iterations; a region of every shell equals the plain
iteration on the device (2e-5, FP32 sums in another order); with a
tolerance the device stops at the oracle's iteration.
"""
import numpy as np
import pytest

import loc_inputs as LI

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


def _thick_core(K=64, core=16):
    model = LI.cloud1d_two_level(K=K)
    ab = np.full(K, 1e-10)
    ab[:core] = 1e-7
    model["abundance"] = ab
    return model


def _tex_err(oracle, mol, x, x_ref):
    tg, tr = oracle.tex(mol, x), oracle.tex(mol, x_ref)
    sel = x_ref[:, mol["line_u"]].T >= 1e-6
    return float(np.max(np.abs(tg[sel] / tr[sel] - 1.0)))


CASES = {
    "two_level_thick_core": (LI.two_level_molecule, _thick_core, 16, 3),
    "rotor_more_rays": (lambda: LI.rotor_molecule(n_levels=8),
                        lambda: LI.cloud1d_rotor(K=48, n_ch=64, n_rays=71), 11, 2),
    "rotor_power_rays": (lambda: LI.rotor_molecule(n_levels=8),
                         lambda: dict(LI.cloud1d_rotor(K=48, n_ch=64, n_rays=40), ray_power=1.7), 20, 2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sub_iterations_match_oracle(loc, oracle, case):
    mk_mol, mk_model, k_sub, n_sub = CASES[case]
    mol, model = mk_mol(), mk_model()
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=5, window_sigmas=8.0, sub_iters=n_sub, sub_shells=k_sub)
        assert rep["iterations"] == 5
        x = m.populations()
    x_ref, _ = oracle.iterate_1d_sub(mol, model, 5, n_sub, k_sub)
    assert _tex_err(oracle, mol, x, x_ref) < 1e-4


def test_whole_cloud_region_equals_plain_iteration(loc):
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.cloud1d_rotor(K=32, n_ch=48)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=6, window_sigmas=8.0, steps_per_chunk=-1)
        x_plain = m.populations()
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=2, window_sigmas=8.0, sub_iters=2, sub_shells=32)
        x_sub = m.populations()
    np.testing.assert_allclose(x_sub, x_plain, rtol=2e-5, atol=1e-14)


def test_tolerance_stops_with_the_oracle(loc, oracle):
    mol, model = LI.two_level_molecule(), _thick_core()
    _, d = oracle.iterate_1d_sub(mol, model, 30, 4, 16)
    k = int(np.argmax(d < 1e-4))
    assert d[k] < 8e-5 and d[k - 1] > 1.25e-4          # away from the threshold
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=100, tol_tex=1e-4, window_sigmas=8.0, sub_iters=4, sub_shells=16)
    assert rep["status"] == 0 and rep["iterations"] == k + 1
    with loc.Model(model, mol) as m:
        plain = m.iterate(max_iter=100, tol_tex=1e-4, window_sigmas=8.0)
    assert plain["status"] == 0 and plain["iterations"] > 2 * rep["iterations"]


def test_sub_iteration_options_are_checked(loc):
    mol = LI.two_level_molecule()
    with loc.Model(_thick_core(K=16, core=4), mol) as m:
        for bad in (dict(sub_iters=2, sub_shells=0), dict(sub_iters=2, sub_shells=17),
                    dict(sub_iters=2, sub_shells=4, level_cutoff=1e-8), dict(sub_iters=-1)):
            with pytest.raises(loc.LocError) as e:
                m.iterate(max_iter=1, **bad)
            assert e.value.status == loc.LOC_EINVAL
    with loc.Model(LI.small_grid3d(N=4, n_ch=16), LI.rotor_molecule(n_levels=4)) as m:
        with pytest.raises(loc.LocError) as e:
            m.iterate(max_iter=1, sub_iters=1, sub_shells=1)
        assert e.value.status == loc.LOC_EINVAL
