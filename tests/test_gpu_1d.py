"""GPU parity of the 1D path (Sect. 2, 2.1) against the FP64 oracle, through
the C ABI.

Tolerances: the march runs in FP32 (profile, optical depth, intensity);
per-cell accumulators are FP32 sums of O(100) positive terms, so a single
ray simulation agrees with the oracle to ~1e-5 relative (the bar here is
2e-5 for SIJ/ESC/NORM).  Excitation temperatures after a fixed number of
iterations and emergent spectra must agree to 1e-4 relative (spectra:
relative to the spectrum's peak), the accuracy target of the method.
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


def _tex_err(mol, x_ref, m, oracle, mask_pop=1e-6):
    tref = oracle.tex(mol, x_ref)
    worst = 0.0
    for t in range(tref.shape[0]):
        tg = m.tex(t)
        u = mol["line_u"][t]
        sel = x_ref[:, u] >= mask_pop
        if sel.any():
            worst = max(worst, float(np.max(np.abs(tg[sel] / tref[t, sel] - 1.0))))
    return worst


@pytest.mark.parametrize("precision", ["fp32", "fp64acc"])
def test_march_radiation_matches_oracle_two_level(loc, oracle, precision):
    mol = LI.two_level_molecule()
    model = LI.cloud1d_two_level()
    with loc.Model(model, mol) as m:
        m.march(precision=precision)
        sij, esc, norm = m.radiation()
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    rs, re_, rn = oracle.march_1d(mol, model, Kp, S)
    np.testing.assert_allclose(norm, rn, rtol=2e-5)
    np.testing.assert_allclose(sij, rs, rtol=2e-5)
    np.testing.assert_allclose(esc, re_, rtol=2e-5)


def test_two_level_iterations_match_oracle(loc, oracle):
    mol = LI.two_level_molecule()
    model = LI.cloud1d_two_level()
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=20)
        assert rep["iterations"] == 20
        assert rep["segments"] == 32 * 33
        x_ref, d_ref = oracle.iterate_1d(mol, model, 20)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4
        np.testing.assert_allclose(m.populations(), x_ref, rtol=1e-4)
        # emergent spectra at every ray's impact parameter and at p = 0
        R = model["radius"][-1]
        p = np.concatenate([[0.0], (np.arange(32) + 0.5) * R / 32, [1.2 * R]])
        T = m.spectra(0, p)
    Tref = oracle.spectra_1d(mol, model, x_ref, 0, p)
    peak = np.abs(Tref).max(axis=1, keepdims=True)
    peak[peak == 0] = 1.0
    assert np.max(np.abs(T - Tref) / peak) < 1e-4


def test_rotor_full_size_fifty_iterations(loc, oracle):
    """1D rotor cloud at its full size (256 shells, 12 levels, 256 channels),
    50 ALI iterations, FP32 march vs FP64 oracle."""
    mol = LI.rotor_molecule()
    model = LI.cloud1d_rotor()
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=50, window_sigmas=0.0)
        x_ref, _ = oracle.iterate_1d(mol, model, 50)
        err = _tex_err(mol, x_ref, m, oracle)
        T = m.spectra(0, [0.0, 0.5 * model["radius"][-1]])
    assert rep["iterations"] == 50
    assert err < 1e-4, err
    Tref = oracle.spectra_1d(mol, model, x_ref, 0, [0.0, 0.5 * model["radius"][-1]])
    assert np.max(np.abs(T - Tref)) / np.abs(Tref).max() < 1e-4


@pytest.mark.parametrize("window", [0.0, 8.0])
@pytest.mark.parametrize("lines_per_pass", [0, 1, 5])
def test_rotor_modes_match_oracle(loc, oracle, window, lines_per_pass):
    mol = LI.rotor_molecule(n_levels=8)
    model = LI.cloud1d_rotor(K=40, n_ch=96)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=8, window_sigmas=window, lines_per_pass=lines_per_pass)
        x_ref, _ = oracle.iterate_1d(mol, model, 8)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4


@pytest.mark.parametrize("run", [-1, 1, 7, 16, 33])
@pytest.mark.parametrize("window,precision", [(0.0, "fp32"), (8.0, "fp32"), (8.0, "fp64acc")])
def test_runs_of_steps_match_oracle(loc, oracle, run, window, precision):
    """Rays cut into runs of `run` steps (affine map per run, scan along the
    ray, march from each run's entering intensity) give the whole-ray
    accumulators: one-step runs, odd lengths that leave a ragged last run,
    runs longer than the short rays."""
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.cloud1d_rotor(K=48, n_ch=80, n_rays=40)
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=window, precision=precision, steps_per_chunk=run, lines_per_pass=2)
        sij, esc, norm = m.radiation()
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    rs, re_, rn = oracle.march_1d(mol, model, Kp, S)
    np.testing.assert_allclose(norm, rn, rtol=2e-5)
    np.testing.assert_allclose(sij, rs, rtol=2e-5, atol=1e-12 * np.abs(rs).max())
    np.testing.assert_allclose(esc, re_, rtol=2e-5)


def test_runs_full_size_autotuned(loc, oracle):
    """Full-size rotor cloud with the autotuned launch shape (lines per warp
    and run length) over 50 iterations with the channel window."""
    mol = LI.rotor_molecule()
    model = LI.cloud1d_rotor()
    with loc.Model(model, mol) as m:
        per, run, ms = m.autotune(window_sigmas=8.0)
        assert ms > 0 and (run == -1 or run in (8, 16, 32, 64, 128))      # the candidates
        m.reset()
        m.iterate(max_iter=50, window_sigmas=8.0)
        x_ref, _ = oracle.iterate_1d(mol, model, 50)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4
        # every fixed run length from the same state agrees with whole rays
        m.reset()
        m.march(window_sigmas=8.0, steps_per_chunk=-1)
        ref = m.radiation()
        for run in (16, 64):
            m.march(window_sigmas=8.0, steps_per_chunk=run)
            got = m.radiation()
            for a, b in zip(got, ref):
                np.testing.assert_allclose(a, b, rtol=2e-5, atol=1e-12 * np.abs(b).max())


def test_lambda_iteration_and_fp64_accumulation(loc, oracle):
    mol = LI.two_level_molecule()
    model = LI.cloud1d_two_level(K=24, abundance=1e-8)
    for ali in (True, False):
        for prec in ("fp32", "fp64acc"):
            with loc.Model(model, mol) as m:
                m.iterate(max_iter=10, ali=ali, precision=prec)
                x_ref, _ = oracle.iterate_1d(mol, model, 10, ali=ali)
                assert _tex_err(mol, x_ref, m, oracle) < 1e-4


@pytest.mark.parametrize("K,n_rays,n_ch", [(1, 1, 1), (1, 7, 33), (3, 2, 64), (9, 31, 31),
                                           (64, 64, 1024), (300, 300, 40)])
def test_edge_shapes(loc, oracle, K, n_rays, n_ch):
    """Single shell, fewer or more rays than shells (shells without rays get
    the background), one channel, the maximum channel count, ragged channel
    counts that leave partial warps."""
    mol = LI.rotor_molecule(n_levels=4)
    model = LI.cloud1d_rotor(K=K, n_ch=n_ch, n_rays=n_rays)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=3)
        x_ref, _ = oracle.iterate_1d(mol, model, 3)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4


def test_convergence_stop_and_resume(loc, oracle):
    mol = LI.two_level_molecule()
    model = LI.cloud1d_two_level()
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=200, tol_tex=1e-4)
        assert rep["status"] == loc.LOC_OK
        assert rep["max_rel_dtex"] < 1e-4
        assert rep["iterations"] < 200
        x_conv = m.populations()
        # checkpoint / resume: two more iterations from the saved state
        m.iterate(max_iter=2)
        x_a = m.populations()
        m.set_populations(x_conv)
        m.iterate(max_iter=2)
        np.testing.assert_allclose(m.populations(), x_a, rtol=1e-6)
    # not converged within max_iter -> LOC_ENOTCONV with the work done
    with loc.Model(model, mol) as m:
        rep = m.iterate(max_iter=2, tol_tex=1e-12)
        assert rep["status"] == loc.LOC_ENOTCONV and rep["iterations"] == 2


def test_invalid_arguments(loc):
    mol = LI.two_level_molecule()
    good = LI.cloud1d_two_level(K=4)
    bad = dict(good)
    bad["radius"] = good["radius"][::-1].copy()
    with pytest.raises(loc.LocError) as e:
        loc.Model(bad, mol)
    assert e.value.status == loc.LOC_EINVAL
    bad = dict(good)
    bad["n_ch"] = 2000
    with pytest.raises(loc.LocError):
        loc.Model(bad, mol)
    with loc.Model(good) as m:
        with pytest.raises(loc.LocError) as e:
            m.iterate(max_iter=1)
        assert e.value.status == loc.LOC_ESTATE
        m.set_molecule(mol)
        with pytest.raises(loc.LocError):
            m.iterate(max_iter=0)
        with pytest.raises(loc.LocError):
            m.tex(5)
        with pytest.raises(loc.LocError):
            m.set_populations(np.zeros(3))


def test_duplicate_level_pairs_rejected(loc):
    """A molecule with two lines (or two collision entries) on the same pair
    of levels is rejected by loc_set_molecule."""
    rot = LI.rotor_molecule(n_levels=4)
    good = LI.cloud1d_two_level(K=4)
    dup_line = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rot.items()}
    dup_line["line_u"] = dup_line["line_u"].copy()
    dup_line["line_l"] = dup_line["line_l"].copy()
    dup_line["line_u"][1], dup_line["line_l"][1] = dup_line["line_l"][0], dup_line["line_u"][0]
    dup_coll = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rot.items()}
    dup_coll["coll_u"][1], dup_coll["coll_l"][1] = dup_coll["coll_u"][0], dup_coll["coll_l"][0]
    with loc.Model(good) as m:
        for bad in (dup_line, dup_coll):
            with pytest.raises(loc.LocError) as e:
                m.set_molecule(bad)
            assert e.value.status == loc.LOC_EINVAL
        m.set_molecule(rot)
        m.iterate(max_iter=1)


@pytest.mark.parametrize("ray_power,steps_per_chunk", [(2.0, -1), (2.0, 16), (0.6, 0)])
def test_power_law_rays_match_oracle(loc, oracle, ray_power, steps_per_chunk):
    """Impact parameters following a power law (Sect. 2.1): ray geometry,
    weights, one ray simulation and the ALI iterations agree with the oracle;
    whole rays and runs of steps alike."""
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.cloud1d_rotor(K=40, n_ch=96)
    model["n_rays"] = 60
    model["ray_power"] = ray_power
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=8.0, steps_per_chunk=steps_per_chunk)
        sij, esc, norm = m.radiation()
        x = oracle.lte_populations(mol, model["t_kin"])
        Kp, S = oracle.line_params(mol, model, x)
        rs, re_, rn = oracle.march_1d(mol, model, Kp, S)
        np.testing.assert_allclose(norm, rn, rtol=2e-5)
        np.testing.assert_allclose(sij, rs, rtol=5e-5, atol=1e-7 * np.abs(rs).max())
        np.testing.assert_allclose(esc, re_, rtol=5e-5, atol=1e-7 * np.abs(re_).max())
        m.reset()
        m.iterate(max_iter=12, window_sigmas=8.0, steps_per_chunk=steps_per_chunk)
        x_ref, _ = oracle.iterate_1d(mol, model, 12)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4
    bad = dict(model)
    bad["ray_power"] = -1.0
    with pytest.raises(loc.LocError):
        loc.Model(bad, mol)


def test_level_cutoff_truncates_lines_within_tolerance(loc, oracle):
    """Per-cell line truncation (the paper's suggested optimisation, Sect. 4):
    lines whose two levels are empty in a cell are left out there.  The
    populations match the oracle's truncated iteration level by level (down
    to 1e-20), the monitored excitation temperatures also match the
    untruncated oracle, the ray simulation computes fewer updates (line
    groups of 4, so that whole groups fall below the cutoff in the cold
    inner cells), and the spectra (which never truncate) agree."""
    mol = LI.rotor_molecule(n_levels=20)
    model = LI.cloud1d_rotor(K=64, n_ch=128)
    n_iter = 20
    kw = dict(max_iter=n_iter, window_sigmas=8.0, profile=True, lines_per_pass=4)
    with loc.Model(model, mol) as m:
        full = m.iterate(**kw)
        m.reset()
        cut = m.iterate(level_cutoff=1e-8, **kw)
        x_ref, _ = oracle.iterate_1d(mol, model, n_iter)
        assert _tex_err(mol, x_ref, m, oracle) < 1e-4
        x_cut, _ = oracle.iterate_1d(mol, model, n_iter, level_cutoff=1e-8)
        assert _tex_err(mol, x_cut, m, oracle) < 1e-4
        xg = m.populations()
        sel = x_cut > 1e-20
        assert np.max(np.abs(xg[sel] / x_cut[sel] - 1.0)) < 1e-3
        R = model["radius"][-1]
        p = np.array([0.0, 0.3 * R, 0.8 * R])
        T = m.spectra(0, p)
        with pytest.raises(loc.LocError):
            m.iterate(max_iter=1, level_cutoff=1e-3)
    assert cut["computed_updates"] < 0.9 * full["computed_updates"]
    Tref = oracle.spectra_1d(mol, model, x_ref, 0, p)
    peak = np.abs(Tref).max(axis=1, keepdims=True)
    assert np.max(np.abs(T - Tref) / peak) < 1e-4
