"""Hyperfine lines on the device against the oracle (Sect. 2.1: lines with
hyperfine structure and LTE between the components; the profile of such a
line is the strength-weighted sum of its components' channel fractions, each
shifted by its velocity offset).

Synthetic triplet on the J = 1-0 line of the rotor (offsets -1.1, 0, +0.7
km/s, strengths 0.2, 0.5, 0.3), as the paper's HCN test treats only the
lowest line's structure.  Tolerances as for plain lines: one ray simulation
2e-5 relative, T_ex 1e-4 after a fixed number of iterations, spectra 1e-4 of
the peak; with and without the channel window (which widens to hold every
component).
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


def _mol(n_levels=6):
    return LI.with_hyperfine(LI.rotor_molecule(n_levels=n_levels), line=0)


def _model():
    return LI.cloud1d_rotor(K=40, n_ch=96)


@pytest.mark.parametrize("window", [0.0, 8.0])
def test_hyperfine_radiation_matches_oracle(loc, oracle, window):
    mol, model = _mol(), _model()
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=window)
        sij, esc, norm = m.radiation()
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    rs, re_, rn = oracle.march_1d(mol, model, Kp, S)
    np.testing.assert_allclose(norm, rn, rtol=2e-5)
    np.testing.assert_allclose(sij, rs, rtol=2e-5, atol=1e-12 * np.abs(rs).max())
    np.testing.assert_allclose(esc, re_, rtol=2e-5)


def test_hyperfine_iterations_and_spectra_match_oracle(loc, oracle):
    mol, model = _mol(), _model()
    R = model["radius"][-1]
    p = [0.0, 0.3 * R, 0.8 * R]
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=10, window_sigmas=8.0)
        x = m.populations()
        spec = m.spectra(0, p)
    xr, _ = oracle.iterate_1d(mol, model, 10)
    tg, tr = oracle.tex(mol, x), oracle.tex(mol, xr)
    sel = xr[:, mol["line_u"]].T >= 1e-6
    assert np.max(np.abs(tg[sel] / tr[sel] - 1.0)) < 1e-4
    sref = oracle.spectra_1d(mol, model, xr, 0, p)
    peak = np.abs(sref).max(axis=1, keepdims=True)
    assert np.max(np.abs(spec - sref) / peak) < 1e-4
    # the multiplet differs from the plain line's spectrum
    plain = oracle.spectra_1d(LI.rotor_molecule(n_levels=6), model, xr, 0, p)
    assert np.max(np.abs(plain - sref) / peak) > 1e-2


def test_single_unshifted_component_equals_plain_line(loc):
    base = LI.rotor_molecule(n_levels=6)
    one = LI.with_hyperfine(base, line=0, offsets_kms=(0.0,), strengths=(1.0,))
    model = _model()
    out = []
    for mol in (base, one):
        with loc.Model(model, mol) as m:
            m.iterate(max_iter=4, window_sigmas=8.0, steps_per_chunk=-1)
            out.append(m.populations())
    np.testing.assert_allclose(out[1], out[0], rtol=2e-5, atol=1e-14)


def test_hyperfine_is_refused_where_it_is_not_built(loc):
    mol = _mol(4)
    with loc.Model(LI.small_grid3d(N=4, n_ch=16)) as m:
        with pytest.raises(loc.LocError) as e:
            m.set_molecule(mol)
        assert e.value.status == loc.LOC_EINVAL
    with loc.Server(max_slots=2) as srv:
        with pytest.raises(loc.LocError) as e:
            srv.submit(_model(), mol, max_iter=2)
        assert e.value.status == loc.LOC_EINVAL
    bad = dict(mol, hf_w=np.array([0.5, 0.2, 0.2]))
    with loc.Model(_model()) as m:
        with pytest.raises(loc.LocError) as e:
            m.set_molecule(bad)
        assert e.value.status == loc.LOC_EINVAL
