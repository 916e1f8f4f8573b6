"""GPU parity of the 3D emergent maps (loc_map3d: the final line-of-sight
integration of Sect. 2 for grids and octrees) against the FP64 oracle,
through the C ABI.

Both sides take the same populations (read back from the device after a
few ALI iterations).  Tolerance: |dT| <= 1e-4 max|T| over each map (the
spectra tolerance, relative to the peak).  Small models are compared pixel
by pixel for every level and several directions; the full-size grid and
octree on sampled pixels (the oracle computes only those).
"""
import numpy as np
import pytest

import loc_inputs as LI

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def loc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_12609_gb300 import build, loc as L
    build.build()
    L.load()
    return L


def _check(T_gpu, T_ref, rows=None):
    if rows is not None:
        T_gpu, T_ref = T_gpu[rows], T_ref[rows]
    peak = np.abs(T_ref).max()
    assert peak > 0
    err = np.abs(T_gpu - T_ref).max() / peak
    assert err < TOL, f"map mismatch {err:.3g}"


@pytest.mark.parametrize("n_ch", [16, 70])
def test_grid_maps_match_oracle(loc, oracle, n_ch):
    mol = LI.rotor_molecule(n_levels=5)
    model = LI.small_grid3d(N=6, n_ch=n_ch, nside=1, abundance=3e-6)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=2, window_sigmas=8.0)
        x = m.populations()
        for d in (0, 5, 11):
            for t in (0, 2):
                _check(m.map3d(t, d), oracle.map_3d(mol, model, x, t, model["dirs"][d]))


def test_octree_maps_match_oracle(loc, oracle):
    mol = LI.rotor_molecule(n_levels=4)
    model = LI.small_octree(N=4, levels=2, n_ch=20, nside=1, refine_frac=0.3)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=2, window_sigmas=8.0)
        x = m.populations()
        for d in (1, 6):
            for lam in range(model["levels"] + 1):
                T = m.map3d(1, d, level=lam)
                assert T.shape == ((4 << lam) ** 2, 20)
                _check(T, oracle.map_3d(mol, model, x, 1, model["dirs"][d], lam=lam))


def test_lte_maps_match_oracle(loc, oracle):
    """The LTE variant of the maps (the paper contrasts LTE and non-LTE line
    emission, Sect. 3.3): populations reset to Boltzmann at T_kin on the
    device, compared with the oracle's own LTE populations and map."""
    mol = LI.rotor_molecule(n_levels=5)
    for model in (LI.small_grid3d(N=6, n_ch=24, nside=1, abundance=3e-6),
                  LI.small_octree(N=4, levels=2, n_ch=20, nside=1, refine_frac=0.3)):
        with loc.Model(model, mol) as m:
            m.iterate(max_iter=2, window_sigmas=8.0)
            m.reset()
            x = m.populations()
            leaf = (model["refine"] == 0) if model["geometry"] == "octree3d" else slice(None)
            x_lte = oracle.lte_populations(mol, np.asarray(model["t_kin"])[leaf])
            np.testing.assert_allclose(x, x_lte, rtol=1e-10, atol=1e-300)
            lam = model.get("levels", 0)
            for d in (0, 3):
                _check(m.map3d(0, d, level=lam),
                       oracle.map_3d(mol, model, x_lte, 0, model["dirs"][d], lam=lam))


def test_grid_full_size_sampled(loc, oracle):
    model = LI.grid3d_cloud()
    mol = LI.rotor_molecule()
    stride = 997
    with loc.Model(model, mol) as m:
        x = m.populations()
        T = m.map3d(0, 21)
    ref = oracle.map_3d(mol, model, x, 0, model["dirs"][21], pix_stride=stride)
    rows = np.arange(0, len(T), stride)
    _check(T, ref, rows)


def test_octree_full_size_sampled(loc, oracle):
    model = LI.octree_cloud()
    mol = LI.rotor_molecule(n_levels=4)
    stride = 4099
    lam = 3
    with loc.Model(model, mol) as m:
        x = m.populations()
        T = m.map3d(0, 9, level=lam)
    ref = oracle.map_3d(mol, model, x, 0, model["dirs"][9], lam=lam, pix_stride=stride)
    rows = np.arange(0, len(T), stride)
    _check(T, ref, rows)


def test_map_arguments(loc):
    mol = LI.rotor_molecule(n_levels=4)
    grid = LI.small_grid3d(N=4, n_ch=16, nside=1)
    with loc.Model(grid, mol) as m:
        for bad in (dict(t=0, d=12, level=0), dict(t=0, d=-1, level=0), dict(t=3, d=0, level=0),
                    dict(t=0, d=0, level=1)):
            with pytest.raises(loc.LocError) as e:
                m.map3d(bad["t"], bad["d"], level=bad["level"])
            assert e.value.status == loc.LOC_EINVAL
    one_d = LI.cloud1d_two_level(K=4)
    with loc.Model(one_d, LI.two_level_molecule()) as m:
        with pytest.raises(loc.LocError):
            loc.loc_map3d(m.h, 0, 0, 0, 4, one_d["n_ch"])
