"""GPU parity of the octree path (Sect. 2.2) against the FP64 oracle, through
the C ABI.

* Path lists are integer-exact: the set of active segments the device
  traversal produces for a direction (root rays, rays created at refined
  cells, terminations) equals the oracle's, compared as sorted records
  (creation level, i, j, z0, dz, leaf).
* One ray simulation agrees to 2e-5 relative, T_ex after a fixed number of
  iterations to 1e-4.
* Full size (64^3 root, 5 levels, 7.9e6 leaves): the oracle cannot walk every
  lattice line, so (a) the per-leaf path-length invariant (exactly H_L per
  direction) is checked for every leaf, (b) a sample of device segments is
  checked against the oracle's walk of the same lines, (c) an isothermal
  cloud at the background temperature keeps the mean intensity at n_bg.
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


def _leaf_index(model):
    r = np.asarray(model["refine"]) == 0
    idx = np.cumsum(r) - 1
    return np.where(r, idx, -1)


def _levels(model):
    r = np.asarray(model["refine"])
    N = model["n_root"]
    lev = np.zeros(len(r), int)
    start, end, L = 0, N ** 3, 0
    while start < end:
        nref = int(r[start:end].sum())
        lev[end:end + 8 * nref] = L + 1
        start, end, L = end, end + 8 * nref, L + 1
    return lev


def _oracle_records(oracle, model, d):
    lf = _leaf_index(model)
    N, Lmax = model["n_root"], model["levels"]
    recs = []
    for lam in range(Lmax + 1):
        M = N << lam
        for i in range(M):
            for j in range(M):
                if lam and i % 2 == 0 and j % 2 == 0:
                    continue
                s = oracle.octree_line_segments(model, d, lam, i, j)
                for z0, dz, cell, lev, act in s:
                    if act:
                        recs.append((lam, i, j, z0, dz, lf[cell], lev))
    recs = np.array(recs, np.int64).reshape(-1, 7)
    return recs[np.lexsort(recs.T[::-1])]


@pytest.mark.parametrize("shape", [(1, 2, 1.0, 1), (2, 2, 0.4, 2), (4, 2, 0.3, 2), (3, 3, 0.35, 2)])
def test_octree_paths_bit_exact(loc, oracle, shape):
    N, levels, frac, nside = shape
    model = LI.small_octree(N=N, levels=levels, refine_frac=frac, nside=nside, n_ch=8)
    mol = LI.rotor_molecule(n_levels=3)
    with loc.Model(model, mol) as m:
        for d in range(0, len(model["dirs"]), 3):
            got = m.trace_octree(d)
            got = got[np.lexsort(got.T[::-1])]
            ref = _oracle_records(oracle, model, model["dirs"][d])
            assert got.shape == ref.shape, (d, got.shape, ref.shape)
            np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("window", [0.0, 8.0])
def test_octree_march_radiation(loc, oracle, window):
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.small_octree(N=4, levels=2, refine_frac=0.3, nside=2, n_ch=24, abundance=3e-5)
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=window)
        sij, esc, norm = m.radiation()
    lm = oracle.leaf_model(model)
    x = oracle.lte_populations(mol, lm["t_kin"])
    Kp, S = oracle.line_params(mol, lm, x)
    rs, re_, rn = oracle.march_octree(mol, model, Kp, S)
    np.testing.assert_allclose(norm, rn, rtol=2e-5)
    np.testing.assert_allclose(sij, rs, rtol=2e-5, atol=1e-12 * np.abs(rs).max())
    np.testing.assert_allclose(esc, re_, rtol=2e-5)


def test_octree_iterations(loc, oracle):
    mol = LI.rotor_molecule(n_levels=6)
    model = LI.small_octree(N=4, levels=2, refine_frac=0.3, nside=2, n_ch=24, abundance=1e-4)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=3, window_sigmas=8.0)
        x_ref, _ = oracle.iterate_octree(mol, model, 3)
        tref = oracle.tex(mol, x_ref)
        for t in range(tref.shape[0]):
            sel = x_ref[:, mol["line_u"][t]] >= 1e-6
            if sel.any():
                err = np.max(np.abs(m.tex(t)[sel] / tref[t, sel] - 1.0))
                assert err < 1e-4, (t, err)


def test_octree_iterations_with_level_cutoff(loc, oracle):
    """Per-cell line truncation on an octree: populations per leaf (down to
    1e-20) and T_ex against the oracle's truncated iteration."""
    mol = LI.rotor_molecule(n_levels=14)
    model = LI.small_octree(N=4, levels=2, refine_frac=0.3, nside=2, n_ch=24, abundance=1e-4)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=3, window_sigmas=8.0, level_cutoff=1e-8)
        xg = m.populations()
        x_ref, _ = oracle.iterate_octree(mol, model, 3, level_cutoff=1e-8)
        tref = oracle.tex(mol, x_ref)
        for t in range(tref.shape[0]):
            sel = x_ref[:, mol["line_u"][t]] >= 1e-6
            if sel.any():
                err = np.max(np.abs(m.tex(t)[sel] / tref[t, sel] - 1.0))
                assert err < 1e-4, (t, err)
    sel = x_ref > 1e-20
    assert np.max(np.abs(xg[sel] / x_ref[sel] - 1.0)) < 1e-3


def test_octree_medium_size_radiation(loc, oracle):
    """12^3 root, 3 levels, all 48 directions, 11 lines."""
    mol = LI.rotor_molecule()
    model = LI.small_octree(N=12, levels=3, refine_frac=0.15, nside=2, n_ch=24, box_pc=0.2,
                            abundance=1e-5, seed=5)
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=8.0)
        sij, esc, norm = m.radiation()
    lm = oracle.leaf_model(model)
    x = oracle.lte_populations(mol, lm["t_kin"])
    Kp, S = oracle.line_params(mol, lm, x)
    rs, re_, rn = oracle.march_octree(mol, model, Kp, S)
    np.testing.assert_allclose(norm, rn, rtol=2e-5, atol=1e-7 * rn.max())
    for t in range(len(mol["line_nu"])):
        np.testing.assert_allclose(sij[t], rs[t], rtol=5e-5, atol=1e-6 * np.abs(rs[t]).max())
        np.testing.assert_allclose(esc[t], re_[t], rtol=5e-5, atol=1e-6 * np.abs(re_[t]).max())


def test_octree_full_size_invariants(loc, oracle):
    model = LI.octree_cloud()
    mol = LI.rotor_molecule(n_levels=4)
    lev = _levels(model)[np.asarray(model["refine"]) == 0]
    HL = (1 << 24) >> lev
    lf = _leaf_index(model)
    leaf_cell = np.flatnonzero(np.asarray(model["refine"]) == 0)
    with loc.Model(model, mol) as m:
        info = m.info()
        assert info["n_cells"] == len(leaf_cell)
        for d in (0, 17, 40):
            s = m.octree_path_sums(d)
            assert np.array_equal(s, HL), d
        # sampled device segments appear in the oracle's walk of the same line
        recs = m.trace_octree(7, cap=3000)
        rng = np.random.default_rng(3)
        for r in recs[rng.choice(len(recs), size=60, replace=False)]:
            lam, i, j, z0, dz, leaf, lv = (int(v) for v in r)
            segs = oracle.octree_line_segments(model, model["dirs"][7], lam, i, j)
            hit = segs[(segs[:, 0] == z0) & (segs[:, 1] == dz)]
            assert len(hit) == 1 and hit[0, 4] == 1
            assert lf[hit[0, 2]] == leaf and hit[0, 3] == lv


def test_octree_full_size_isothermal(loc):
    model = LI.octree_cloud()
    model["t_kin"] = np.full_like(model["t_kin"], model["t_bg"])
    mol = LI.rotor_molecule(n_levels=4)
    with loc.Model(model, mol) as m:
        m.march(window_sigmas=8.0)
        sij, esc, norm = m.radiation()
    h, k = 6.62607015e-27, 1.380649e-16
    nbg = 1.0 / np.expm1(h * mol["line_nu"][:3] / (k * model["t_bg"]))
    S = nbg[:, None]
    Jbar = (sij + S * (norm - esc)) / norm
    np.testing.assert_allclose(Jbar / S, 1.0, rtol=3e-5)


def test_octree_replay_equals_walk(loc, oracle):
    """The recorded paths (default) and the tree walk in every march
    (octree_paths = 1) apply the same steps in the same order: the
    accumulators agree to FP32 atomic-ordering noise, and the report says
    which one ran."""
    mol = LI.rotor_molecule()
    model = LI.small_octree(N=12, levels=3, refine_frac=0.15, nside=2, n_ch=24, box_pc=0.2,
                            abundance=1e-5, seed=5)
    out = {}
    for paths in (0, 1):
        with loc.Model(dict(model, octree_paths=paths), mol) as m:
            rep = m.iterate(max_iter=1, window_sigmas=8.0, lines_per_pass=4)
            out[paths] = (rep, m.radiation())
    assert out[0][0]["path_records"] >= out[0][0]["segments"] > 0
    assert out[1][0]["path_records"] == 0
    for a, b in zip(out[0][1], out[1][1]):
        np.testing.assert_allclose(a, b, rtol=2e-6, atol=1e-9 * np.abs(b).max())


def test_octree_recorders_agree(loc):
    """The one-walk recorder (a chunk pool, then the contiguous layout) and
    the two-walk one (count, then record; octree_paths = 2) write the same
    records: the same record count, and the replayed marches agree to FP32
    atomic-ordering noise."""
    mol = LI.rotor_molecule()
    model = LI.octree_cloud(N=10)
    out = {}
    for paths in (0, 2):
        with loc.Model(dict(model, octree_paths=paths), mol) as m:
            rep = m.iterate(max_iter=1, window_sigmas=8.0, lines_per_pass=6)
            out[paths] = (rep, m.radiation())
    assert out[0][0]["path_records"] == out[2][0]["path_records"] > out[0][0]["segments"] > 0
    for a, b in zip(out[0][1], out[2][1]):
        np.testing.assert_allclose(a, b, rtol=2e-6, atol=1e-9 * np.abs(b).max())


@pytest.fixture(scope="module")
def bench_recipe_octree(oracle):
    """The bench's octree recipe (refined up to 5 levels where n > 8 x mean,
    64 channels, 48 directions, 11 lines) on a 12^3 root: 57,077 leaves.
    Oracle: the radiation of one march at LTE and the populations after 3
    ALI iterations."""
    model = LI.octree_cloud(N=12)
    mol = LI.rotor_molecule()
    assert model["levels"] == 5
    lm = oracle.leaf_model(model)
    x0 = oracle.lte_populations(mol, lm["t_kin"])
    Kp, S = oracle.line_params(mol, lm, x0)
    rad = oracle.march_octree(mol, model, Kp, S)
    x3, _ = oracle.iterate_octree(mol, model, 3)
    return model, mol, rad, x3


@pytest.mark.parametrize("per", [6, 11, 0])
def test_octree_bench_launch_shapes(loc, oracle, bench_recipe_octree, per):
    """Parity at the launch shapes of the bench's octree: 6 and 11 lines per
    warp and the autotuned choice (per = 0), 8-sigma window, replayed paths."""
    model, mol, (rs, re_, rn), x3 = bench_recipe_octree
    with loc.Model(model, mol) as m:
        if per == 0:
            m.autotune(window_sigmas=8.0)
        m.march(window_sigmas=8.0, lines_per_pass=per)
        sij, esc, norm = m.radiation()
        m.reset()
        rep = m.iterate(max_iter=3, window_sigmas=8.0, lines_per_pass=per)
        assert rep["path_records"] > 0
        tex = [m.tex(t) for t in range(len(mol["line_nu"]))]
    np.testing.assert_allclose(norm, rn, rtol=2e-5, atol=1e-7 * rn.max())
    for t in range(len(mol["line_nu"])):
        np.testing.assert_allclose(sij[t], rs[t], rtol=5e-5, atol=1e-6 * np.abs(rs[t]).max())
        np.testing.assert_allclose(esc[t], re_[t], rtol=5e-5, atol=1e-6 * np.abs(re_[t]).max())
    tref = oracle.tex(mol, x3)
    for t in range(tref.shape[0]):
        sel = x3[:, mol["line_u"][t]] >= 1e-6
        if sel.any():
            err = np.max(np.abs(tex[t][sel] / tref[t, sel] - 1.0))
            assert err < 1e-4, (t, err)


def test_octree_full_size_one_direction(loc, oracle):
    """The bench's full-size octree (64^3 root refined up to 5 levels:
    7,929,328 leaves; 11 lines, 64 channels, 48 directions) at the bench's
    launch shape (6 lines per warp, compensated FP32, 8-sigma window,
    replayed paths): the ray simulation of one direction (dir_range) against
    the oracle's march of that direction, every leaf's SIJ, ESC and NORM.
    The oracle gets a model whose direction table holds that direction
    alone, so its step weights carry 1 instead of 1/48 for the direction's
    share: its sums are 48 times the device's."""
    model = LI.octree_cloud(N=64)
    mol = LI.rotor_molecule()
    d = 5
    n_dir = len(model["dirs"])
    lm = oracle.leaf_model(model)
    x0 = oracle.lte_populations(mol, lm["t_kin"])
    Kp, S = oracle.line_params(mol, lm, x0)
    rs, re_, rn = oracle.march_octree(mol, dict(model, dirs=np.asarray(model["dirs"])[d:d + 1]), Kp, S)
    with loc.Model(model, mol) as m:
        m.march(dir_range=(d, d + 1), window_sigmas=8.0, lines_per_pass=6)
        sij, esc, norm = (np.asarray(a) * n_dir for a in m.radiation())
    assert rn.min() > 0.0                           # every leaf is crossed in every direction
    np.testing.assert_allclose(norm, rn, rtol=2e-5, atol=1e-7 * rn.max())
    for t in range(len(mol["line_nu"])):
        np.testing.assert_allclose(sij[t], rs[t], rtol=5e-5, atol=1e-6 * np.abs(rs[t]).max())
        np.testing.assert_allclose(esc[t], re_[t], rtol=5e-5, atol=1e-6 * np.abs(re_[t]).max())
