"""Pins of the oracle's 3D emergent maps (Sect. 2: the final line-of-sight
integration after convergence, here for regular grids and octrees).

* Uniform static cube: every pixel's ray crosses the periodic model once
  along the main axis, a path N h0 / |d_m|, so
  T = (h nu / k)(S - n_bg)(1 - e^{-tau}) with tau = K phi N h0 / |d_m| for
  any direction (oblique ones included) and any refinement of the cube.
* Refinement invariance: an octree whose children copy their parent's
  values shows, along an axis, the regular grid's map (pixel (i, j) of level
  lam lies in root column (i >> lam, j >> lam)).
* Pixel layout: a dense rod of cells along the main axis lights the pixel
  (i, j) given by its position on the transverse axes a and b.
* Optically thin limit on a moving grid: the map equals the sum of the
  emissivities K phi(v_los) s (S - n_bg) along the ray (brute-force sum over
  the oracle's own grid path), to O(tau).
"""
import numpy as np
import pytest

import loc_inputs as LI

H = 6.62607015e-27
KB = 1.380649e-16
AMU = 1.66053906660e-24
F = 24


def planck_occ(nu, T):
    return 1.0 / np.expm1(H * nu / (KB * T))


def _uniform(g, n_h2=3e4, abundance=1e-8, t_kin=20.0):
    n = len(g["n_h2"])
    g = dict(g)
    g["n_h2"] = np.full(n, n_h2)
    g["abundance"] = np.full(n, abundance)
    g["t_kin"] = np.full(n, t_kin)
    for key in ("vx", "vy", "vz"):
        g[key] = np.zeros(n)
    return g


def _refine_copy(g, flags0, second=True):
    """Octree from a regular grid: root cells with flags0 are split into 8
    children that copy the parent's values; with `second`, the first child
    of every refined root cell is split again (levels = 2)."""
    N = g["n_root"]
    nc0 = N ** 3
    keys = ("n_h2", "t_kin", "sigma_turb", "abundance", "vx", "vy", "vz")
    vals = {k: list(np.asarray(g[k], float)) for k in keys}
    refine = [int(f) for f in flags0]
    parent = list(range(nc0))
    lvl1 = []
    for c in range(nc0):
        if flags0[c]:
            for o in range(8):
                lvl1.append(c)
    start1 = nc0
    for c in lvl1:
        for k in keys:
            vals[k].append(vals[k][c])
        parent.append(c)
    refine += [0] * len(lvl1)
    levels = 1
    if second and lvl1:
        levels = 2
        for q in range(0, len(lvl1), 8):
            refine[start1 + q] = 1
        for q in range(0, len(lvl1), 8):
            src = start1 + q
            for o in range(8):
                for k in keys:
                    vals[k].append(vals[k][src])
                parent.append(parent[src])
        refine += [0] * (8 * (len(lvl1) // 8))
    out = dict(g)
    out.update({k: np.array(v) for k, v in vals.items()})
    out.update(geometry="octree3d", levels=levels, refine=np.array(refine, np.int32))
    return out, np.array(parent)


def test_uniform_cube_closed_form_grid_and_octree(oracle):
    mol = LI.two_level_molecule()
    g = _uniform(LI.small_grid3d(N=4, n_ch=16, nside=1))
    nc = len(g["n_h2"])
    x = np.tile([0.35, 0.65], (nc, 1))
    Kp, S = oracle.line_params(mol, g, x)
    sig = np.sqrt(g["sigma_turb"][0] ** 2 + KB * 20.0 / (mol["mass_amu"] * AMU))
    phi = oracle.profile(g["n_ch"], g["v_min"], g["dv"], 0.0, sig)
    nbg = planck_occ(mol["line_nu"][0], g["t_bg"])
    T0 = H * mol["line_nu"][0] / KB
    flags = (np.arange(nc) % 5 == 0).astype(int)
    o, _ = _refine_copy(g, flags)
    xo = np.tile([0.35, 0.65], ((o["refine"] == 0).sum(), 1))
    for d in g["dirs"]:
        m = int(np.argmax(np.abs(d)))
        tau = Kp[0, 0] * phi * g["n_root"] * g["h0"] / abs(d[m])
        want = T0 * (S[0, 0] - nbg) * -np.expm1(-tau)
        # I - n_bg in FP64 keeps ~1e-16 n_bg absolute accuracy in the far wings
        atol = 1e-12 * np.abs(want).max()
        Tg = oracle.map_3d(mol, g, x, 0, d)
        np.testing.assert_allclose(Tg, np.broadcast_to(want, Tg.shape), rtol=1e-11, atol=atol)
        for lam in (0, 1, 2):
            To = oracle.map_3d(mol, o, xo, 0, d, lam=lam)
            assert To.shape == ((4 << lam) ** 2, 16)
            np.testing.assert_allclose(To, np.broadcast_to(want, To.shape), rtol=1e-11, atol=atol)


@pytest.mark.parametrize("d", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, -1, 0)])
def test_refinement_invariance_along_axes(oracle, d):
    mol = LI.rotor_molecule(n_levels=4)
    g = LI.small_grid3d(N=4, n_ch=24, nside=1, abundance=3e-5)
    nc = len(g["n_h2"])
    x = oracle.lte_populations(mol, g["t_kin"])
    flags = (g["n_h2"] > np.median(g["n_h2"])).astype(int)
    o, parent = _refine_copy(g, flags)
    leaf = np.flatnonzero(o["refine"] == 0)
    xo = x[parent[leaf]]
    d = np.array(d, float)
    Tg = oracle.map_3d(mol, g, x, 1, d)
    assert np.abs(Tg).max() > 0
    for lam in (0, 1, 2):
        M = 4 << lam
        To = oracle.map_3d(mol, o, xo, 1, d, lam=lam).reshape(M, M, -1)
        ii, jj = np.meshgrid(np.arange(M) >> lam, np.arange(M) >> lam, indexing="ij")
        want = Tg.reshape(4, 4, -1)[ii, jj]
        np.testing.assert_allclose(To, want, rtol=1e-10, atol=1e-12 * np.abs(Tg).max())


@pytest.mark.parametrize("d,rod_axis,pos,pix", [
    ((0, 0, 1), 2, (2, 1), (2, 1)),
    ((0, 0, -1), 2, (2, 1), (2, 1)),
    ((1, 0, 0), 0, (1, 3), (1, 3)),
    ((-1, 0, 0), 0, (1, 3), (1, 3)),
    ((0, -1, 0), 1, (3, 0), (3, 0)),
])
def test_pixel_layout(oracle, d, rod_axis, pos, pix):
    """A rod of dense cells along the main axis at transverse position pos
    (coordinates along axes a < b) is seen in pixel pix = (i, j)."""
    mol = LI.two_level_molecule()
    N = 4
    g = _uniform(LI.small_grid3d(N=N, n_ch=16), abundance=1e-12)
    ix, iy, iz = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    idx = (iz * N + iy) * N + ix
    coords = [ix, iy, iz]
    others = [ax for ax in range(3) if ax != rod_axis]
    sel = (coords[others[0]] == pos[0]) & (coords[others[1]] == pos[1])
    g["abundance"][idx[sel]] = 1e-8
    x = np.tile([0.35, 0.65], (N ** 3, 1))
    T = oracle.map_3d(mol, g, x, 0, np.array(d, float)).reshape(N, N, -1)
    peak = np.unravel_index(np.argmax(T.max(axis=2)), (N, N))
    assert peak == pix
    assert T[pix].max() > 100 * np.delete(T.reshape(N * N, -1), pix[0] * N + pix[1], axis=0).max()


def test_thin_limit_sum_of_emissivities_oblique(oracle):
    mol = LI.rotor_molecule(n_levels=4)
    g = LI.small_grid3d(N=5, n_ch=32, nside=2, abundance=1e-12)
    N = g["n_root"]
    x = oracle.lte_populations(mol, g["t_kin"] * 0.0 + 12.0)
    Kp, S = oracle.line_params(mol, g, x)
    t = 1
    nbg = planck_occ(mol["line_nu"][t], g["t_bg"])
    T0 = H * mol["line_nu"][t] / KB
    for d in g["dirs"][[3, 17, 30]]:
        m = int(np.argmax(np.abs(d)))
        unit = g["h0"] / 2.0 ** F / abs(d[m])
        T = oracle.map_3d(mol, g, x, t, d)
        for pix in (0, 7, 13, 24):
            cells, dz = oracle.paths_grid3d(N, d, pix // N, pix % N)
            want = np.zeros(g["n_ch"])
            for c, dzz in zip(cells, dz):
                sig = np.sqrt(g["sigma_turb"][c] ** 2 + KB * g["t_kin"][c] / (mol["mass_amu"] * AMU))
                vlos = g["vx"][c] * d[0] + g["vy"][c] * d[1] + g["vz"][c] * d[2]
                phi = oracle.profile(g["n_ch"], g["v_min"], g["dv"], vlos, sig)
                want += Kp[t, c] * phi * dzz * unit * (S[t, c] - nbg)
            want *= T0
            assert np.abs(want).max() > 0
            np.testing.assert_allclose(T[pix], want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
