"""Pins of the oracle's octree ray tracing (Sect. 2.2).

* Geometry: the segment walk of every lattice line equals a brute-force
  run-length encoding of the leaf hit at each integer main-axis coordinate
  (small fixed-point precision), with activity = leaf level >= creation level.
* Constant path length: per direction, every leaf receives exactly H_L of
  active main-axis path (H_L = its size in fixed-point units), so the
  paper's constant path length per cell (up to the 0.5^L size factor) holds
  exactly, and refined cells none; for all 48 directions.
* A uniformly refined octree equals the regular grid of twice the
  resolution (all lines active from the upstream face, background start).
* Split rays, closed form: a partially refined grid crossed along an axis;
  the rays created at the refined cell's upstream face start with the
  intensity of the coarse ray at that face (uniform static medium -> slab
  formulas).
Parity unpinned beyond these: the intensity given to side rays (rays that
enter a refined cell through a side face) is our reading of the side-ray
rule and has no independent closed form.
"""
import numpy as np
import pytest

import loc_inputs as LI

H = 6.62607015e-27
KB = 1.380649e-16
AMU = 1.66053906660e-24


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


def _children(model):
    r = np.asarray(model["refine"])
    N = model["n_root"]
    child = -np.ones(len(r), np.int64)
    nxt = N ** 3
    for c in range(len(r)):
        if r[c]:
            child[c] = nxt
            nxt += 8
    assert nxt == len(r)
    return child


def _brute_line(model, child, F, d, lam, i, j, info):
    N, Lmax = model["n_root"], model["levels"]
    H0 = 1 << F
    E = N * H0
    o = (H0 >> Lmax) // 2
    m, a, b = info["m"], info["a"], info["b"]
    runs = []
    for z in range(E):
        A = (o + i * (H0 >> lam) + (info["qa"] * z >> F)) % E
        B = (o + j * (H0 >> lam) + (info["qb"] * z >> F)) % E
        pos = [0, 0, 0]
        pos[m], pos[a], pos[b] = z, A, B
        p = [(E - 1 - pos[ax]) if info["flip"][ax] else pos[ax] for ax in range(3)]
        c = ((p[2] >> F) * N + (p[1] >> F)) * N + (p[0] >> F)
        L = 0
        while child[c] >= 0:
            L += 1
            s = F - L
            c = child[c] + (((p[0] >> s) & 1) | (((p[1] >> s) & 1) << 1) | (((p[2] >> s) & 1) << 2))
        if runs and runs[-1][2] == c:
            runs[-1][1] += 1
        else:
            runs.append([z, 1, c, L, int(L >= lam)])
    return runs


@pytest.mark.parametrize("seed", [11, 12])
def test_octree_segments_brute_force(oracle, seed):
    model = LI.small_octree(N=2, levels=2, seed=seed, refine_frac=0.4)
    child = _children(model)
    F = 5
    dirs = LI.healpix_ring_directions(2)
    N, Lmax = model["n_root"], model["levels"]
    for d in dirs[::5]:
        info = oracle.dir_info(d, F)
        for lam in range(Lmax + 1):
            M = N << lam
            for i in range(M):
                for j in range(M):
                    if lam and i % 2 == 0 and j % 2 == 0:
                        continue
                    got = oracle.octree_line_segments(model, d, lam, i, j, F)
                    ref = np.array(_brute_line(model, child, F, d, lam, i, j, info), np.int64)
                    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("shape", [(2, 2, 0.4), (4, 2, 0.3), (3, 3, 0.35)])
def test_octree_constant_path_length_exact(oracle, shape):
    N, levels, frac = shape
    model = LI.small_octree(N=N, levels=levels, refine_frac=frac)
    lev = _levels(model)
    lf = np.asarray(model["refine"]) == 0
    Hc = (1 << 24) >> lev
    for d in LI.healpix_ring_directions(2):
        s = oracle.octree_path_sums(model, d)
        assert np.all(s[lf] == Hc[lf])
        assert np.all(s[~lf] == 0)


def test_uniformly_refined_octree_equals_fine_grid(oracle):
    N = 3
    mol = LI.rotor_molecule(n_levels=4)
    fine = LI.small_grid3d(N=2 * N, n_ch=20, nside=2, abundance=2e-5)
    # octree: every root cell refined once, children carry the fine-grid values
    nc0 = N ** 3
    refine = np.concatenate([np.ones(nc0, np.int32), np.zeros(8 * nc0, np.int32)])
    order = []                                  # fine-grid index of each child
    for c in range(nc0):
        ix, iy, iz = c % N, (c // N) % N, c // (N * N)
        for o in range(8):
            fx, fy, fz = 2 * ix + (o & 1), 2 * iy + ((o >> 1) & 1), 2 * iz + ((o >> 2) & 1)
            order.append((fz * 2 * N + fy) * 2 * N + fx)
    order = np.array(order)
    octm = dict(geometry="octree3d", n_root=N, h0=2 * fine["h0"], levels=1, refine=refine,
                dirs=fine["dirs"], n_ch=fine["n_ch"], v_min=fine["v_min"], dv=fine["dv"],
                t_bg=fine["t_bg"])
    for key in ("n_h2", "t_kin", "sigma_turb", "abundance", "vx", "vy", "vz"):
        octm[key] = np.concatenate([np.zeros(nc0), np.asarray(fine[key])[order]])
    x = oracle.lte_populations(mol, fine["t_kin"])
    Kp, S = oracle.line_params(mol, fine, x)
    rs, re_, rn = oracle.march_grid3d(mol, fine, Kp, S)
    os_, oe, on = oracle.march_octree(mol, octm, Kp[:, order], S[:, order])
    # the octree's level-1 lattice equals the fine grid's up to the rounding of
    # floor(q z / 2^F) at half the scale: one fixed-point unit in 2^23
    np.testing.assert_allclose(on, rn[order], rtol=1e-6)
    np.testing.assert_allclose(os_, rs[:, order], rtol=1e-6)
    np.testing.assert_allclose(oe, re_[:, order], rtol=1e-6)


def test_split_rays_axis_aligned_closed_form(oracle):
    """2x2x2 root grid, cell (0,0,1) refined, uniform static medium, one ray
    direction +z.  Column (0,0): the coarse ray crosses root cell (0,0,0),
    then the refined cell, where three new rays start at its upstream face
    with the coarse ray's intensity; every ray then crosses two half cells."""
    N = 2
    mol = LI.two_level_molecule()
    refine = np.zeros(N ** 3 + 8, np.int32)
    refine[(1 * N + 0) * N + 0] = 1             # cell ix=0, iy=0, iz=1
    nc = len(refine)
    h0 = 1.0e16
    model = dict(geometry="octree3d", n_root=N, h0=h0, levels=1, refine=refine,
                 n_h2=np.full(nc, 2e4), t_kin=np.full(nc, 20.0), sigma_turb=np.full(nc, 2e4),
                 abundance=np.full(nc, 1e-8), vx=np.zeros(nc), vy=np.zeros(nc), vz=np.zeros(nc),
                 dirs=np.array([[0.0, 0.0, 1.0]]), n_ch=24, v_min=-1.5e5, dv=1.25e4, t_bg=2.73)
    lm = oracle.leaf_model(model)
    x = np.tile([0.4, 0.6], (len(lm["n_h2"]), 1))
    Kp, S = oracle.line_params(mol, lm, x)
    SIJ, ESC, NORM = oracle.march_octree(mol, model, Kp, S)
    sig = np.sqrt(2e4 ** 2 + KB * 20.0 / (mol["mass_amu"] * AMU))
    phi = oracle.profile(24, -1.5e5, 1.25e4, 0.0, sig)
    nbg = 1.0 / np.expm1(H * mol["line_nu"][0] / (KB * 2.73))
    K, Sv = Kp[0, 0], S[0, 0]

    def jext(depth_h0, step_h0):
        tau0 = K * phi * h0 * depth_h0
        tau1 = K * phi * h0 * step_h0
        Iin = nbg * np.exp(-tau0) - Sv * np.expm1(-tau0)
        f = -np.expm1(-tau1) / tau1
        return (phi * Iin * f).sum() / phi.sum()

    lf = oracle.leaves(model)
    lev = _levels(model)[lf]
    # leaf coordinates
    for k, c in enumerate(lf):
        if lev[k] == 0:
            iz = c // (N * N)
            expect = jext(iz, 1.0)
        else:
            o = (c - N ** 3) % 8
            cz = (o >> 2) & 1
            expect = jext(1.0 + 0.5 * cz, 0.5)    # entered at the refined cell's face (depth 1)
        assert SIJ[0, k] / NORM[k] == pytest.approx(expect, rel=1e-12)
        assert NORM[k] == pytest.approx(phi.sum(), rel=1e-13)
