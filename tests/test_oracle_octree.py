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
* Split rays, oblique: a uniform absorber (S = 0) with a refined slab and a
  doubly refined sub-slab crossed along every direction whose main axis is
  the slab normal: each leaf's SIJ equals the mean of n_bg e^(-a z) over its
  depths (new rays at the slab's face, their termination where it ends, the
  resumed parent).
* Side rays, bounded: in the same absorber on random trees, no leaf has less
  than the exact field and none more than the field 2 h0 higher up, the
  largest extrapolation the side-ray rule allows.
Parity unpinned beyond these: the exact intensity given to side rays (rays
that enter a refined cell through a side face) is our reading of the
side-ray rule, which extrapolates the creating ray's intensity at the
refined cell's upstream face (Sect. 2.2) and has no closed form.
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


def _leaf_boxes(model):
    """Lower corner (cm, per axis) and size (cm) of every cell, from the
    level-ordered refinement flags (root cell (z N + y) N + x; child octant
    bits x = 1, y = 2, z = 4)."""
    r = np.asarray(model["refine"])
    N, h0 = model["n_root"], model["h0"]
    nc = len(r)
    lo = np.zeros((nc, 3))
    size = np.zeros(nc)
    for c in range(N ** 3):
        lo[c] = (c % N * h0, (c // N) % N * h0, c // (N * N) * h0)
        size[c] = h0
    child = _children(model)
    for c in range(nc):
        if child[c] >= 0:
            hh = size[c] / 2
            for o in range(8):
                k = child[c] + o
                lo[k] = lo[c] + hh * np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1])
                size[k] = hh
    return lo, size


def _absorber_sij(model, mol, lo, size, Kt, phi, d, lead=0.0):
    """Closed-form SIJ [line][leaf] of a static absorber without emission
    crossed along d (one direction), if every line at main-axis depth z
    carries n_bg e^(-a_k max(z - lead, 0)), a_k = K phi_k / |d_m| (lead = 0:
    the exact field; lead > 0: the field of rays that started up to `lead`
    deeper than the depth whose intensity they took).  With S = 0 a step's
    I_in (1 - e^-tau) / tau is the step's mean intensity, and each leaf's
    lateral square holds exactly one active lattice line at every depth of
    the leaf (its main-axis path is exactly its size, pinned above), so SIJ
    = sum_k phi_k x the mean of that field over the leaf's depths
    [zL, zL + H]; for lead = 0, n_bg e^(-a_k zL) (1 - e^(-a_k H)) / (a_k H)."""
    m = int(np.argmax(np.abs(d)))
    width = model["n_root"] * model["h0"]
    zL = (lo[:, m] if d[m] > 0 else width - lo[:, m] - size) - lead
    z0 = np.maximum(zL, 0.0)[:, None]                       # attenuated part [z0, zL + H]
    flat = (np.minimum(zL + size, 0.0) - np.minimum(zL, 0.0))[:, None]   # unattenuated part
    Ha = np.maximum((zL + size)[:, None] - z0, 0.0)
    nbg = 1.0 / np.expm1(H * np.asarray(mol["line_nu"]) / (KB * model["t_bg"]))
    out = []
    for t in range(len(Kt)):
        a = Kt[t] * phi[None, :] / abs(d[m])                       # per cm of depth
        aH = a * Ha
        ratio = np.where(aH > 0, -np.expm1(-aH) / np.where(aH > 0, aH, 1.0), 1.0)
        mean = nbg[t] * (flat + np.exp(-a * z0) * Ha * ratio) / size[:, None]
        out.append((phi[None, :] * mean).sum(axis=1))
    return np.array(out)


def _absorber(model, mol):
    """Static, isothermal version of `model` and the inputs of an absorber
    without emission: K per line (peak depth 1.5 and 4 across the model),
    S = 0; the channel fractions from scipy's erf."""
    from scipy.special import erf
    nc = len(model["refine"])
    model = dict(model, t_kin=np.full(nc, 15.0), sigma_turb=np.full(nc, 0.2e5),
                 vx=np.zeros(nc), vy=np.zeros(nc), vz=np.zeros(nc))
    sig = np.sqrt(0.2e5 ** 2 + KB * 15.0 / (mol["mass_amu"] * AMU))
    vk = model["v_min"] + (np.arange(model["n_ch"]) + 0.5) * model["dv"]
    s2 = np.sqrt(2.0) * sig
    phi = 0.5 * (erf((vk + 0.5 * model["dv"]) / s2) - erf((vk - 0.5 * model["dv"]) / s2))
    T = len(mol["line_nu"])
    Kt = np.array([1.5, 4.0])[:T] / (phi.max() * model["n_root"] * model["h0"])
    n_leaf = len(oracle_leaves(model))
    Kp = np.repeat(Kt[:, None], n_leaf, axis=1)
    return model, Kt, phi, Kp, np.zeros_like(Kp)


def oracle_leaves(model):
    return np.flatnonzero(np.asarray(model["refine"]) == 0)


@pytest.mark.parametrize("N", [2, 3])
def test_uniform_absorber_refined_slab_closed_form(oracle, N):
    """Rays split at a refined region's upstream face, terminated where it
    ends, and the resumed parent, pinned for oblique directions: a root
    layer refined across the whole (laterally periodic) model, the lower
    half of its children refined again, crossed along directions whose main
    axis is the slab normal (no side faces to enter through, so every new
    ray starts at the slab's upstream face).  Every leaf matches the
    closed form of a uniform absorber to rounding."""
    mol = LI.rotor_molecule(n_levels=3)
    base = LI.small_octree(N=N, levels=1, refine_frac=0.3, n_ch=24)
    nroot = N ** 3
    lay = [c for c in range(nroot) if c // (N * N) == N - 1]          # top root layer
    refine = np.zeros(nroot + 8 * len(lay) + 8 * 4 * len(lay), np.int32)
    refine[lay] = 1
    first = nroot
    for k in range(len(lay)):
        for o in range(4):                                              # child octants z = 0
            refine[first + 8 * k + o] = 1
    model = dict(base, levels=2, refine=refine, n_h2=np.full(len(refine), 1e4),
                 abundance=np.full(len(refine), 1e-8))
    model, Kt, phi, Kp, S = _absorber(model, mol)
    lo, size = _leaf_boxes(model)
    lf = oracle.leaves(model)
    lo, size = lo[lf], size[lf]
    assert set(np.round(size / model["h0"], 6)) == {1.0, 0.5, 0.25}
    dirs = [d for d in LI.healpix_ring_directions(2) if np.argmax(np.abs(d)) == 2]
    assert len(dirs) >= 8 and min(d[2] for d in dirs) < 0 < max(d[2] for d in dirs)
    for d in dirs:
        SIJ, ESC, NORM = oracle.march_octree(mol, dict(model, dirs=np.asarray(d)[None, :]), Kp, S)
        np.testing.assert_allclose(NORM, phi.sum(), rtol=1e-13)
        np.testing.assert_allclose(SIJ, _absorber_sij(model, mol, lo, size, Kt, phi, d), rtol=1e-10)


@pytest.mark.parametrize("shape", [(2, 2, 0.4), (3, 3, 0.35), (4, 2, 0.3)])
def test_uniform_absorber_side_rays_bounded(oracle, shape):
    """Side rays (rays started where a line enters a refined cell through a
    side face) take the intensity the creating line had at the cell's
    upstream face (Sect. 2.2: an extrapolation over less than the size of
    the refined cell).  In a uniform absorber no ray can then carry more
    attenuation than the exact field, and none less than the field 2 h0
    higher up (n_bg e^(-a max(z - 2 h0, 0))): per leaf, the closed forms of
    these two fields bound SIJ; the leaves that no side ray crosses meet
    the lower bound, and the side rays of these trees raise others above
    it (this bounds the rule; its exact value is our reading)."""
    N, levels, frac = shape
    mol = LI.rotor_molecule(n_levels=3)
    model, Kt, phi, Kp, S = _absorber(LI.small_octree(N=N, levels=levels, refine_frac=frac, n_ch=24), mol)
    lo, size = _leaf_boxes(model)
    lf = oracle.leaves(model)
    lo, size = lo[lf], size[lf]
    exact_frac, raised = [], 0
    for d in LI.healpix_ring_directions(2)[::5]:
        SIJ, ESC, NORM = oracle.march_octree(mol, dict(model, dirs=np.asarray(d)[None, :]), Kp, S)
        np.testing.assert_allclose(NORM, phi.sum(), rtol=1e-13)
        lo_b = _absorber_sij(model, mol, lo, size, Kt, phi, d)
        hi_b = _absorber_sij(model, mol, lo, size, Kt, phi, d, lead=2 * model["h0"])
        assert np.all(SIJ >= lo_b * (1 - 1e-12))
        assert np.all(SIJ <= hi_b * (1 + 1e-12))
        eq = np.isclose(SIJ, lo_b, rtol=1e-10, atol=0).all(axis=0)
        exact_frac.append(eq.mean())
        raised += int((~eq).sum())
    assert min(exact_frac) > 0.1 and raised > 0
