"""Pins of the oracle's ray geometry.

1D (Sect. 2.1): every equidistant ray's path lengths add up to its chord,
the shell sequence and entry cosines agree with brute-force sampling along
the ray, and the weights sum(A_j s) converge to the shell volumes.

3D (Sect. 2.2): the constant-path-length property -- per direction every
cell is crossed by a total of exactly one cell size of main-axis length --
holds exactly in the integer geometry for all 48 HEALPix directions, and the
event-based segment walk equals a brute-force run-length encoding over every
integer main-axis coordinate at small fixed-point precision.
"""
import numpy as np
import pytest

import loc_inputs as LI


@pytest.mark.parametrize("K,n_rays", [(1, 1), (5, 5), (7, 13), (32, 32)])
def test_1d_chords(oracle, K, n_rays):
    m = LI.cloud1d_two_level(K=K, n_rays=n_rays)
    R = m["radius"]
    for j in range(n_rays):
        p = (j + 0.5) * R[-1] / n_rays
        cell, s, cosv = oracle.paths_1d(m, j)
        assert s.sum() == pytest.approx(2.0 * np.sqrt(R[-1] ** 2 - p ** 2), rel=1e-13)
        t = int(np.argmax(R > p))
        expect = list(range(K - 1, t - 1, -1)) + list(range(t, K))
        assert list(cell) == expect
        assert np.all(s > 0)


def test_1d_brute_force_sampling(oracle):
    K, n_rays = 6, 9
    m = LI.cloud1d_two_level(K=K, n_rays=n_rays)
    R = m["radius"]
    for j in range(n_rays):
        p = (j + 0.5) * R[-1] / n_rays
        cell, s, cosv = oracle.paths_1d(m, j)
        zmax = np.sqrt(R[-1] ** 2 - p ** 2)
        nz = 100000
        runs, lens = [], []
        # inbound half (z < 0) and outbound half (z > 0) sampled separately:
        # the tangent shell is one step per half
        for lo, hi in ((-zmax, 0.0), (0.0, zmax)):
            dz = (hi - lo) / nz
            z = lo + (np.arange(nz) + 0.5) * dz
            shell = np.searchsorted(R, np.sqrt(p * p + z * z), side="right")
            cut = np.flatnonzero(np.diff(shell)) + 1
            for blk in np.split(shell, cut):
                runs.append(int(blk[0]))
                lens.append(len(blk) * dz)
        assert runs == list(cell)
        np.testing.assert_allclose(lens, s, rtol=0, atol=2 * zmax / nz)
        # entry cosine of each step: z/r at the step's start point
        z0 = -zmax + np.concatenate([[0.0], np.cumsum(s)[:-1]])
        r0 = np.sqrt(p * p + z0 * z0)
        np.testing.assert_allclose(cosv, z0 / r0, atol=1e-12)


@pytest.mark.parametrize("ray_power", [1.0, 2.0, 0.7])
def test_1d_weights_converge_to_volumes(oracle, ray_power):
    """sum_j A_j s_jk -> shell volume as the rays get denser, for equidistant
    and power-law impact parameters (Sect. 2.1)."""
    K = 4
    errs = []
    for n_rays in (500, 4000):
        m = LI.cloud1d_two_level(K=K, n_rays=n_rays)
        m["ray_power"] = ray_power
        R = m["radius"]
        W = oracle.weights_1d(m)
        V = 4.0 / 3.0 * np.pi * (R ** 3 - np.concatenate([[0.0], R[:-1]]) ** 3)
        errs.append(np.abs(W / V - 1.0).max())
    assert errs[1] < 2e-5
    assert errs[1] < errs[0] / 5.0


def _brute_segments(N, F, d, i, j, info):
    """Run-length encoding of the cell hit at every integer z (definition)."""
    H = 1 << F
    E = N * H
    o = H // 2
    m, a, b = info["m"], info["a"], info["b"]
    flip = info["flip"]
    cells, dzs = [], []
    for z in range(E):
        A = (o + i * H + (info["qa"] * z >> F)) % E
        B = (o + j * H + (info["qb"] * z >> F)) % E
        pos = [0, 0, 0]
        pos[m], pos[a], pos[b] = z, A, B
        ci = [((E - 1 - pos[ax]) if flip[ax] else pos[ax]) // H for ax in range(3)]
        c = (ci[2] * N + ci[1]) * N + ci[0]
        if cells and cells[-1] == c:
            dzs[-1] += 1
        else:
            cells.append(c)
            dzs.append(1)
    return cells, dzs


@pytest.mark.parametrize("nside", [1, 2])
def test_3d_brute_force_small_F(oracle, nside):
    N, F = 3, 5
    dirs = LI.healpix_ring_directions(nside)
    for d in dirs[::3]:
        info = oracle.dir_info(d, F)
        for i in range(N):
            for j in range(N):
                cells, dz = oracle.paths_grid3d(N, d, i, j, F)
                bc, bd = _brute_segments(N, F, d, i, j, info)
                assert list(cells) == bc
                assert list(dz) == bd


def test_3d_direction_decomposition(oracle):
    d = np.array([0.3, -0.8, 0.52])
    d /= np.linalg.norm(d)
    info = oracle.dir_info(d, 24)
    assert (info["m"], info["a"], info["b"]) == (1, 0, 2)
    assert info["flip"] == (0, 1, 0)
    assert info["qa"] == int(np.floor(2 ** 24 * 0.3 / 0.8 + 0.5))
    assert info["qb"] == int(np.floor(2 ** 24 * 0.52 / 0.8 + 0.5))


@pytest.mark.parametrize("N", [2, 5])
def test_3d_constant_path_length_exact(oracle, N):
    """Per direction, every cell receives exactly H0 units of main-axis path
    (Sect. 2.2: same path length in all cells); every line spans N H0."""
    F = 24
    H = 1 << F
    for d in LI.healpix_ring_directions(2):
        tot = np.zeros(N ** 3, np.int64)
        for i in range(N):
            for j in range(N):
                cells, dz = oracle.paths_grid3d(N, d, i, j, F)
                assert dz.sum() == N * H
                assert np.all(dz > 0)
                np.add.at(tot, cells, dz)
        assert np.all(tot == H)


def test_1d_power_law_rays(oracle):
    """Power-law impact parameters: the annuli tile the projected disk, ray j
    passes at R ((j + 1/2) / n)^a (so a = 1 is the equidistant default) and
    concentrates towards the centre for a > 1."""
    m = LI.cloud1d_two_level(K=8, n_rays=12)
    R = m["radius"][-1]
    base = [oracle.paths_1d(m, j) for j in range(12)]
    m["ray_power"] = 1.0
    for j in range(12):
        for u, v in zip(base[j], oracle.paths_1d(m, j)):
            np.testing.assert_array_equal(u, v)
    for a in (2.0, 3.0):
        m["ray_power"] = a
        for j in range(12):
            cell, s, _ = oracle.paths_1d(m, j)
            p = R * ((j + 0.5) / 12) ** a
            assert s.sum() == pytest.approx(2.0 * np.sqrt(R * R - p * p), rel=1e-13)
            assert cell.min() == np.searchsorted(m["radius"], p, side="right")
    # the weights of all rays add up to the volume covered: sum_k W_k = sum_j A_j 2 z_j
    m["ray_power"] = 2.0
    W = oracle.weights_1d(m)
    b = R * (np.arange(13) / 12.0) ** 2.0
    A = np.pi * (b[1:] ** 2 - b[:-1] ** 2)
    assert A.sum() == pytest.approx(np.pi * R * R, rel=1e-14)
    p = R * ((np.arange(12) + 0.5) / 12) ** 2.0
    assert W.sum() == pytest.approx((A * 2.0 * np.sqrt(R * R - p * p)).sum(), rel=1e-13)
