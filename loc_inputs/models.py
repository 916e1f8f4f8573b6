"""Seeded synthetic cloud models (1D shells, 3D regular grids, octrees).

Units are CGS throughout: lengths in cm, velocities in cm/s, densities in
cm^-3, temperatures in K.  Every dict carries its velocity-channel grid:
channel k covers [v_min + k dv, v_min + (k+1) dv].

1D model dict (geometry "shells1d"):
  radius[K]      outer radius of each shell, increasing, cm
  n_h2[K], t_kin[K], sigma_turb[K] (cm/s), abundance[K], v[K] (radial, cm/s)
  n_ch, v_min, dv, n_rays, t_bg

3D regular grid dict (geometry "grid3d"): cells indexed x-fastest,
  idx = (iz * N + iy) * N + ix, cube side N * h0.
  n_root, h0, n_h2[N^3], t_kin, sigma_turb, abundance, vx, vy, vz,
  dirs[n_dir, 3], n_ch, v_min, dv, t_bg
"""
import numpy as np

from .healpix import healpix_ring_directions

PC = 3.0856775814913673e18
KMS = 1.0e5
SEED_BASE = 2009_12609


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _channels(n_ch, half_width_kms):
    v_min = -half_width_kms * KMS
    dv = 2.0 * half_width_kms * KMS / n_ch
    return n_ch, v_min, dv


def _thermal_sigma_max(t_kin_max, sigma_turb_kms, mass_amu):
    k_b = 1.380649e-16
    amu = 1.66053906660e-24
    return np.sqrt((sigma_turb_kms * KMS) ** 2 + k_b * t_kin_max / (mass_amu * amu)) / KMS


def cloud1d_two_level(K=32, n_ch=64, n_rays=None, radius_pc=0.1,
                      density_scale=1.0, infall_scale=1.0, t_kin=20.0,
                      abundance=1.0e-9, half_width_kms=2.0):
    """1D infall core of the two-level test: equidistant shells to R,
    n_H2 = min(1e6, 1e5 (r/0.005 pc)^-1.5), constant T_kin, abundance 1e-9,
    sigma_turb 0.2 km/s, v = -0.3 (r/R)^-0.5 km/s, properties evaluated at each
    shell's mid radius; 64 channels over +-2 km/s, one ray per shell."""
    R = radius_pc * PC
    k = np.arange(K, dtype=np.float64)
    radius = (k + 1.0) * R / K
    r_mid = (k + 0.5) * R / K
    n_h2 = density_scale * np.minimum(1.0e6, 1.0e5 * (r_mid / (0.005 * PC)) ** -1.5)
    v = infall_scale * -0.3 * (r_mid / R) ** -0.5 * KMS
    nch, vmin, dv = _channels(n_ch, half_width_kms)
    return dict(geometry="shells1d", radius=radius, n_h2=n_h2,
                t_kin=np.full(K, float(t_kin)), sigma_turb=np.full(K, 0.2 * KMS),
                abundance=np.full(K, float(abundance)), v=v,
                n_ch=nch, v_min=vmin, dv=dv,
                n_rays=K if n_rays is None else int(n_rays), t_bg=2.73)


def cloud1d_rotor(K=256, n_ch=256, seed=SEED_BASE + 1, radius_pc=0.1,
                  abundance=1.0e-5, sigma_ln=0.3, mass_amu=28.0,
                  density_scale=1.0, infall_scale=1.0, t_scale=1.0,
                  r_clamp_frac=0.0, n_rays=None, t_core=0.0, r_core_frac=0.15):
    """1D core for the multilevel rotor: power-law density perturbed by a
    seeded lognormal factor exp(sigma_ln g - sigma_ln^2/2), g ~ N(0,1) per
    shell, T_kin = 10 + 20 r/R K, the same infall law as the two-level core,
    band half-width max(2, max|v| + 6 sigma_max) km/s.  t_core > 0 adds a
    heated centre (an embedded source): T_kin + t_core exp(-(r / r_core)^2)
    with r_core = r_core_frac R."""
    rng = _rng(seed)
    R = radius_pc * PC
    k = np.arange(K, dtype=np.float64)
    radius = (k + 1.0) * R / K
    r_mid = (k + 0.5) * R / K
    r_eval = np.maximum(r_mid, r_clamp_frac * R)
    g = rng.standard_normal(K)
    n_h2 = density_scale * np.minimum(1.0e6, 1.0e5 * (r_eval / (0.005 * PC)) ** -1.5)
    n_h2 = n_h2 * np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    t_kin = t_scale * (10.0 + 20.0 * r_mid / R)
    if t_core > 0.0:
        t_kin = t_kin + t_core * np.exp(-(r_mid / (r_core_frac * R)) ** 2)
    v = infall_scale * -0.3 * (r_eval / R) ** -0.5 * KMS
    sig_max = _thermal_sigma_max(t_kin.max(), 0.2, mass_amu)
    half = max(2.0, np.abs(v).max() / KMS + 6.0 * sig_max)
    nch, vmin, dv = _channels(n_ch, half)
    return dict(geometry="shells1d", radius=radius, n_h2=n_h2, t_kin=t_kin,
                sigma_turb=np.full(K, 0.2 * KMS),
                abundance=np.full(K, float(abundance)), v=v,
                n_ch=nch, v_min=vmin, dv=dv,
                n_rays=K if n_rays is None else int(n_rays), t_bg=2.73)


def uniform_sphere(K=8, n_ch=32, n_rays=None, radius_pc=0.1, n_h2=1.0e4,
                   t_kin=20.0, abundance=1.0e-9, sigma_turb_kms=0.2,
                   v_kms=0.0, half_width_kms=2.0, t_bg=2.73):
    """Static (or uniformly expanding, v_kms) homogeneous sphere on K
    equidistant shells: the special case with closed-form answers."""
    R = radius_pc * PC
    k = np.arange(K, dtype=np.float64)
    nch, vmin, dv = _channels(n_ch, half_width_kms)
    return dict(geometry="shells1d", radius=(k + 1.0) * R / K,
                n_h2=np.full(K, float(n_h2)), t_kin=np.full(K, float(t_kin)),
                sigma_turb=np.full(K, sigma_turb_kms * KMS),
                abundance=np.full(K, float(abundance)),
                v=np.full(K, v_kms * KMS), n_ch=nch, v_min=vmin, dv=dv,
                n_rays=K if n_rays is None else int(n_rays), t_bg=float(t_bg))


def serving_requests(n=4096, seed=SEED_BASE + 4, rate_hz=None,
                     k_range=(32, 1024), ch_choices=(64, 128, 256, 512),
                     level_range=(2, 20)):
    """Stream of 1D model requests: shells ~ U{32..1024}, channels from
    {64,128,256,512}, rotor ladder truncated to U{2..20} levels; density,
    infall and T_kin scale factors each log-uniform in [0.1, 10].  Returns a
    list of dicts with keys model, n_levels, arrival_s (Poisson arrivals at
    rate_hz, or all at t=0 when rate_hz is None) and seed."""
    rng = _rng(seed)
    out = []
    t = 0.0
    for i in range(n):
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        nch = int(rng.choice(np.array(ch_choices)))
        nlev = int(rng.integers(level_range[0], level_range[1] + 1))
        f = 10.0 ** rng.uniform(-1.0, 1.0, size=3)
        mseed = int(rng.integers(0, 2 ** 31 - 1))
        if rate_hz:
            t += rng.exponential(1.0 / rate_hz)
        model = cloud1d_rotor(K=K, n_ch=nch, seed=mseed, density_scale=f[0],
                              infall_scale=f[1], t_scale=f[2], r_clamp_frac=0.05)
        out.append(dict(model=model, n_levels=nlev, arrival_s=t, seed=mseed))
    return out


# ----------------------------------------------------------------------------
# 3D fields
# ----------------------------------------------------------------------------

def _grf(rng, N, index=-11.0 / 3.0):
    """Unit-variance Gaussian random field on an N^3 periodic grid with power
    spectrum P(k) ~ k^index (k = 0 mode removed)."""
    w = rng.standard_normal((N, N, N))
    f = np.fft.fftn(w)
    kx = np.fft.fftfreq(N)
    kk = np.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kx[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    amp[kk > 0] = kk[kk > 0] ** (index / 2.0)
    g = np.real(np.fft.ifftn(f * amp))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else np.zeros_like(g)     # N = 1: a uniform field


def _fields3d(N, seed, mean_density=1.0e4, sigma_ln=1.0, v_rms_kms=1.0):
    rng = _rng(seed)
    g = _grf(rng, N)
    n_h2 = np.exp(np.log(mean_density) - 0.5 * sigma_ln ** 2 + sigma_ln * g)
    vel = [_grf(rng, N) * (v_rms_kms * KMS / np.sqrt(3.0)) for _ in range(3)]
    # arrays come out [i0][i1][i2]; read them as [iz][iy][ix] (x fastest)
    return n_h2, vel


def grid3d_cloud(N=128, n_ch=128, seed=SEED_BASE + 2, box_pc=1.0, t_kin=15.0,
                 abundance=1.0e-6, half_width_kms=3.0, nside=2):
    """Regular N^3 grid: lognormal density from a -11/3 Gaussian random
    field (sigma_ln 1, mean 1e4 cm^-3), three independent velocity
    components with the same spectrum and 3D rms 1 km/s, T_kin 15 K,
    sigma_turb 0.2 km/s, 128 channels over +-3 km/s, 48 HEALPix directions.
    Box 1 pc and abundance 1e-6 give the J=1-0 line line-of-sight optical
    depths of a few on average and up to ~100 through the densest cells
    (partially optically thick)."""
    n_h2, (vx, vy, vz) = _fields3d(N, seed)
    M = N ** 3
    nch, vmin, dv = _channels(n_ch, half_width_kms)
    return dict(geometry="grid3d", n_root=N, h0=box_pc * PC / N,
                n_h2=n_h2.reshape(M), t_kin=np.full(M, float(t_kin)),
                sigma_turb=np.full(M, 0.2 * KMS),
                abundance=np.full(M, float(abundance)),
                vx=vx.reshape(M), vy=vy.reshape(M), vz=vz.reshape(M),
                dirs=healpix_ring_directions(nside), n_ch=nch, v_min=vmin,
                dv=dv, t_bg=2.73)


def small_grid3d(N=4, n_ch=16, seed=7, box_pc=0.05, abundance=1.0e-4, nside=1):
    """A few-cell regular grid for brute-force and parity tests."""
    return grid3d_cloud(N=N, n_ch=n_ch, seed=seed, box_pc=box_pc,
                        abundance=abundance, nside=nside)


def _octree_from_fields(N, n0, v0, levels, threshold, rng, cascade_ln=0.5, cascade_v_kms=0.2,
                        refine_mask=None):
    """Level-ordered octree: level-0 cells in raster order (x fastest), then
    the 8 children (octant cx + 2 cy + 4 cz) of every refined cell of the
    previous level, in the order of their parents.  A cell is refined when
    its density exceeds `threshold` (or where refine_mask says so for the
    root level) and it is above the deepest level.  Children draw
    ln n_child = ln n_parent + cascade_ln g - cascade_ln^2 / 2 and
    v_child = v_parent + cascade_v 2^(-L/3) g_vec (seeded)."""
    dens = [n0.reshape(-1)]
    vel = [v0.reshape(-1, 3)]
    refine = []
    for L in range(levels + 1):
        d = dens[L]
        if L < levels:
            if L == 0 and refine_mask is not None:
                r = refine_mask.reshape(-1).astype(np.int32)
            else:
                r = (d > threshold).astype(np.int32)
        else:
            r = np.zeros(len(d), np.int32)
        refine.append(r)
        if L == levels or not r.any():
            break
        par = np.flatnonzero(r)
        ln = np.repeat(np.log(d[par]), 8) + cascade_ln * rng.standard_normal(8 * len(par)) - 0.5 * cascade_ln ** 2
        dv = cascade_v_kms * KMS * 2.0 ** (-(L + 1) / 3.0)
        vv = np.repeat(vel[L][par], 8, axis=0) + dv * rng.standard_normal((8 * len(par), 3))
        dens.append(np.exp(ln))
        vel.append(vv)
    n_h2 = np.concatenate(dens)
    v = np.concatenate(vel)
    flags = np.concatenate(refine).astype(np.int32)
    return n_h2, v, flags, len(refine) - 1


def octree_cloud(N=64, levels=5, n_ch=64, seed=SEED_BASE + 3, box_pc=1.0, t_kin=15.0,
                 abundance=1.0e-6, half_width_kms=3.0, nside=2, refine_factor=8.0):
    """Octree cloud: 64^3 root with the lognormal density and velocity fields of
    the regular-grid cloud, refined (up to `levels` levels) wherever the
    density exceeds refine_factor x the mean 1e4 cm^-3; sub-root values from
    a seeded multiplicative cascade.  Dict keys: geometry "octree3d", n_root,
    h0, levels, refine[n_cells] (level-ordered flags), per-cell n_h2, t_kin,
    sigma_turb, abundance, vx, vy, vz, dirs, channel grid, t_bg."""
    rng = _rng(seed)
    n0, (vx, vy, vz) = _fields3d(N, seed)
    v0 = np.stack([vx.reshape(-1), vy.reshape(-1), vz.reshape(-1)], axis=1)
    n_h2, v, flags, depth = _octree_from_fields(N, n0, v0, levels, refine_factor * 1.0e4, rng)
    M = len(n_h2)
    nch, vmin, dv = _channels(n_ch, half_width_kms)
    return dict(geometry="octree3d", n_root=N, h0=box_pc * PC / N, levels=depth,
                refine=flags, n_h2=n_h2, t_kin=np.full(M, float(t_kin)),
                sigma_turb=np.full(M, 0.2 * KMS), abundance=np.full(M, float(abundance)),
                vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(),
                dirs=healpix_ring_directions(nside), n_ch=nch, v_min=vmin, dv=dv, t_bg=2.73)


def small_octree(N=4, levels=2, n_ch=16, seed=11, box_pc=0.05, abundance=1.0e-5, nside=1,
                 refine_frac=0.3):
    """A few-cell octree for brute-force and parity tests: about refine_frac
    of the cells of each level are refined (threshold at that quantile of
    the level's densities)."""
    rng = _rng(seed)
    n0, (vx, vy, vz) = _fields3d(N, seed)
    v0 = np.stack([vx.reshape(-1), vy.reshape(-1), vz.reshape(-1)], axis=1)
    thr = float(np.quantile(n0, 1.0 - refine_frac)) if N > 1 else 0.0
    mask = n0.reshape(-1) > thr if N > 1 else np.ones(1, bool)
    n_h2, v, flags, depth = _octree_from_fields(N, n0, v0, levels, thr, rng, refine_mask=mask)
    M = len(n_h2)
    nch, vmin, dv = _channels(n_ch, 3.0)
    return dict(geometry="octree3d", n_root=N, h0=box_pc * PC / N, levels=depth,
                refine=flags, n_h2=n_h2, t_kin=np.full(M, 15.0),
                sigma_turb=np.full(M, 0.2 * KMS), abundance=np.full(M, float(abundance)),
                vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(),
                dirs=healpix_ring_directions(nside), n_ch=nch, v_min=vmin, dv=dv, t_bg=2.73)
