"""FP64 CPU oracle of the LOC ALI line-transfer hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product library
never imports this package and shares no code with it.

The arithmetic lives in ``loc_oracle.c`` (plain C, FP64, OpenMP over rays or
lines); this module builds it with gcc and marshals numpy arrays to it.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "loc_oracle.c")
_LIB = os.path.join(_HERE, "liblocoracle.so")
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force=False):
    """Compile loc_oracle.c into liblocoracle.so next to it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Molecule(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("n_lines", ctypes.c_int),
                ("n_coll", ctypes.c_int),
                ("energy_K", _d), ("g", _d), ("mass_amu", ctypes.c_double),
                ("line_u", _i), ("line_l", _i), ("line_A", _d), ("line_nu", _d),
                ("coll_u", _i), ("coll_l", _i), ("coll_k", _d),
                ("hf_off", _i), ("hf_v", _d), ("hf_w", _d)]


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.lo_max_rel_dtex.restype = ctypes.c_double
        _lib.lo_bg_occupation.restype = ctypes.c_double
        _lib.lo_bg_occupation.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.lo_paths_grid3d.restype = ctypes.c_int64
        _lib.lo_num_threads.restype = ctypes.c_int
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    if a.dtype == np.float64:
        return a.ctypes.data_as(_d)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_i)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_i64)
    raise TypeError(a.dtype)


class _Mol:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, mol, n_levels=None):
        L = len(mol["g"]) if n_levels is None else int(n_levels)
        self.arrs = dict(
            energy_K=_f64(mol["energy_K"][:L]), g=_f64(mol["g"][:L]),
        )
        lu = np.asarray(mol["line_u"], np.int32)
        ll = np.asarray(mol["line_l"], np.int32)
        keep = (lu < L) & (ll < L)
        self.arrs.update(line_u=np.ascontiguousarray(lu[keep]),
                         line_l=np.ascontiguousarray(ll[keep]),
                         line_A=_f64(np.asarray(mol["line_A"])[keep]),
                         line_nu=_f64(np.asarray(mol["line_nu"])[keep]))
        cu = np.asarray(mol["coll_u"], np.int32)
        cl = np.asarray(mol["coll_l"], np.int32)
        keepc = (cu < L) & (cl < L)
        self.arrs.update(coll_u=np.ascontiguousarray(cu[keepc]),
                         coll_l=np.ascontiguousarray(cl[keepc]),
                         coll_k=_f64(np.asarray(mol["coll_k"])[keepc]))
        # hyperfine components of the kept lines (hf_n per line, offsets and
        # strengths concatenated in line order)
        hf = None
        if mol.get("hf_n") is not None:
            n = np.asarray(mol["hf_n"], np.int64)
            off = np.concatenate([[0], np.cumsum(n)])
            idx = np.concatenate([np.arange(off[t], off[t + 1]) for t in np.flatnonzero(keep)] + [[]])
            idx = idx.astype(np.int64)
            kn = n[keep]
            self.arrs.update(hf_off=np.ascontiguousarray(np.concatenate([[0], np.cumsum(kn)]), np.int32),
                             hf_v=_f64(np.asarray(mol["hf_v"], np.float64)[idx]),
                             hf_w=_f64(np.asarray(mol["hf_w"], np.float64)[idx]))
            hf = self.arrs
        a = self.arrs
        self.L = L
        self.T = len(a["line_u"])
        self.nu = a["line_nu"]
        self.s = _Molecule(L, self.T, len(a["coll_u"]), _p(a["energy_K"]), _p(a["g"]),
                           float(mol["mass_amu"]), _p(a["line_u"]), _p(a["line_l"]),
                           _p(a["line_A"]), _p(a["line_nu"]), _p(a["coll_u"]),
                           _p(a["coll_l"]), _p(a["coll_k"]),
                           _p(hf["hf_off"]) if hf else None, _p(hf["hf_v"]) if hf else None,
                           _p(hf["hf_w"]) if hf else None)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def n_threads():
    return _load().lo_num_threads()


def bg_occupation(nu, t_bg):
    return _load().lo_bg_occupation(float(nu), float(t_bg))


def lte_populations(mol, t_kin, n_levels=None):
    lib = _load()
    M = _Mol(mol, n_levels)
    t = _f64(t_kin)
    x = np.zeros((len(t), M.L))
    lib.lo_lte_populations(M.L, _p(M.arrs["energy_K"]), _p(M.arrs["g"]), len(t), _p(t), _p(x))
    return x


def profile(n_ch, v_min, dv, v_los, sigma):
    lib = _load()
    phi = np.zeros(n_ch)
    lib.lo_profile(int(n_ch), ctypes.c_double(v_min), ctypes.c_double(dv),
                   ctypes.c_double(v_los), ctypes.c_double(sigma), _p(phi))
    return phi


def line_params(mol, model, x, n_levels=None):
    """(Kp, S) as [line][cell] arrays for populations x[cell][level]."""
    lib = _load()
    M = _Mol(mol, n_levels)
    n = len(model["n_h2"])
    Kp = np.zeros((M.T, n))
    S = np.zeros((M.T, n))
    lib.lo_line_params(M.ref, n, _p(_f64(model["n_h2"])), _p(_f64(model["abundance"])),
                       ctypes.c_double(model["dv"]), _p(_f64(x)), _p(Kp), _p(S))
    return Kp, S


def _ray_power(model):
    """Exponent a of the impact parameters p_j = R ((j + 1/2) / n)^a (1: equidistant)."""
    a = float(model.get("ray_power", 0.0) or 0.0)
    return ctypes.c_double(a if a > 0.0 else 1.0)


def paths_1d(model, j):
    """Segment list (cell, s, cos) of ray j of a 1D model."""
    lib = _load()
    R = _f64(model["radius"])
    K = len(R)
    cell = np.zeros(2 * K + 2, np.int32)
    s = np.zeros(2 * K + 2)
    cv = np.zeros(2 * K + 2)
    n = lib.lo_paths_1d(K, _p(R), int(model["n_rays"]), _ray_power(model), int(j), _p(cell), _p(s),
                        _p(cv))
    return cell[:n].copy(), s[:n].copy(), cv[:n].copy()


def weights_1d(model):
    lib = _load()
    R = _f64(model["radius"])
    W = np.zeros(len(R))
    lib.lo_weights_1d(len(R), _p(R), int(model["n_rays"]), _ray_power(model), _p(W))
    return W


def march_1d(mol, model, Kp, S, n_levels=None):
    """One ray simulation of a 1D model -> (SIJ[line][cell], ESC, NORM[cell])."""
    lib = _load()
    M = _Mol(mol, n_levels)
    K = len(model["radius"])
    SIJ = np.zeros((M.T, K))
    ESC = np.zeros((M.T, K))
    NORM = np.zeros(K)
    lib.lo_march_1d(M.ref, K, _p(_f64(model["radius"])), _p(_f64(model["t_kin"])),
                    _p(_f64(model["sigma_turb"])), _p(_f64(model["v"])),
                    int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                    ctypes.c_double(model["dv"]), int(model["n_rays"]), _ray_power(model),
                    ctypes.c_double(model["t_bg"]), _p(_f64(Kp)), _p(_f64(S)),
                    _p(SIJ), _p(ESC), _p(NORM))
    return SIJ, ESC, NORM


def march_1d_sub(mol, model, Kp, S, k_sub, mode, Ib=None, n_levels=None):
    """Ray simulation with the region of the k_sub innermost shells.
    mode 0: all rays; returns (SIJ, ESC, NORM, Ib) with Ib[j][line][channel]
    the intensity ray j carries into the region.  mode 1: the region's steps
    of the rays that reach it, starting from Ib; returns (SIJ, ESC, NORM)."""
    lib = _load()
    M = _Mol(mol, n_levels)
    K = len(model["radius"])
    SIJ = np.zeros((M.T, K))
    ESC = np.zeros((M.T, K))
    NORM = np.zeros(K)
    j_end = sub_rays_1d(model, k_sub)
    if mode == 0:
        Ib = np.zeros((max(j_end, 1), M.T, int(model["n_ch"])))
    else:
        Ib = _f64(Ib)
    lib.lo_march_1d_sub(M.ref, K, _p(_f64(model["radius"])), _p(_f64(model["t_kin"])),
                        _p(_f64(model["sigma_turb"])), _p(_f64(model["v"])),
                        int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                        ctypes.c_double(model["dv"]), int(model["n_rays"]), _ray_power(model),
                        ctypes.c_double(model["t_bg"]), _p(_f64(Kp)), _p(_f64(S)), int(k_sub),
                        int(mode), int(j_end), _p(Ib), _p(SIJ), _p(ESC), _p(NORM))
    return (SIJ, ESC, NORM, Ib[:j_end]) if mode == 0 else (SIJ, ESC, NORM)


def sub_rays_1d(model, k_sub):
    """Number of rays (j < j_end) that cross the k_sub innermost shells."""
    lib = _load()
    R = _f64(model["radius"])
    return lib.lo_sub_rays_1d(len(R), _p(R), int(model["n_rays"]), _ray_power(model), int(k_sub))


def iterate_1d_sub(mol, model, n_iter, n_sub, k_sub, ali=True, x0=None, n_levels=None):
    """n_iter ALI iterations, each followed by n_sub sub-iterations of the
    k_sub innermost shells.  Returns (x, dtex[n_iter])."""
    lib = _load()
    M = _Mol(mol, n_levels)
    K = len(model["radius"])
    x = lte_populations(mol, model["t_kin"], n_levels) if x0 is None else _f64(x0).copy()
    dt = np.zeros(max(1, n_iter))
    bad = lib.lo_iterate_1d_sub(M.ref, K, _p(_f64(model["radius"])), _p(_f64(model["n_h2"])),
                                _p(_f64(model["t_kin"])), _p(_f64(model["sigma_turb"])),
                                _p(_f64(model["abundance"])), _p(_f64(model["v"])),
                                int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                                ctypes.c_double(model["dv"]), int(model["n_rays"]), _ray_power(model),
                                ctypes.c_double(model["t_bg"]), int(bool(ali)), int(n_iter),
                                int(n_sub), int(k_sub), _p(x), _p(dt))
    if bad:
        raise ArithmeticError(f"{bad} singular rate matrices")
    return x, dt[:n_iter]


def line_off(mol, x, cutoff, n_levels=None):
    """Per-cell line truncation mask [line][cell] (uint8) for populations x."""
    lib = _load()
    M = _Mol(mol, n_levels)
    x = _f64(x)
    n = x.shape[0]
    off = np.zeros((M.T, n), np.uint8)
    lib.lo_line_off(M.ref, n, _p(x), ctypes.c_double(cutoff),
                    off.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return off


def se_solve(mol, model, SIJ, ESC, NORM, S, ali=True, n_levels=None, off=None):
    """Equilibrium populations; off: optional [line][cell] truncation mask
    (those lines take J = n_bg, beta = 1)."""
    lib = _load()
    M = _Mol(mol, n_levels)
    n = len(model["n_h2"])
    x = np.zeros((n, M.L))
    if off is None:
        offp = None
    else:
        off = np.ascontiguousarray(off, dtype=np.uint8)
        offp = off.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    bad = lib.lo_se_solve_off(M.ref, n, _p(_f64(model["n_h2"])), _p(_f64(model["t_kin"])),
                              ctypes.c_double(model["t_bg"]), int(bool(ali)), _p(_f64(SIJ)),
                              _p(_f64(ESC)), _p(_f64(NORM)), _p(_f64(S)), offp, _p(x))
    if bad:
        raise ArithmeticError(f"{bad} singular rate matrices")
    return x


def tex(mol, x, n_levels=None):
    lib = _load()
    M = _Mol(mol, n_levels)
    x = _f64(x)
    n = x.shape[0]
    out = np.zeros((M.T, n))
    lib.lo_tex(M.ref, n, _p(x), _p(out))
    return out


def max_rel_dtex(mol, x_old, x_new, n_levels=None):
    lib = _load()
    M = _Mol(mol, n_levels)
    x_old = _f64(x_old)
    return lib.lo_max_rel_dtex(M.ref, x_old.shape[0], _p(x_old), _p(_f64(x_new)))


def iterate_1d(mol, model, n_iter, ali=True, x0=None, n_levels=None, level_cutoff=0.0):
    """Run n_iter ALI iterations from LTE (or x0), with per-cell line
    truncation when level_cutoff > 0.  Returns (x, dtex[n_iter])."""
    lib = _load()
    M = _Mol(mol, n_levels)
    K = len(model["radius"])
    x = lte_populations(mol, model["t_kin"], n_levels) if x0 is None else _f64(x0).copy()
    dt = np.zeros(max(1, n_iter))
    bad = lib.lo_iterate_1d_cut(M.ref, K, _p(_f64(model["radius"])), _p(_f64(model["n_h2"])),
                                _p(_f64(model["t_kin"])), _p(_f64(model["sigma_turb"])),
                                _p(_f64(model["abundance"])), _p(_f64(model["v"])),
                                int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                                ctypes.c_double(model["dv"]), int(model["n_rays"]), _ray_power(model),
                                ctypes.c_double(model["t_bg"]), int(bool(ali)), int(n_iter),
                                ctypes.c_double(level_cutoff), _p(x), _p(dt))
    if bad:
        raise ArithmeticError(f"{bad} singular rate matrices")
    return x, dt[:n_iter]


def spectra_1d(mol, model, x, line, p, n_levels=None):
    """T_RJ [n_p][n_ch] for impact parameters p (cm)."""
    lib = _load()
    M = _Mol(mol, n_levels)
    K = len(model["radius"])
    p = _f64(np.atleast_1d(p))
    out = np.zeros((len(p), int(model["n_ch"])))
    lib.lo_spectra_1d(M.ref, int(line), K, _p(_f64(model["radius"])), _p(_f64(model["n_h2"])),
                      _p(_f64(model["t_kin"])), _p(_f64(model["sigma_turb"])),
                      _p(_f64(model["abundance"])), _p(_f64(model["v"])),
                      int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                      ctypes.c_double(model["dv"]), ctypes.c_double(model["t_bg"]),
                      _p(_f64(x)), len(p), _p(p), _p(out))
    return out


# ---------------------------------------------------------------------------
# 3D regular grid
# ---------------------------------------------------------------------------
FIXED_BITS = 24


def dir_info(d, F=FIXED_BITS):
    lib = _load()
    mabf = np.zeros(6, np.int32)
    q = np.zeros(2, np.int64)
    lib.lo_dir_info(_p(_f64(d)), int(F), _p(mabf), _p(q))
    return dict(m=int(mabf[0]), a=int(mabf[1]), b=int(mabf[2]),
                flip=tuple(int(v) for v in mabf[3:]), qa=int(q[0]), qb=int(q[1]))


def paths_grid3d(N, d, i, j, F=FIXED_BITS):
    """(cells, dz) of root line (i, j) for direction d on an N^3 grid."""
    lib = _load()
    cap = 4 * N + 16
    cells = np.zeros(cap, np.int64)
    dz = np.zeros(cap, np.int64)
    n = lib.lo_paths_grid3d(int(N), int(F), _p(_f64(d)), ctypes.c_int64(i), ctypes.c_int64(j),
                            _p(cells), _p(dz), ctypes.c_int64(cap))
    if n < 0:
        raise RuntimeError("segment buffer too small")
    return cells[:n].copy(), dz[:n].copy()


def march_grid3d(mol, model, Kp, S, F=FIXED_BITS, dir_range=None, ray_stride=1,
                 n_levels=None):
    lib = _load()
    M = _Mol(mol, n_levels)
    N = int(model["n_root"])
    nc = N ** 3
    dirs = _f64(model["dirs"])
    nd = len(dirs)
    lo, hi = (0, nd) if dir_range is None else dir_range
    SIJ = np.zeros((M.T, nc))
    ESC = np.zeros((M.T, nc))
    NORM = np.zeros(nc)
    lib.lo_march_grid3d(M.ref, N, ctypes.c_double(model["h0"]), int(F),
                        _p(_f64(model["t_kin"])), _p(_f64(model["sigma_turb"])),
                        _p(_f64(model["vx"])), _p(_f64(model["vy"])), _p(_f64(model["vz"])),
                        nd, _p(dirs), int(lo), int(hi), int(ray_stride),
                        int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                        ctypes.c_double(model["dv"]), ctypes.c_double(model["t_bg"]),
                        _p(_f64(Kp)), _p(_f64(S)), _p(SIJ), _p(ESC), _p(NORM))
    return SIJ, ESC, NORM


def _truncated_step(mol, model, x, march, ali, level_cutoff, n_levels):
    """One ALI iteration with per-cell line truncation (lo_line_off reading):
    off lines get Kp = S = 0 in the march and J = n_bg, beta = 1 in the solve."""
    Kp, S = line_params(mol, model, x, n_levels)
    off = line_off(mol, x, level_cutoff, n_levels)
    Kp[off == 1] = 0.0
    S[off == 1] = 0.0
    SIJ, ESC, NORM = march(Kp, S)
    return se_solve(mol, model, SIJ, ESC, NORM, S, ali, n_levels, off=off)


def iterate_grid3d(mol, model, n_iter, ali=True, x0=None, F=FIXED_BITS, n_levels=None,
                   level_cutoff=0.0):
    """n_iter ALI iterations on a regular grid (per-cell line truncation when
    level_cutoff > 0).  Returns (x, dtex[n_iter])."""
    lib = _load()
    M = _Mol(mol, n_levels)
    N = int(model["n_root"])
    x = lte_populations(mol, model["t_kin"], n_levels) if x0 is None else _f64(x0).copy()
    if level_cutoff > 0.0:
        dt = np.zeros(n_iter)
        for it in range(n_iter):
            xn = _truncated_step(mol, model, x, lambda K_, S_: march_grid3d(mol, model, K_, S_, F, n_levels=n_levels),
                                 ali, level_cutoff, n_levels)
            dt[it] = max_rel_dtex(mol, x, xn, n_levels)
            x = xn
        return x, dt
    dt = np.zeros(max(1, n_iter))
    dirs = _f64(model["dirs"])
    bad = lib.lo_iterate_grid3d(M.ref, N, ctypes.c_double(model["h0"]), int(F),
                                _p(_f64(model["n_h2"])), _p(_f64(model["t_kin"])),
                                _p(_f64(model["sigma_turb"])), _p(_f64(model["abundance"])),
                                _p(_f64(model["vx"])), _p(_f64(model["vy"])), _p(_f64(model["vz"])),
                                len(dirs), _p(dirs), int(model["n_ch"]),
                                ctypes.c_double(model["v_min"]), ctypes.c_double(model["dv"]),
                                ctypes.c_double(model["t_bg"]), int(bool(ali)), int(n_iter),
                                _p(x), _p(dt))
    if bad:
        raise ArithmeticError(f"{bad} singular rate matrices")
    return x, dt[:n_iter]


# ---------------------------------------------------------------------------
# octree
# ---------------------------------------------------------------------------

def _tree_args(model):
    refine = np.ascontiguousarray(model["refine"], dtype=np.int32)
    return int(model["n_root"]), int(model["levels"]), refine


def octree_line_segments(model, d, lam, i, j, F=FIXED_BITS):
    """Segments (z0, dz, cell, level, active) of lattice line (lam, i, j)."""
    lib = _load()
    N, Lmax, refine = _tree_args(model)
    cap = 1 << 16
    out = np.zeros((cap, 5), np.int64)
    lib.lo_octree_line_segments.restype = ctypes.c_int64
    n = lib.lo_octree_line_segments(N, Lmax, int(F), ctypes.c_int64(len(refine)), _p(refine),
                                    _p(_f64(d)), int(lam), ctypes.c_int64(i), ctypes.c_int64(j),
                                    _p(out), ctypes.c_int64(cap))
    if n < 0:
        raise ValueError("inconsistent refinement flags")
    return out[:n].copy()


def octree_path_sums(model, d, F=FIXED_BITS):
    """Per-cell total active main-axis path of one direction (int64)."""
    lib = _load()
    N, Lmax, refine = _tree_args(model)
    out = np.zeros(len(refine), np.int64)
    lib.lo_octree_path_sums.restype = ctypes.c_int64
    n = lib.lo_octree_path_sums(N, Lmax, int(F), ctypes.c_int64(len(refine)), _p(refine),
                                _p(_f64(d)), _p(out))
    if n < 0:
        raise ValueError("inconsistent refinement flags")
    return out


def leaves(model):
    return np.flatnonzero(np.asarray(model["refine"]) == 0)


def march_octree(mol, model, Kp_leaf, S_leaf, F=FIXED_BITS, n_levels=None):
    """One ray simulation on an octree; K, S given per leaf [line][leaf];
    returns SIJ, ESC [line][leaf] and NORM [leaf]."""
    lib = _load()
    M = _Mol(mol, n_levels)
    N, Lmax, refine = _tree_args(model)
    nc = len(refine)
    lf = leaves(model)
    Kp = np.zeros((M.T, nc))
    S = np.zeros((M.T, nc))
    Kp[:, lf] = Kp_leaf
    S[:, lf] = S_leaf
    SIJ = np.zeros((M.T, nc))
    ESC = np.zeros((M.T, nc))
    NORM = np.zeros(nc)
    dirs = _f64(model["dirs"])
    r = lib.lo_march_octree(M.ref, N, Lmax, int(F), ctypes.c_int64(nc), _p(refine),
                            ctypes.c_double(model["h0"]), _p(_f64(model["t_kin"])),
                            _p(_f64(model["sigma_turb"])), _p(_f64(model["vx"])),
                            _p(_f64(model["vy"])), _p(_f64(model["vz"])), len(dirs), _p(dirs),
                            int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                            ctypes.c_double(model["dv"]), ctypes.c_double(model["t_bg"]),
                            _p(Kp), _p(S), _p(SIJ), _p(ESC), _p(NORM))
    if r != 0:
        raise ValueError("inconsistent refinement flags")
    return SIJ[:, lf], ESC[:, lf], NORM[lf]


def leaf_model(model):
    """Per-leaf view of an octree model (for line parameters and the SE)."""
    lf = leaves(model)
    out = dict(model)
    for key in ("n_h2", "t_kin", "sigma_turb", "abundance", "vx", "vy", "vz"):
        out[key] = np.asarray(model[key])[lf]
    return out


def iterate_octree(mol, model, n_iter, ali=True, x0=None, F=FIXED_BITS, n_levels=None,
                   level_cutoff=0.0):
    """n_iter ALI iterations on an octree; populations per leaf (per-cell line
    truncation when level_cutoff > 0)."""
    lm = leaf_model(model)
    x = lte_populations(mol, lm["t_kin"], n_levels) if x0 is None else _f64(x0).copy()
    dt = np.zeros(n_iter)
    for it in range(n_iter):
        if level_cutoff > 0.0:
            xn = _truncated_step(mol, lm, x, lambda K_, S_: march_octree(mol, model, K_, S_, F, n_levels),
                                 ali, level_cutoff, n_levels)
        else:
            Kp, S = line_params(mol, lm, x, n_levels)
            SIJ, ESC, NORM = march_octree(mol, model, Kp, S, F, n_levels)
            xn = se_solve(mol, lm, SIJ, ESC, NORM, S, ali, n_levels)
        dt[it] = max_rel_dtex(mol, x, xn, n_levels)
        x = xn
    return x, dt


def map_3d(mol, model, x, line, d, lam=0, pix_stride=1, F=FIXED_BITS, n_levels=None):
    """Emergent map of a 3D model (grid or octree) along unit direction d:
    T_RJ [M * M][n_ch], M = n_root << lam, pixel (i, j) at row i * M + j
    (i along the direction's first transverse axis, j along the second);
    x: populations per cell (grid) or per leaf (octree).  Only pixels with
    index % pix_stride == 0 are computed (others are 0)."""
    lib = _load()
    M_ = _Mol(mol, n_levels)
    N = int(model["n_root"])
    if model["geometry"] == "octree3d":
        _, Lmax, refine = _tree_args(model)
        lf = leaves(model)
        Kl, Sl = line_params(mol, leaf_model(model), x, n_levels)
        nc = len(refine)
        Kp = np.zeros((M_.T, nc))
        S = np.zeros((M_.T, nc))
        Kp[:, lf] = Kl
        S[:, lf] = Sl
    else:
        Lmax, nc = 0, N ** 3
        refine = np.zeros(nc, np.int32)
        Kp, S = line_params(mol, model, x, n_levels)
        if lam != 0:
            raise ValueError("a regular grid has level-0 pixels only")
    Mp = N << lam
    T = np.zeros((Mp * Mp, int(model["n_ch"])))
    lib.lo_map_3d.restype = ctypes.c_int
    r = lib.lo_map_3d(M_.ref, int(line), N, int(Lmax), int(F), ctypes.c_int64(nc), _p(refine),
                      ctypes.c_double(model["h0"]), _p(_f64(model["t_kin"])),
                      _p(_f64(model["sigma_turb"])), _p(_f64(model["vx"])), _p(_f64(model["vy"])),
                      _p(_f64(model["vz"])), _p(_f64(d)), int(lam), ctypes.c_int64(pix_stride),
                      int(model["n_ch"]), ctypes.c_double(model["v_min"]),
                      ctypes.c_double(model["dv"]), ctypes.c_double(model["t_bg"]),
                      _p(_f64(Kp)), _p(_f64(S)), _p(T))
    if r != 0:
        raise ValueError("inconsistent refinement flags")
    return T
