"""Thin ctypes binding of the LOC C ABI (include/loc.h).

Functions carry the C names (loc_create_model, loc_set_molecule,
loc_iterate, ...) and only marshal numpy arrays into the C structs; every
step of the method runs in the CUDA library.  The library must be built
(``paper_2009_12609_gb300.build.build()``); if it is missing, loading fails
with an error -- there is no fallback implementation.

Device memory is requested from PyTorch's caching allocator (through the
C allocator hook) and work is queued on PyTorch's current CUDA stream, so
the library composes with other CUDA work of the process.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LOC_OK = 0
LOC_EINVAL = -1
LOC_ENOMEM = -2
LOC_ECUDA = -3
LOC_ETIMEOUT = -4
LOC_ENOTCONV = -5
LOC_ESTATE = -6
LOC_EBUSY = -7

LOC_SHELLS_1D = 1
LOC_GRID_3D = 2
LOC_OCTREE_3D = 3

LOC_FP32_MARCH = 0
LOC_FP64_ACC = 1
LOC_FP32_PLAIN = 2

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class loc_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", _vp)]


class loc_model_desc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("n_shells", ctypes.c_int), ("radius", _d),
                ("n_rays", ctypes.c_int), ("n_root", ctypes.c_int), ("h0", ctypes.c_double),
                ("n_dir", ctypes.c_int), ("dirs", _d), ("octree_levels", ctypes.c_int),
                ("octree_refine", _i32), ("octree_n_cells", ctypes.c_int64),
                ("n_h2", _d), ("t_kin", _d), ("sigma_turb", _d), ("abundance", _d),
                ("v", _d), ("vx", _d), ("vy", _d), ("vz", _d),
                ("n_ch", ctypes.c_int), ("v_min", ctypes.c_double), ("dv", ctypes.c_double),
                ("t_bg", ctypes.c_double), ("stream", _vp),
                ("allocator", ctypes.POINTER(loc_allocator)), ("ray_power", ctypes.c_double),
                ("octree_paths", ctypes.c_int)]


class loc_molecule_desc(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("energy_K", _d), ("g", _d),
                ("mass_amu", ctypes.c_double), ("n_lines", ctypes.c_int),
                ("line_u", _i32), ("line_l", _i32), ("line_A", _d), ("line_nu", _d),
                ("n_coll", ctypes.c_int), ("coll_u", _i32), ("coll_l", _i32),
                ("coll_k", _d), ("hf_n", _i32), ("hf_v", _d), ("hf_w", _d)]


class loc_iter_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol_tex", ctypes.c_double),
                ("ali", ctypes.c_int), ("precision", ctypes.c_int),
                ("lines_per_pass", ctypes.c_int), ("window_sigmas", ctypes.c_double),
                ("profile", ctypes.c_int), ("steps_per_chunk", ctypes.c_int),
                ("level_cutoff", ctypes.c_double), ("dir_begin", ctypes.c_int),
                ("dir_end", ctypes.c_int), ("sub_iters", ctypes.c_int), ("sub_shells", ctypes.c_int)]


class loc_iter_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("max_rel_dtex", ctypes.c_double),
                ("segments", ctypes.c_int64), ("updates", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("n_maser_cells", ctypes.c_int64),
                ("march_ms", ctypes.c_double), ("se_ms", ctypes.c_double),
                ("params_ms", ctypes.c_double), ("march_launches", ctypes.c_int64),
                ("computed_updates", ctypes.c_double), ("nominal_updates", ctypes.c_double),
                ("path_records", ctypes.c_int64),
                ("coll_table", ctypes.c_int)]


class loc_radiation_buffers_t(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_lines", ctypes.c_int),
                ("acc", _vp), ("acc_c", _vp), ("norm", _vp), ("norm_c", _vp),
                ("acc64", _vp), ("norm64", _vp)]


class loc_server_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("iters_per_launch", ctypes.c_int), ("window_sigmas", ctypes.c_double),
                ("device", ctypes.c_int), ("max_queue", ctypes.c_int)]


class loc_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int),
                ("iterations", ctypes.c_int), ("max_rel_dtex", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("n_cells", ctypes.c_int64),
                ("n_levels", ctypes.c_int), ("updates", ctypes.c_double)]


class loc_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("active", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("device_bytes_in_use", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("models_per_s", ctypes.c_double)]


class LocError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"[{status}] {msg}")
        self.status = status


_lib = None

# every symbol include/loc.h declares
EXPORTS = ["loc_last_error", "loc_version", "loc_create_model", "loc_set_molecule",
           "loc_iterate", "loc_march", "loc_get_radiation", "loc_get_populations",
           "loc_set_populations", "loc_get_tex", "loc_spectra", "loc_model_info",
           "loc_trace_ray", "loc_sync", "loc_destroy", "loc_reset_populations",
           "loc_radiation1d_noalloc", "loc_autotune", "loc_server_create",
           "loc_server_submit", "loc_server_poll", "loc_server_stats", "loc_server_destroy",
           "loc_trace_octree", "loc_octree_path_sums", "loc_map3d", "loc_check_recip",
           "loc_radiation_buffers", "loc_solve"]


def library_path():
    return _build.LIB


def load():
    """Load libloc_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} missing "
                          "(run paper_2009_12609_gb300.build.build())")
    lib = ctypes.CDLL(path)
    lib.loc_last_error.restype = ctypes.c_char_p
    lib.loc_version.restype = ctypes.c_char_p
    lib.loc_create_model.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(loc_model_desc)]
    lib.loc_set_molecule.argtypes = [_vp, ctypes.POINTER(loc_molecule_desc)]
    lib.loc_iterate.argtypes = [_vp, ctypes.POINTER(loc_iter_opts), ctypes.POINTER(loc_iter_report)]
    lib.loc_march.argtypes = [_vp, ctypes.POINTER(loc_iter_opts)]
    lib.loc_reset_populations.argtypes = [_vp]
    lib.loc_autotune.argtypes = [_vp, ctypes.POINTER(loc_iter_opts), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.loc_get_radiation.argtypes = [_vp, _d, _d, _d, ctypes.c_size_t, ctypes.c_size_t]
    lib.loc_get_populations.argtypes = [_vp, _d, ctypes.c_size_t]
    lib.loc_set_populations.argtypes = [_vp, _d, ctypes.c_size_t]
    lib.loc_get_tex.argtypes = [_vp, ctypes.c_int, _d, ctypes.c_size_t]
    lib.loc_spectra.argtypes = [_vp, ctypes.c_int, _d, ctypes.c_int, _d, ctypes.c_size_t]
    lib.loc_map3d.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, ctypes.c_size_t]
    lib.loc_model_info.argtypes = [_vp, _i64, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), _i64]
    lib.loc_trace_ray.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                  _i64, _i64, ctypes.c_int64, _i64]
    lib.loc_sync.argtypes = [_vp]
    lib.loc_check_recip.argtypes = [_d, _d, ctypes.c_size_t]
    lib.loc_trace_octree.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_int64, _i64]
    lib.loc_octree_path_sums.argtypes = [_vp, ctypes.c_int, _i64, ctypes.c_size_t]
    lib.loc_destroy.argtypes = [_vp]
    lib.loc_destroy.restype = None
    lib.loc_radiation1d_noalloc.argtypes = [
        ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double,
        ctypes.c_double, ctypes.c_int, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]
    lib.loc_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(loc_server_opts)]
    lib.loc_server_submit.argtypes = [_vp, ctypes.POINTER(loc_model_desc),
                                      ctypes.POINTER(loc_molecule_desc),
                                      ctypes.POINTER(loc_iter_opts), ctypes.POINTER(ctypes.c_uint64)]
    lib.loc_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(loc_result),
                                    _d, ctypes.c_size_t]
    lib.loc_server_stats.argtypes = [_vp, ctypes.POINTER(loc_server_counters)]
    lib.loc_server_destroy.argtypes = [_vp]
    lib.loc_server_destroy.restype = None
    _lib = lib
    return lib


def _check(status):
    if status != LOC_OK:
        raise LocError(status, load().loc_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pd(a):
    return None if a is None else a.ctypes.data_as(_d)


def _torch_allocator():
    """loc_allocator backed by PyTorch's caching allocator on the current
    device and stream."""
    import torch
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:           # out of memory -> NULL, the library reports LOC_ENOMEM
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    return loc_allocator(fa, ff, None), (fa, ff)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _Keep:
    """Holds numpy arrays referenced by a C struct until the call returns."""

    def __init__(self):
        self.items = []

    def __call__(self, a):
        self.items.append(a)
        return a


def model_desc(model, keep, stream=None, allocator=None):
    """loc_model_desc from a model dict (see loc_inputs)."""
    d = loc_model_desc()
    geo = model["geometry"]
    for key in ("n_h2", "t_kin", "sigma_turb", "abundance"):
        setattr(d, key, _pd(keep(_f64(model[key]))))
    if geo == "shells1d":
        d.geometry = LOC_SHELLS_1D
        d.n_shells = len(model["radius"])
        d.radius = _pd(keep(_f64(model["radius"])))
        d.n_rays = int(model.get("n_rays", 0) or 0)
        d.ray_power = float(model.get("ray_power", 0.0) or 0.0)
        d.v = _pd(keep(_f64(model["v"])))
    elif geo in ("grid3d", "octree3d"):
        d.geometry = LOC_GRID_3D if geo == "grid3d" else LOC_OCTREE_3D
        d.n_root = int(model["n_root"])
        d.h0 = float(model["h0"])
        dirs = keep(_f64(model["dirs"]))
        d.n_dir = len(dirs)
        d.dirs = _pd(dirs)
        for key in ("vx", "vy", "vz"):
            setattr(d, key, _pd(keep(_f64(model[key]))))
        if geo == "octree3d":
            ref = keep(np.ascontiguousarray(model["refine"], dtype=np.int32))
            d.octree_levels = int(model["levels"])
            d.octree_refine = ref.ctypes.data_as(_i32)
            d.octree_n_cells = len(ref)
            d.octree_paths = int(model.get("octree_paths", 0) or 0)
    else:
        raise ValueError(f"unknown geometry {geo}")
    d.n_ch = int(model["n_ch"])
    d.v_min = float(model["v_min"])
    d.dv = float(model["dv"])
    d.t_bg = float(model["t_bg"])
    d.stream = stream
    d.allocator = ctypes.pointer(allocator) if allocator is not None else None
    return d


def molecule_desc(mol, keep, n_levels=None):
    L = len(mol["g"]) if n_levels is None else int(n_levels)
    m = loc_molecule_desc()
    m.n_levels = L
    m.energy_K = _pd(keep(_f64(mol["energy_K"][:L])))
    m.g = _pd(keep(_f64(mol["g"][:L])))
    m.mass_amu = float(mol["mass_amu"])
    lu = np.asarray(mol["line_u"])
    ll = np.asarray(mol["line_l"])
    sel = (lu < L) & (ll < L)
    m.n_lines = int(sel.sum())
    m.line_u = keep(np.ascontiguousarray(lu[sel], np.int32)).ctypes.data_as(_i32)
    m.line_l = keep(np.ascontiguousarray(ll[sel], np.int32)).ctypes.data_as(_i32)
    m.line_A = _pd(keep(_f64(np.asarray(mol["line_A"])[sel])))
    m.line_nu = _pd(keep(_f64(np.asarray(mol["line_nu"])[sel])))
    cu = np.asarray(mol["coll_u"])
    cl = np.asarray(mol["coll_l"])
    selc = (cu < L) & (cl < L)
    m.n_coll = int(selc.sum())
    m.coll_u = keep(np.ascontiguousarray(cu[selc], np.int32)).ctypes.data_as(_i32)
    m.coll_l = keep(np.ascontiguousarray(cl[selc], np.int32)).ctypes.data_as(_i32)
    m.coll_k = _pd(keep(_f64(np.asarray(mol["coll_k"])[selc])))
    if mol.get("hf_n") is not None:
        # hyperfine components of the kept lines, in line order
        n = np.asarray(mol["hf_n"], np.int64)
        off = np.concatenate([[0], np.cumsum(n)])
        idx = np.concatenate([np.arange(off[t], off[t + 1]) for t in np.flatnonzero(sel)] + [[]])
        idx = idx.astype(np.int64)
        m.hf_n = keep(np.ascontiguousarray(n[sel], np.int32)).ctypes.data_as(_i32)
        m.hf_v = _pd(keep(_f64(np.asarray(mol["hf_v"], np.float64)[idx])))
        m.hf_w = _pd(keep(_f64(np.asarray(mol["hf_w"], np.float64)[idx])))
    return m


def iter_opts(max_iter=1, tol_tex=0.0, ali=True, precision="fp32", lines_per_pass=0,
              window_sigmas=0.0, profile=False, steps_per_chunk=0, level_cutoff=0.0,
              dir_range=(0, 0), sub_iters=0, sub_shells=0):
    prec = {"fp32": LOC_FP32_MARCH, "fp64acc": LOC_FP64_ACC, "fp32plain": LOC_FP32_PLAIN}[precision]
    return loc_iter_opts(int(max_iter), float(tol_tex), int(bool(ali)), prec,
                         int(lines_per_pass), float(window_sigmas), int(bool(profile)),
                         int(steps_per_chunk), float(level_cutoff), int(dir_range[0]),
                         int(dir_range[1]), int(sub_iters), int(sub_shells))


# --------------------------------------------------------------------------
# functions with the C names
# --------------------------------------------------------------------------

def loc_last_error():
    return load().loc_last_error().decode()


def loc_version():
    return load().loc_version().decode()


def loc_create_model(model, stream=None, torch_memory=True):
    """Returns an opaque handle (int).  With torch_memory the device memory
    comes from PyTorch's caching allocator and work goes to its current
    stream; the allocator callbacks are kept alive in the returned Model."""
    lib = load()
    keep = _Keep()
    alloc = None
    if torch_memory:
        alloc, cbs = _torch_allocator()
        keep(cbs)
        if stream is None:
            stream = _current_stream()
    d = model_desc(model, keep, stream=stream, allocator=alloc)
    h = _vp()
    _check(lib.loc_create_model(ctypes.byref(h), ctypes.byref(d)))
    return h.value, keep


def loc_set_molecule(h, mol, n_levels=None):
    keep = _Keep()
    m = molecule_desc(mol, keep, n_levels)
    _check(load().loc_set_molecule(h, ctypes.byref(m)))


def loc_iterate(h, **opts):
    o = iter_opts(**opts)
    r = loc_iter_report()
    s = load().loc_iterate(h, ctypes.byref(o), ctypes.byref(r))
    if s not in (LOC_OK, LOC_ENOTCONV):
        _check(s)
    return dict(status=s, iterations=r.iterations, max_rel_dtex=r.max_rel_dtex,
                segments=r.segments, updates=r.updates, kernel_ms=r.kernel_ms,
                n_maser_cells=r.n_maser_cells, march_ms=r.march_ms, se_ms=r.se_ms,
                params_ms=r.params_ms, march_launches=r.march_launches,
                computed_updates=r.computed_updates, nominal_updates=r.nominal_updates,
                path_records=r.path_records,
                coll_table=r.coll_table)


def loc_solve(h, **opts):
    o = iter_opts(**opts)
    r = loc_iter_report()
    _check(load().loc_solve(h, ctypes.byref(o), ctypes.byref(r)))
    return dict(iterations=r.iterations, max_rel_dtex=r.max_rel_dtex)


def loc_radiation_buffers(h):
    """Device addresses and element counts of the accumulators:
    {name: (address, n_elements, numpy dtype)}."""
    b = loc_radiation_buffers_t()
    _check(load().loc_radiation_buffers(h, ctypes.byref(b)))
    nlc, nc = 2 * b.n_cells * b.n_lines, b.n_cells
    return {"acc": (b.acc, nlc, np.float32), "acc_c": (b.acc_c, nlc, np.float32),
            "norm": (b.norm, nc, np.float32), "norm_c": (b.norm_c, nc, np.float32),
            "acc64": (b.acc64, nlc, np.float64), "norm64": (b.norm64, nc, np.float64)}


def loc_autotune(h, **opts):
    """Returns (lines per warp, steps per chunk (-1: whole rays), ms)."""
    per = ctypes.c_int()
    chunk = ctypes.c_int()
    ms = ctypes.c_double()
    o = iter_opts(**opts)
    _check(load().loc_autotune(h, ctypes.byref(o), ctypes.byref(per), ctypes.byref(chunk),
                               ctypes.byref(ms)))
    return per.value, chunk.value, ms.value


def loc_reset_populations(h):
    _check(load().loc_reset_populations(h))


def loc_march(h, **opts):
    o = iter_opts(**opts)
    _check(load().loc_march(h, ctypes.byref(o)))


def loc_model_info(h):
    nc = ctypes.c_int64()
    nl = ctypes.c_int()
    nt = ctypes.c_int()
    ns = ctypes.c_int64()
    _check(load().loc_model_info(h, ctypes.byref(nc), ctypes.byref(nl), ctypes.byref(nt),
                                 ctypes.byref(ns)))
    return dict(n_cells=nc.value, n_levels=nl.value, n_lines=nt.value, segments=ns.value)


def loc_get_radiation(h):
    info = loc_model_info(h)
    nc, nt = info["n_cells"], info["n_lines"]
    sij = np.zeros((nt, nc))
    esc = np.zeros((nt, nc))
    norm = np.zeros(nc)
    _check(load().loc_get_radiation(h, _pd(sij), _pd(esc), _pd(norm), sij.size, norm.size))
    return sij, esc, norm


def loc_get_populations(h):
    info = loc_model_info(h)
    x = np.zeros((info["n_cells"], info["n_levels"]))
    _check(load().loc_get_populations(h, _pd(x), x.size))
    return x


def loc_set_populations(h, x):
    x = _f64(x)
    _check(load().loc_set_populations(h, _pd(x), x.size))


def loc_get_tex(h, t):
    info = loc_model_info(h)
    out = np.zeros(info["n_cells"])
    _check(load().loc_get_tex(h, int(t), _pd(out), out.size))
    return out


def loc_spectra(h, t, p_cm, n_ch):
    p = _f64(np.atleast_1d(p_cm))
    out = np.zeros((len(p), int(n_ch)))
    _check(load().loc_spectra(h, int(t), _pd(p), len(p), _pd(out), out.size))
    return out


def loc_map3d(h, t, d, level, n_pix_side, n_ch):
    """T_RJ [M * M][n_ch] map of line t along direction d, M = n_pix_side."""
    out = np.zeros((int(n_pix_side) ** 2, int(n_ch)))
    _check(load().loc_map3d(h, int(t), int(d), int(level), _pd(out), out.size))
    return out


def loc_check_recip(d):
    """The solve's reciprocal of every element of d, evaluated on the device."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    r = np.empty_like(d)
    _check(load().loc_check_recip(d.ctypes.data_as(_d), r.ctypes.data_as(_d), d.size))
    return r


def loc_trace_ray(h, d, i, j, cap=1 << 16):
    cells = np.zeros(cap, np.int64)
    dz = np.zeros(cap, np.int64)
    n = ctypes.c_int64()
    _check(load().loc_trace_ray(h, int(d), int(i), int(j), cells.ctypes.data_as(_i64),
                                dz.ctypes.data_as(_i64), cap, ctypes.byref(n)))
    return cells[:n.value].copy(), dz[:n.value].copy()


def loc_radiation1d_noalloc(n_shells, n_rays, radius, v_rad, inv_s2sig, n_ch, v_min, dv,
                            n_lines, ks, nbg, window_sigmas, j_ext, beta, stream=None):
    """Allocation-free 1D radiation field; every array argument is a device
    pointer (int) owned by the caller.  Raises LocError on a bad argument."""
    _check(load().loc_radiation1d_noalloc(
        int(n_shells), int(n_rays), radius, v_rad, inv_s2sig, int(n_ch), float(v_min),
        float(dv), int(n_lines), ks, nbg, float(window_sigmas), j_ext, beta, stream))


def loc_trace_octree(h, d, cap=1 << 22):
    out = np.zeros((cap, 7), np.int64)
    n = ctypes.c_int64()
    _check(load().loc_trace_octree(h, int(d), out.ctypes.data_as(_i64), cap, ctypes.byref(n)))
    return out[:min(n.value, cap)].copy()


def loc_octree_path_sums(h, d):
    info = loc_model_info(h)
    out = np.zeros(info["n_cells"], np.int64)
    _check(load().loc_octree_path_sums(h, int(d), out.ctypes.data_as(_i64), out.size))
    return out


def loc_sync(h):
    _check(load().loc_sync(h))


def loc_destroy(h):
    load().loc_destroy(h)


class Model:
    """Owning wrapper: one model handle with its molecule."""

    def __init__(self, model, mol=None, n_levels=None, stream=None, torch_memory=True):
        self.model = model
        self.h, self._keep = loc_create_model(model, stream=stream, torch_memory=torch_memory)
        if mol is not None:
            self.set_molecule(mol, n_levels)

    def set_molecule(self, mol, n_levels=None):
        loc_set_molecule(self.h, mol, n_levels)

    def iterate(self, **opts):
        return loc_iterate(self.h, **opts)

    def reset(self):
        loc_reset_populations(self.h)

    def autotune(self, **opts):
        return loc_autotune(self.h, **opts)

    def march(self, **opts):
        loc_march(self.h, **opts)

    def solve(self, **opts):
        return loc_solve(self.h, **opts)

    def n_dir(self):
        """Directions of the model's table (1 for 1D models)."""
        return len(self.model["dirs"]) if "dirs" in self.model else 1

    def radiation_buffers(self):
        return loc_radiation_buffers(self.h)

    def radiation(self):
        return loc_get_radiation(self.h)

    def populations(self):
        return loc_get_populations(self.h)

    def set_populations(self, x):
        loc_set_populations(self.h, x)

    def tex(self, t):
        return loc_get_tex(self.h, t)

    def spectra(self, t, p_cm):
        return loc_spectra(self.h, t, p_cm, self.model["n_ch"])

    def map3d(self, t, d, level=0):
        """Emergent map of line t along direction d of the model's table:
        T_RJ [M * M][n_ch], M = n_root << level, pixel (i, j) at i * M + j."""
        return loc_map3d(self.h, t, d, level, int(self.model["n_root"]) << int(level),
                         self.model["n_ch"])

    def info(self):
        return loc_model_info(self.h)

    def trace_ray(self, d, i, j, cap=1 << 16):
        return loc_trace_ray(self.h, d, i, j, cap)

    def trace_octree(self, d, cap=1 << 22):
        return loc_trace_octree(self.h, d, cap)

    def octree_path_sums(self, d):
        return loc_octree_path_sums(self.h, d)

    def sync(self):
        loc_sync(self.h)

    def close(self):
        if self.h:
            loc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------------------
# continuous-batching server
# --------------------------------------------------------------------------

def loc_server_create(max_slots=256, mem_budget_bytes=16 << 30, iters_per_launch=4,
                      window_sigmas=8.0, device=0, max_queue=0):
    o = loc_server_opts(int(max_slots), int(mem_budget_bytes), int(iters_per_launch),
                        float(window_sigmas), int(device), int(max_queue))
    h = _vp()
    _check(load().loc_server_create(ctypes.byref(h), ctypes.byref(o)))
    return h.value


def loc_server_submit(h, model, mol, n_levels=None, **opts):
    keep = _Keep()
    d = model_desc(model, keep)
    m = molecule_desc(mol, keep, n_levels)
    o = iter_opts(**opts)
    t = ctypes.c_uint64()
    _check(load().loc_server_submit(h, ctypes.byref(d), ctypes.byref(m), ctypes.byref(o),
                                    ctypes.byref(t)))
    return t.value


def loc_server_poll(h, ticket, n_cells, n_levels, timeout_ms=60000):
    r = loc_result()
    x = np.zeros((int(n_cells), int(n_levels)))
    _check(load().loc_server_poll(h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r),
                                  _pd(x), x.size))
    res = dict(ticket=r.ticket, status=r.status, iterations=r.iterations,
               max_rel_dtex=r.max_rel_dtex, latency_ms=r.latency_ms, n_cells=r.n_cells,
               n_levels=r.n_levels, updates=r.updates)
    return res, x


def loc_server_stats(h):
    c = loc_server_counters()
    s = load().loc_server_stats(h, ctypes.byref(c))
    return dict(status=s, submitted=c.submitted, completed=c.completed, active=c.active,
                queued=c.queued, device_bytes_in_use=c.device_bytes_in_use, p50_ms=c.p50_ms,
                p99_ms=c.p99_ms, mean_ms=c.mean_ms, models_per_s=c.models_per_s)


def loc_server_destroy(h):
    load().loc_server_destroy(h)


class Server:
    """Owning wrapper of a loc_server; remembers each ticket's result shape."""

    def __init__(self, **opts):
        self.h = loc_server_create(**opts)
        self.shape = {}

    def submit(self, model, mol, n_levels=None, **opts):
        t = loc_server_submit(self.h, model, mol, n_levels, **opts)
        L = len(mol["g"]) if n_levels is None else int(n_levels)
        self.shape[t] = (len(model["radius"]), L)
        return t

    def poll(self, ticket, timeout_ms=60000):
        K, L = self.shape[ticket]
        out = loc_server_poll(self.h, ticket, K, L, timeout_ms)
        self.shape.pop(ticket, None)
        return out

    def stats(self):
        return loc_server_stats(self.h)

    def close(self):
        if self.h:
            loc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
