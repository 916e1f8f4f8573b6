"""The allocation-free entry point loc_radiation1d_noalloc.

It serves callers that cannot call cudaMalloc -- an application whose device
memory belongs to another allocator, or a latency-critical loop in which an
allocation would synchronise the device.  They pass their own device buffers
and the library keeps its intermediates in one fixed device array.

The tests call it through the C ABI and compare J_ext = SIJ / NORM and
beta = ESC / NORM with the allocating path (loc_create_model + loc_march +
loc_get_radiation) on the same cloud, within the 2e-5 relative tolerance of
the other one-simulation parity tests (FP32 march, atomic summation order):
  * the same call twice in a row (the fixed array keeps the first call's
    contents, so the second call checks that stale data is cleared);
  * the documented maxima (256 shells or 256 rays, 1024 channels, a
    32-level molecule's 31 lines) with n_rays != n_shells, where the layout
    comes closest to the array's size;
  * a large call followed by a small one, so that leftover ray offsets,
    steps or accumulators of the larger model would show in the smaller;
and that a size beyond the array's limit is refused.  The file is named to
be collected last.
"""
import numpy as np
import pytest

import loc_inputs as LI

pytestmark = pytest.mark.gpu

H = 6.62607015e-27
KB = 1.380649e-16
AMU = 1.66053906660e-24
WINDOW = 8.0


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_12609_gb300 import build, loc
    build.build()
    loc.load()
    return torch, loc


def _case(env, oracle, K, n_rays, n_levels, n_ch):
    """Reference J_ext and beta from the allocating path, and the caller's
    device buffers for the same inputs."""
    torch, loc = env
    mol = LI.rotor_molecule(n_levels=n_levels)
    model = LI.cloud1d_rotor(K=K, n_ch=n_ch, n_rays=n_rays)
    T = len(mol["line_nu"])
    with loc.Model(model, mol) as m:             # populations start at LTE
        m.march(window_sigmas=WINDOW)
        sij, esc, norm = m.radiation()
    ref = ((sij / norm).T, (esc / norm).T)       # [shell][line]
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    ks = np.ascontiguousarray(np.stack([Kp.T, S.T], axis=-1), dtype=np.float32)
    sigma = np.sqrt(model["sigma_turb"] ** 2 + KB * model["t_kin"] / (mol["mass_amu"] * AMU))
    inv = (1.0 / (np.sqrt(2.0) * sigma)).astype(np.float32)
    nbg = (1.0 / np.expm1(H * mol["line_nu"] / (KB * model["t_bg"]))).astype(np.float32)
    dev = torch.device("cuda")
    bufs = dict(radius=torch.tensor(model["radius"], dtype=torch.float64, device=dev),
                v=torch.tensor(model["v"], dtype=torch.float32, device=dev),
                inv=torch.tensor(inv, device=dev), ks=torch.tensor(ks, device=dev),
                nbg=torch.tensor(nbg, device=dev),
                j=torch.empty((K, T), dtype=torch.float32, device=dev),
                b=torch.empty((K, T), dtype=torch.float32, device=dev))
    return dict(K=K, n_rays=n_rays, T=T, model=model, ref=ref, bufs=bufs)


def _call(env, c):
    torch, loc = env
    b, model = c["bufs"], c["model"]
    b["j"].fill_(float("nan"))
    b["b"].fill_(float("nan"))
    loc.loc_radiation1d_noalloc(c["K"], c["n_rays"], b["radius"].data_ptr(), b["v"].data_ptr(),
                                b["inv"].data_ptr(), model["n_ch"], model["v_min"], model["dv"],
                                c["T"], b["ks"].data_ptr(), b["nbg"].data_ptr(), WINDOW,
                                b["j"].data_ptr(), b["b"].data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def _check(c):
    np.testing.assert_allclose(c["bufs"]["j"].cpu().numpy(), c["ref"][0], rtol=2e-5)
    np.testing.assert_allclose(c["bufs"]["b"].cpu().numpy(), c["ref"][1], rtol=2e-5)


def test_noalloc_matches_allocating_path(env, oracle):
    c = _case(env, oracle, K=96, n_rays=0, n_levels=9, n_ch=128)
    for _ in range(2):
        _call(env, c)
        _check(c)
    torch, loc = env
    b = c["bufs"]
    with pytest.raises(loc.LocError) as e:
        loc.loc_radiation1d_noalloc(300, 0, b["radius"].data_ptr(), b["v"].data_ptr(),
                                    b["inv"].data_ptr(), c["model"]["n_ch"], c["model"]["v_min"],
                                    c["model"]["dv"], c["T"], b["ks"].data_ptr(), b["nbg"].data_ptr(),
                                    WINDOW, b["j"].data_ptr(), b["b"].data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == loc.LOC_EINVAL and "256" in str(e.value)


@pytest.mark.parametrize("K,n_rays", [(256, 240), (180, 256)])
def test_noalloc_at_the_documented_maxima(env, oracle, K, n_rays):
    c = _case(env, oracle, K=K, n_rays=n_rays, n_levels=32, n_ch=1024)
    _call(env, c)
    _check(c)


def test_noalloc_large_call_then_small_call(env, oracle):
    big = _case(env, oracle, K=256, n_rays=256, n_levels=20, n_ch=512)
    small = _case(env, oracle, K=40, n_rays=33, n_levels=6, n_ch=96)
    _call(env, big)
    _check(big)
    _call(env, small)
    _check(small)
    _call(env, big)
    _check(big)
