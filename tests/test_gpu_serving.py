"""GPU tests of the continuous-batching server (batched 1D ALI solves).

Each request's result must not depend on what else is in the batch: the
batched kernels run the same per-step and per-cell device routines as the
single-model path, and the only difference is the order of FP32 atomic
additions, so populations agree with a single-model solve of the same
request to 2e-5 relative (same bound as one ray simulation) and with the
FP64 oracle to the usual 1e-4 in T_ex.  Requests submitted while others run
are admitted and overtake long ones; a small memory budget queues requests
without losing any.
"""
import time

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


def _requests(n, seed, k_range=(32, 160)):
    return LI.serving_requests(n=n, seed=seed, k_range=k_range, ch_choices=(64, 128, 256, 512),
                               level_range=(2, 12))


def _single(loc, req, n_iter, window):
    mol = LI.rotor_molecule(n_levels=req["n_levels"])
    with loc.Model(req["model"], mol) as m:
        m.iterate(max_iter=n_iter, window_sigmas=window)
        return m.populations()


def test_batch_matches_single_model_path(loc, oracle):
    reqs = _requests(10, seed=101)
    n_iter, window = 12, 8.0
    with loc.Server(max_slots=16, iters_per_launch=3, window_sigmas=window) as srv:
        tickets = [srv.submit(r["model"], LI.rotor_molecule(n_levels=r["n_levels"]),
                              max_iter=n_iter) for r in reqs]
        results = [srv.poll(t, timeout_ms=120000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["status"] == 0
    for r, (res, x) in zip(reqs, results):
        assert res["iterations"] == n_iter and res["status"] == 0
        np.testing.assert_allclose(x, _single(loc, r, n_iter, window), rtol=2e-5, atol=1e-14)
    # two of them against the oracle (T_ex to 1e-4)
    for r, (res, x) in list(zip(reqs, results))[:2]:
        mol = LI.rotor_molecule(n_levels=r["n_levels"])
        xr, _ = oracle.iterate_1d(mol, r["model"], n_iter)
        tg, tr = oracle.tex(mol, x), oracle.tex(mol, xr)
        sel = xr[:, mol["line_u"][:tr.shape[0]]].T >= 1e-6
        assert np.max(np.abs(tg[sel] / tr[sel] - 1.0)) < 1e-4


def test_batch_level_cutoff_matches_single_model_path(loc, oracle):
    """Per-cell line truncation in the batched server equals the single-model
    path with the same cutoff, and stays within tolerance of the oracle."""
    reqs = _requests(6, seed=404)
    n_iter, window, cut = 10, 8.0, 1e-8
    with loc.Server(max_slots=8, iters_per_launch=2, window_sigmas=window) as srv:
        tickets = [srv.submit(r["model"], LI.rotor_molecule(n_levels=r["n_levels"]),
                              max_iter=n_iter, level_cutoff=cut) for r in reqs]
        results = [srv.poll(t, timeout_ms=120000) for t in tickets]
    for r, (res, x) in zip(reqs, results):
        assert res["status"] == 0
        mol = LI.rotor_molecule(n_levels=r["n_levels"])
        with loc.Model(r["model"], mol) as m:
            m.iterate(max_iter=n_iter, window_sigmas=window, level_cutoff=cut)
            xs = m.populations()
        np.testing.assert_allclose(x, xs, rtol=2e-5, atol=1e-14)
    r, (res, x) = reqs[0], results[0]
    mol = LI.rotor_molecule(n_levels=r["n_levels"])
    xr, _ = oracle.iterate_1d(mol, r["model"], n_iter)
    tg, tr = oracle.tex(mol, x), oracle.tex(mol, xr)
    sel = xr[:, mol["line_u"][:tr.shape[0]]].T >= 1e-6
    assert np.max(np.abs(tg[sel] / tr[sel] - 1.0)) < 1e-4


def test_alone_equals_in_mix(loc):
    reqs = _requests(8, seed=202)
    target = reqs[3]
    mol = LI.rotor_molecule(n_levels=target["n_levels"])
    with loc.Server(max_slots=4, iters_per_launch=2) as srv:
        res_a, x_alone = srv.poll(srv.submit(target["model"], mol, max_iter=15), 60000)
    with loc.Server(max_slots=8, iters_per_launch=2) as srv:
        ts = [srv.submit(r["model"], LI.rotor_molecule(n_levels=r["n_levels"]), max_iter=15)
              for r in reqs]
        out = [srv.poll(t, 120000) for t in ts]
    res_b, x_mix = out[3]
    assert res_a["iterations"] == res_b["iterations"] == 15
    np.testing.assert_allclose(x_mix, x_alone, rtol=2e-5, atol=1e-14)


def test_late_arrival_is_admitted_and_overtakes(loc):
    long_req = _requests(1, seed=303, k_range=(600, 600))[0]
    short_req = _requests(1, seed=304, k_range=(40, 40))[0]
    with loc.Server(max_slots=4, iters_per_launch=1) as srv:
        t_long = srv.submit(long_req["model"], LI.rotor_molecule(n_levels=long_req["n_levels"]),
                            max_iter=400)
        time.sleep(0.05)
        t_short = srv.submit(short_req["model"], LI.rotor_molecule(n_levels=short_req["n_levels"]),
                             max_iter=3)
        r_short, _ = srv.poll(t_short, 60000)
        st = srv.stats()
        assert st["active"] == 1            # the long request is still running
        r_long, _ = srv.poll(t_long, 300000)
    assert r_short["iterations"] == 3 and r_long["iterations"] == 400
    assert r_short["latency_ms"] < r_long["latency_ms"]


def test_convergence_status(loc):
    r = _requests(1, seed=404)[0]
    mol = LI.rotor_molecule(n_levels=r["n_levels"])
    with loc.Server(max_slots=2, iters_per_launch=4) as srv:
        res, _ = srv.poll(srv.submit(r["model"], mol, max_iter=300, tol_tex=1e-4), 120000)
        assert res["status"] == 0 and res["max_rel_dtex"] < 1e-4 and res["iterations"] < 300
        res2, _ = srv.poll(srv.submit(r["model"], mol, max_iter=2, tol_tex=1e-12), 60000)
        assert res2["status"] == loc.LOC_ENOTCONV and res2["iterations"] == 2


def test_memory_budget_queues_without_loss(loc):
    reqs = _requests(12, seed=505)
    with loc.Server(max_slots=64, iters_per_launch=2, mem_budget_bytes=6 << 20) as srv:
        ts = [srv.submit(r["model"], LI.rotor_molecule(n_levels=r["n_levels"]), max_iter=5)
              for r in reqs]
        out = [srv.poll(t, 120000) for t in ts]
        st = srv.stats()
    assert st["completed"] == 12 and all(o[0]["iterations"] == 5 for o in out)
    assert st["device_bytes_in_use"] == 0


def test_server_errors(loc):
    r = _requests(1, seed=606)[0]
    mol = LI.rotor_molecule(n_levels=r["n_levels"])
    with loc.Server(max_slots=2) as srv:
        bad = dict(r["model"])
        bad["radius"] = bad["radius"][::-1].copy()
        with pytest.raises(loc.LocError) as e:
            srv.submit(bad, mol, max_iter=3)
        assert e.value.status == loc.LOC_EINVAL
        t = srv.submit(LI.cloud1d_rotor(K=900, n_ch=512), LI.rotor_molecule(), max_iter=500)
        with pytest.raises(loc.LocError) as e:
            srv.poll(t, timeout_ms=1)
        assert e.value.status == loc.LOC_ETIMEOUT
        with pytest.raises(loc.LocError) as e:
            loc.loc_server_poll(srv.h, 999999, 4, 4, 0)
        assert e.value.status == loc.LOC_EINVAL
    with pytest.raises(loc.LocError):
        loc.Server(max_slots=0)


def test_largest_request_shape_in_a_batch(loc, oracle):
    """The serving stream's largest request shape (1024 shells, 512 channels,
    20 levels / 19 lines) batched with three smaller requests: its
    populations equal the single-model path (2e-5) and its T_ex the FP64
    oracle (1e-4) after 3 iterations."""
    big = dict(model=LI.cloud1d_rotor(K=1024, n_ch=512, seed=77, r_clamp_frac=0.05), n_levels=20)
    reqs = [big] + _requests(3, seed=707)
    n_iter, window = 3, 8.0
    with loc.Server(max_slots=8, iters_per_launch=3, window_sigmas=window) as srv:
        tickets = [srv.submit(r["model"], LI.rotor_molecule(n_levels=r["n_levels"]), max_iter=n_iter)
                   for r in reqs]
        results = [srv.poll(t, timeout_ms=300000) for t in tickets]
    for r, (res, x) in zip(reqs, results):
        assert res["status"] == 0 and res["iterations"] == n_iter
        np.testing.assert_allclose(x, _single(loc, r, n_iter, window), rtol=2e-5, atol=1e-14)
    mol = LI.rotor_molecule(n_levels=20)
    xr, _ = oracle.iterate_1d(mol, big["model"], n_iter)
    x = results[0][1]
    tg, tr = oracle.tex(mol, x), oracle.tex(mol, xr)
    sel = xr[:, mol["line_u"]].T >= 1e-6
    assert np.max(np.abs(tg[sel] / tr[sel] - 1.0)) < 1e-4
