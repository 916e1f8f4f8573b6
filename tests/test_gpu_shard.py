"""Direction sharding of a 3D ALI iteration on the device (Sect. 2.2: the
directions of one radiation-field simulation are independent).

One GPU stands in for two ranks: the two direction shares are marched one
after the other into the same model, the first share's accumulators (seen
through loc_radiation_buffers) are added to the second's, and loc_solve
finishes the iteration -- what an all-reduce between two devices does.  The
summed accumulators must equal one march over all directions to the 2e-5 of
the other one-simulation tests (FP32 sums in another order), and sharded
iterations the plain ones (populations 2e-5).  Regular grid and octree
(replayed paths, whose families are skipped outside the share).
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


MODELS = {
    "grid": lambda: LI.small_grid3d(N=8, n_ch=40, nside=2),
    "octree": lambda: LI.small_octree(N=6, levels=2, refine_frac=0.3, nside=2, n_ch=32, abundance=3e-5),
}


def _two_rank_march(m, opts):
    from paper_2009_12609_gb300 import shard
    n_dir = m.n_dir()
    bufs = shard.accumulator_tensors(m, opts.get("precision", "fp32"))
    m.march(dir_range=shard.direction_range(n_dir, 0, 2), **opts)
    first = [b.clone() for b in bufs]
    m.march(dir_range=shard.direction_range(n_dir, 1, 2), **opts)
    for b, f in zip(bufs, first):
        b += f


@pytest.mark.parametrize("precision", ["fp32", "fp64acc"])
@pytest.mark.parametrize("kind", sorted(MODELS))
def test_direction_shares_sum_to_the_full_march(loc, kind, precision):
    mol = LI.rotor_molecule(n_levels=6)
    model = MODELS[kind]()
    opts = dict(window_sigmas=8.0, precision=precision)
    with loc.Model(model, mol) as m:
        assert m.n_dir() == 48
        m.march(**opts)
        full = m.radiation()
        _two_rank_march(m, opts)
        summed = m.radiation()
    for a, b in zip(summed, full):
        np.testing.assert_allclose(a, b, rtol=2e-5, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("kind", sorted(MODELS))
def test_sharded_iterations_equal_plain_iterations(loc, kind):
    mol = LI.rotor_molecule(n_levels=6)
    model = MODELS[kind]()
    opts = dict(window_sigmas=8.0)
    with loc.Model(model, mol) as m:
        m.iterate(max_iter=3, **opts)
        x_ref = m.populations()
    with loc.Model(model, mol) as m:
        for _ in range(3):
            _two_rank_march(m, opts)
            rep = m.solve(**opts)
            assert rep["iterations"] == 1 and rep["max_rel_dtex"] > 0
        x = m.populations()
    np.testing.assert_allclose(x, x_ref, rtol=2e-5, atol=1e-14)


def test_direction_range_is_checked(loc):
    mol = LI.rotor_molecule(n_levels=4)
    with loc.Model(MODELS["grid"](), mol) as m:
        for bad in ((5, 5), (40, 49), (30, 20)):
            with pytest.raises(loc.LocError) as e:
                m.march(dir_range=bad)
            assert e.value.status == loc.LOC_EINVAL
        with pytest.raises(loc.LocError) as e:
            m.solve(precision="fp64acc")                 # before any march: no radiation
        assert e.value.status == loc.LOC_ESTATE
