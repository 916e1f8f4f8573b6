"""Compensated FP32 accumulation of SIJ / ESC / NORM (Eq. 2: the per-cell
sums over every ray step that crosses a cell) against plain FP32 atomics,
both measured against the FP64 oracle.

Every ray step adds its share into the cell's FP32 accumulators with an
atomic addition.  With compensation (the default) the exact rounding error of
each addition goes into a second FP32 word (TwoSum on the value the atomic
found), and the solve reads the sum of both; without it ('fp32plain') the
rounding errors of up to a few thousand additions per cell pile up.  What
remains with compensation is the FP32 error of the per-step values
themselves (profile, exponential, intensity), which both modes share.

The tests print the largest relative error of each accumulator in both
modes, on workloads where many steps land in one cell (a 1024-shell 1D
cloud: the innermost shell takes 2048 steps), on the octree recipe of the
bench (5 levels, 48 directions) and on one direction of the 128^3 grid (one
or two steps per cell: nothing to compensate).  The bar: the compensated
error stays within the parity tolerance and is never larger than the plain
one by more than the shared per-step noise.
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


def _rel_err(g, r):
    """Largest |g - r| relative to |r|, with values below 1e-6 of the
    largest measured against that floor."""
    floor = 1e-6 * np.abs(r).max()
    return float(np.max(np.abs(g - r) / np.maximum(np.abs(r), floor)))


def _errors(loc, model, mol, ref):
    out = {}
    for prec in ("fp32", "fp32plain"):
        with loc.Model(model, mol) as m:
            m.march(window_sigmas=8.0, precision=prec)
            sij, esc, norm = m.radiation()
        rs, re_, rn = ref
        out[prec] = (_rel_err(sij, rs), _rel_err(esc, re_), _rel_err(norm, rn))
    return out


def _check(name, out, bar):
    for i, acc in enumerate(("SIJ", "ESC", "NORM")):
        c, p = out["fp32"][i], out["fp32plain"][i]
        print(f"compensation {name} {acc}: compensated {c:.3e} plain {p:.3e}")
        assert c < bar, (name, acc, c)
        assert c <= p + 2e-7, (name, acc, c, p)


def test_compensation_1d_1024_shells(loc, oracle):
    mol = LI.rotor_molecule()
    model = LI.cloud1d_rotor(K=1024, n_ch=64)
    x = oracle.lte_populations(mol, model["t_kin"])
    Kp, S = oracle.line_params(mol, model, x)
    ref = oracle.march_1d(mol, model, Kp, S)
    _check("1d_1024_shells", _errors(loc, model, mol, ref), 2e-5)


def test_compensation_octree_bench_recipe(loc, oracle):
    mol = LI.rotor_molecule()
    model = LI.octree_cloud(N=12)
    lm = oracle.leaf_model(model)
    x = oracle.lte_populations(mol, lm["t_kin"])
    Kp, S = oracle.line_params(mol, lm, x)
    ref = oracle.march_octree(mol, model, Kp, S)
    _check("octree_12_root_5_levels", _errors(loc, model, mol, ref), 5e-5)


def test_compensation_grid_128_one_direction(loc, oracle):
    mol = LI.rotor_molecule()
    g = LI.grid3d_cloud()
    g["dirs"] = g["dirs"][:1].copy()
    x = oracle.lte_populations(mol, g["t_kin"])
    Kp, S = oracle.line_params(mol, g, x)
    ref = oracle.march_grid3d(mol, g, Kp, S)
    _check("grid_128_one_direction", _errors(loc, g, mol, ref), 5e-5)
