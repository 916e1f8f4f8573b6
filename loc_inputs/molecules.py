"""Synthetic molecule descriptions (level energies, statistical weights,
radiative lines, collision coefficients).

The paper reads molecular data from LAMDA files; none are available here, so
two synthetic species stand in: a two-level molecule with an HCO+-like
89.19 GHz line and a linear rigid rotor with CO-like constants.  The numbers
are *inputs* of the radiative-transfer method, not part of it.

A molecule is a dict of numpy arrays:
  energy_K[L]   level energy / k_B in kelvin
  g[L]          statistical weight
  mass_amu      molecular mass (thermal line width)
  line_u[T], line_l[T]   upper / lower level index of each radiative line
  line_A[T]     Einstein A_ul [1/s]
  line_nu[T]    rest frequency [Hz]
  coll_u[P], coll_l[P]   collisional pairs (u > l), partner H2
  coll_k[P]     downward rate coefficient k_ul [cm^3/s] (temperature independent)
"""
import numpy as np

# CGS constants used only to tabulate the synthetic molecular data.
_H = 6.62607015e-27
_K = 1.380649e-16
_C = 2.99792458e10
_DEBYE = 1.0e-18


def two_level_molecule(nu=89.19e9, A=4.2e-5, g_u=3.0, g_l=1.0, k_ul=2.0e-10,
                       mass_amu=29.0):
    """Two-level molecule of the 1D test cloud: one line at `nu` with
    Einstein coefficient `A`, weights g_u/g_l and a constant H2 collision
    coefficient k_ul."""
    return dict(
        name="two-level",
        energy_K=np.array([0.0, _H * nu / _K]),
        g=np.array([g_l, g_u], dtype=np.float64),
        mass_amu=float(mass_amu),
        line_u=np.array([1], dtype=np.int32),
        line_l=np.array([0], dtype=np.int32),
        line_A=np.array([A], dtype=np.float64),
        line_nu=np.array([nu], dtype=np.float64),
        coll_u=np.array([1], dtype=np.int32),
        coll_l=np.array([0], dtype=np.int32),
        coll_k=np.array([k_ul], dtype=np.float64),
    )


def rotor_molecule(n_levels=12, B_hz=57.6e9, mu_debye=0.11, mass_amu=28.0,
                   k0=1.0e-10, k_exp=-1.2):
    """Linear rigid rotor truncated at `n_levels` levels J=0..n_levels-1.

    E_J = h B J(J+1), g_J = 2J+1, lines J -> J-1 at nu_J = 2 B J with the
    textbook dipole emission coefficient
        A_J = 64 pi^4 nu^3 mu^2 / (3 h c^3) * J / (2J+1)   (cgs),
    and collisions between every pair u > l with
        k_ul = k0 * (J_u - J_l)^k_exp  [cm^3/s].
    """
    J = np.arange(n_levels, dtype=np.float64)
    energy = _H * B_hz * J * (J + 1.0) / _K
    g = 2.0 * J + 1.0
    Ju = np.arange(1, n_levels)
    nu = 2.0 * B_hz * Ju
    mu = mu_debye * _DEBYE
    A = 64.0 * np.pi ** 4 * nu ** 3 * mu ** 2 / (3.0 * _H * _C ** 3) * Ju / (2.0 * Ju + 1.0)
    cu, cl = [], []
    for u in range(1, n_levels):
        for l in range(u):
            cu.append(u)
            cl.append(l)
    cu = np.array(cu, dtype=np.int32)
    cl = np.array(cl, dtype=np.int32)
    ck = k0 * (cu - cl).astype(np.float64) ** k_exp
    return dict(
        name=f"rotor{n_levels}",
        energy_K=energy,
        g=g,
        mass_amu=float(mass_amu),
        line_u=Ju.astype(np.int32),
        line_l=(Ju - 1).astype(np.int32),
        line_A=A,
        line_nu=nu,
        coll_u=cu,
        coll_l=cl,
        coll_k=ck,
    )


def with_hyperfine(mol, line=0, offsets_kms=(-1.1, 0.0, 0.7), strengths=(0.2, 0.5, 0.3)):
    """The molecule with hyperfine structure on one line: components at
    velocity offsets (km/s) with relative strengths (normalised to sum 1),
    LTE among them; the other lines keep the plain profile.  Synthetic
    values (the paper's examples use NH3 and HCN data, not available here).
    Adds hf_n[T] (components per line, 0 = plain), hf_v (cm/s) and hf_w,
    concatenated in line order."""
    T = len(mol["line_nu"])
    w = np.asarray(strengths, dtype=np.float64)
    out = dict(mol)
    n = np.zeros(T, dtype=np.int32)
    n[line] = len(offsets_kms)
    out["hf_n"] = n
    out["hf_v"] = np.asarray(offsets_kms, dtype=np.float64) * 1.0e5
    out["hf_w"] = w / w.sum()
    out["name"] = mol["name"] + "+hf"
    return out
