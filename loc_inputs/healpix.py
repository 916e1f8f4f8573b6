"""HEALPix RING-scheme pixel centres as unit direction vectors.

The 3D ray directions of the method are taken from a HEALPix pixelisation
(Sect. 2.2 of the paper; pixel-centre formulas of Gorski et al. 2005, ApJ 622,
759, Sect. 4).  N_side = 2 gives the 48 directions used in the paper.  The
table is an input of the ray tracer: both the CUDA library and the oracle
receive it as data.
"""
import numpy as np


def healpix_ring_directions(nside=2):
    """Return the 12 nside^2 pixel centres in RING order as (npix, 3) FP64
    unit vectors (x, y, z)."""
    ns = int(nside)
    z_list, phi_list = [], []
    for i in range(1, 4 * ns):
        if i < ns:                       # north polar cap
            for j in range(1, 4 * i + 1):
                z_list.append(1.0 - i * i / (3.0 * ns * ns))
                phi_list.append(np.pi / (2.0 * i) * (j - 0.5))
        elif i <= 3 * ns:                # equatorial belt
            s = (i - ns + 1) % 2
            for j in range(1, 4 * ns + 1):
                z_list.append(4.0 / 3.0 - 2.0 * i / (3.0 * ns))
                phi_list.append(np.pi / (2.0 * ns) * (j - 0.5 * s))
        else:                            # south polar cap
            ii = 4 * ns - i
            for j in range(1, 4 * ii + 1):
                z_list.append(-(1.0 - ii * ii / (3.0 * ns * ns)))
                phi_list.append(np.pi / (2.0 * ii) * (j - 0.5))
    z = np.array(z_list)
    phi = np.array(phi_list)
    st = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=1)
