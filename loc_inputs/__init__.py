"""Seeded synthetic inputs for the LOC line-transfer hot path.

This package only *describes* clouds, molecules and ray-direction sets as
plain numpy arrays.  It holds none of the method's arithmetic (no profiles,
no path lengths, no optical depths, no rate equations): those live
independently in the CUDA library and in the CPU oracle, which both consume
the dictionaries built here.

All generators take an explicit seed and use numpy's PCG64 bit generator, so
every test, benchmark and oracle run sees byte-identical inputs.
"""
from .molecules import two_level_molecule, rotor_molecule, with_hyperfine
from .models import (cloud1d_two_level, cloud1d_rotor, uniform_sphere,
                     serving_requests, grid3d_cloud, octree_cloud,
                     small_grid3d, small_octree)
from .healpix import healpix_ring_directions

__all__ = [
    "two_level_molecule", "rotor_molecule", "with_hyperfine", "cloud1d_two_level",
    "cloud1d_rotor", "uniform_sphere", "serving_requests", "grid3d_cloud",
    "octree_cloud", "small_grid3d", "small_octree",
    "healpix_ring_directions",
]
