"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This package builds meshes (vertices, hex connectivity, boundary faces), the
velocity-grid description, gas parameters, boundary-condition data and initial
macroparameters.  It holds none of the method's arithmetic: no geometry, no
moments, no Maxwellians, no fluxes.  Every array it returns is plain numpy.
"""
from .meshes import (  # noqa: F401
    BC_FREESTREAM, BC_ZEROGRAD, BC_SYMMETRY, BC_WALL, BC_NAMES, LOCAL_FACES,
    Workload, lattice_hex_mesh, sod_row, cavity, obstacle, specular_box,
    closed_freestream_box, channel, cylinder, cylinder_staircase, uniform_random_tucker_ranks,
)
