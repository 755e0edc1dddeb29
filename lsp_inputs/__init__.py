"""Seeded synthetic potentials shaped like the paper's workloads.

This module is shared by the oracle and by the GPU path's tests and benchmark. It holds only
input construction (grids, velocity fields, potentials, right-hand sides); none of the
preconditioner's arithmetic lives here.
"""

from .potentials import (  # noqa: F401
    WORKLOADS,
    gaussian_source,
    grid_coords,
    helmholtz_gaussian_bump,
    helmholtz_random_bumps,
    make_workload,
    periodic_sqdist,
    schrodinger_random_wells,
)
