"""Seeded synthetic inputs for the overlapping-fragments H/S assembly.

This package only generates inputs (grid, Gaussian-well potential, fragment
boxes, seeded random fragment states).  It holds none of the method's
arithmetic, so both the CPU oracle and the CUDA path may use it.
"""
from .geometry import (  # noqa: F401
    Grid, Fragment, Workload, WindowRule, gaussian_potential, make_workload,
    WORKLOADS, small_workload, random_states, fragment_atoms, tiny_fragments_of, lattice_workload,
)
