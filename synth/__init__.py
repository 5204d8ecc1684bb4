"""Seeded synthetic inputs for the two-species PM step.

This package is shared by the CUDA path's tests/benchmark and by the oracle's
tests.  It draws particle positions and velocities only; it holds none of the
PM method's arithmetic (no codec, deposit, solve, interpolation or update).
"""
from .generators import (  # noqa: F401
    WORKLOADS,
    Workload,
    fermi_dirac_speeds,
    isotropic_velocities,
    lattice_positions,
    lognormal_positions,
    make_workload,
    uniform_positions,
    zeldovich_lattice,
)
