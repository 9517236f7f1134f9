"""Seeded, synthetic model Hamiltonians that feed both the CUDA path and the oracle.

This package holds input generation only: one-electron integrals, two-electron
integrals in chemists' notation (pq|rs), reference occupations and the orbital
partitions of the standard workloads. It contains none of the MBE-FCI method's
arithmetic (no CASCI, no effective Hamiltonian, no increments).
"""

from .hamiltonians import (  # noqa: F401
    Workload,
    hubbard_ring_momentum,
    hubbard_ring_pm,
    pipek_mezey,
    pm_functional,
    hubbard_open_dimer,
    synthetic_molecule,
    random_system,
    block_decoupled_system,
    workload,
    WORKLOAD_NAMES,
)
