"""Seeded synthetic inputs shared by the oracle and the CUDA path (no method arithmetic)."""
from .systems import (SKParams, SK_CARBON_LIKE, SK_FCC_METAL, Workload, WORKLOADS, lattice_positions,
                      workload_positions, sample_atoms, random_symmetric_pair)

__all__ = ["SKParams", "SK_CARBON_LIKE", "SK_FCC_METAL", "Workload", "WORKLOADS", "lattice_positions",
           "workload_positions", "sample_atoms", "random_symmetric_pair"]
