"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input construction only: nuclear geometries, basis-set
tables, seeded molecular-orbital coefficients, Jastrow parameters and initial
walker positions.  It contains none of the LRDMC arithmetic (no wavefunction
values, ratios, energies, weights or branching), so that the CPU oracle and the
CUDA path can both consume it without sharing any of the method.
"""
from .systems import (System, hydrogen_atom_sto, hydrogen_atom_gauss, hydrogen_atom_pz, h2_sto3g,
                      water_methane, hydrogen_chain, hydrogen_cluster, by_name)
from .walkers import initial_walkers, lattice_walkers

__all__ = ["System", "hydrogen_atom_sto", "hydrogen_atom_gauss", "hydrogen_atom_pz", "h2_sto3g",
           "water_methane", "hydrogen_chain", "hydrogen_cluster", "by_name", "initial_walkers",
           "lattice_walkers"]
