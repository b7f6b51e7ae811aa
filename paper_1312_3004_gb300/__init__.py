"""GB300-native Replica-Exchange Wang-Landau sampling (arXiv:1312.3004) for the
periodic 2D q-state Potts model.

The computation runs in the CUDA library behind include/rewl.h
(paper_1312_3004_gb300/_build/librewl.so, built by build.py); this package
only marshals arguments.
"""
from ._lib import RewlError, load  # noqa: F401
from .rewl import (REWL, Batch, Server, bootstrap, canonical, canonical_distribution,  # noqa: F401
                   equal_peak_temperature, ising_energy, join, measure_pipes, specific_heat_peak)

__all__ = ["REWL", "Batch", "Server", "RewlError", "load", "canonical", "canonical_distribution",
           "specific_heat_peak", "equal_peak_temperature", "join", "bootstrap", "ising_energy", "measure_pipes"]
