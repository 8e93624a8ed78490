"""B300-native coupled flood-pedestrian simulation step (arXiv 1908.05232).

The computation lives in ``libfloodped.so`` (CUDA for sm_103a, C ABI in
``include/floodped.h``); this package only builds and binds it.
"""
from . import build
from ._native import (Batch, FloodPedError, FpConfig, Surrogate, PED_DTYPE, Simulation, TICKS, config_for, from_scenario,
                      ped_records, lib)

__all__ = ["Batch", "Surrogate", "build", "FloodPedError", "FpConfig", "PED_DTYPE", "Simulation", "TICKS", "config_for",
           "from_scenario", "ped_records", "lib"]
