"""Seeded synthetic inputs (Si and liquid-water finite-range Gaussian bases).

This package holds input generation only; it contains none of the orbital
minimization arithmetic and is shared by the oracle, the tests and the bench.
"""
from .configs import (Problem, config1, config2, config3, config4_instance, config5_base,
                      silicon, water, spectrum_edges, warm_start_delta, TAU_10RY)

__all__ = ["Problem", "config1", "config2", "config3", "config4_instance", "config5_base",
           "silicon", "water", "spectrum_edges", "warm_start_delta", "TAU_10RY"]
