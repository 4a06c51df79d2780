"""Seeded synthetic inputs (Si and liquid-water finite-range Gaussian bases).

This package holds input generation only; it contains none of the orbital
minimization arithmetic and is shared by the oracle, the tests and the bench.
"""
from .configs import (Problem, si64_sz, si512_dzp, water256_dzp, batch_instance, si4096_sz,
                      silicon, water, spectrum_edges, warm_start_delta, TAU_10RY)

__all__ = ["Problem", "si64_sz", "si512_dzp", "water256_dzp", "batch_instance", "si4096_sz",
           "silicon", "water", "spectrum_edges", "warm_start_delta", "TAU_10RY"]
