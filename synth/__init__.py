"""Seeded synthetic inputs for the THC-RR-CCSD residual.

This module is shared by the CPU oracle and by the CUDA path's tests and
benchmark.  It draws random numbers and assembles the input arrays only;
it holds none of the coupled-cluster arithmetic.
"""
from .generator import (System, DeviceSystem, make_system, make_device_system,
                        random_amplitudes, CONFIGS, config_system)

__all__ = ["System", "DeviceSystem", "make_system", "make_device_system",
           "random_amplitudes", "CONFIGS", "config_system"]
