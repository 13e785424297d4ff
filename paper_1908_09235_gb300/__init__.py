"""GB300 (sm_103a) two-phase lattice Boltzmann step with curved-wall schemes.

The compute path is the CUDA library built from ``csrc/`` (C ABI: include/lbm_gb300.h); the
Python module ``lbm`` is its ctypes binding (it loads the library on first use and never falls
back to the CPU).  Method: Yu, Li & Wen, "Modified curved boundary scheme for two-phase lattice
Boltzmann simulations", arXiv:1908.09235.
"""
from . import lbm, workloads  # noqa: F401

__all__ = ["workloads", "lbm"]
