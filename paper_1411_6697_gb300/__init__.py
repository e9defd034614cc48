"""GB300 (sm_103a) implementation of the MRT lattice Boltzmann kinetic model for combustion.

The hot path -- the per-cell, per-step update of the 16 discrete distribution
functions and the reaction progress -- runs in hand-written CUDA kernels behind
the C ABI of include/lbkm.h; ``lbkm`` is its Python binding.
"""
from .lbkm import Solver, default_params, load, version, LbkmError  # noqa: F401
