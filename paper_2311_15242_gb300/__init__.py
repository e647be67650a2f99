"""GB300-native hybrid lattice Boltzmann / finite-difference solver for
two-phase flow with soluble surfactants (arXiv 2311.15242).

The coupled time step runs in hand-written CUDA kernels for sm_103a behind
the C ABI of ``include/lbs.h``; :mod:`.lbs` is its Python binding.
"""
from .lbs import Batch, Mlp, Solver, LbsError, load, library_path  # noqa: F401
