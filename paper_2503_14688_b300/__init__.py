"""paper_2503_14688_b300 -- the checkerboard Metropolis sweep of the 2D Ising
and Blume-Capel models on one B300, behind the C ABI of libisg.

The heavy lifting is in ``libisg.so`` (sm_103a CUDA kernels, C ABI declared in
``include/isg.h``).  This package is a thin binding: ``_abi`` declares the C
prototypes, ``lattice`` marshals numpy arrays and torch streams into them.
PyTorch is used only for device memory and streams.
"""
from ._abi import (ISG_BLUME_CAPEL, ISG_ISING, IsgError, check, lib)  # noqa: F401
from .lattice import Lattice, Obs, measure_planes_noalloc, xi2, xi_integral  # noqa: F401
from .ensemble import Ensemble  # noqa: F401
from .server import Server  # noqa: F401

ISING = ISG_ISING
BLUME_CAPEL = ISG_BLUME_CAPEL
