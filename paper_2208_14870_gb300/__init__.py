"""GB300-native (sm_103a) lattice Boltzmann solver for quasi-static linear
elasticity on doubly periodic 2D lattices (Boolakee, Geier, De Lorenzis,
arXiv 2208.14870).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); this package only marshals arguments to it.
"""
from .lbm import *  # noqa: F401,F403
from .lbm import Lattice, LBMError, declared_functions, lib, library_path  # noqa: F401

__version__ = "0.1.0"
