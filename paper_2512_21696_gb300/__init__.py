"""GB300-native two-component pseudo-potential lattice Boltzmann step (D3Q19)
with the multiscale models of arXiv 2512.21696 (CSF surface-tension control,
residual components, tensorial resistivity).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI of
``include/lbm.h``; :mod:`.lbm` is its Python binding and :mod:`.synth` the
seeded synthetic input generators.
"""
from . import synth  # noqa: F401
from .lbm import *  # noqa: F401,F403
