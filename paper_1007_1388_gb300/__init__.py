"""GB300-native D3Q19 lattice Boltzmann hot path (patch/block scheme of Feichtinger et al.).

The compute path is liblbm.so (CUDA for sm_103a, C ABI in include/lbm.h);
``paper_1007_1388_gb300.lbm`` is its ctypes binding, ``workloads`` the seeded
synthetic input generators, ``build`` the in-tree compiler driver.
"""
from . import lbm, unet, warmstart, workloads  # noqa: F401
from .lbm import *  # noqa: F401,F403

__version__ = "0.1.0"
