"""Quantized-BVH neighbor search (arXiv:1901.08088) for one GB300 GPU.

The CUDA library ``libqbvh.so`` (C ABI in include/qbvh.h) does all the work;
this package is its Python binding plus the autograd wrapper of the fused
Lennard-Jones pass and the batched many-system runner.
"""
from ._lib import QBVHError, LIB_PATH  # noqa: F401
from .qbvh import *  # noqa: F401,F403
from .qbvh import NeighborList  # noqa: F401
from .lj import LJEnergy, lj_energy, pack_positions  # noqa: F401
from .batch import BatchedNeighborList, PerSystemLoop  # noqa: F401
from . import autotune  # noqa: F401
