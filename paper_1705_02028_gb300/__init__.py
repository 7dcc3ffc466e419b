"""GB300-native residual-distribution solver for the 2-D Euler equations.

Implements one explicit time step of the multidimensional upwind
(residual-distribution) method of Paardekooper (2017) on triangular meshes --
N, LDA and blended B schemes, forward-Euler and two-stage updates -- as
hand-written CUDA kernels for sm_103a behind the C ABI of ``include/rd.h``.

Modules:
  inputs   seeded synthetic meshes and initial states
  binding  ctypes marshalling of the C ABI (Mesh, State, Batch)
  build    in-tree nvcc build of ``_lib/librd.so``
"""
from . import inputs  # noqa: F401
from .binding import Batch, Mesh, State, RDError, load  # noqa: F401

__all__ = ["inputs", "Mesh", "State", "Batch", "RDError", "load"]
