"""nlfem on GB300: GPU assembly of 2D nonlocal FEM operators (arXiv 2207.03921).

The compute path is libnlfem.so (hand-written CUDA for sm_103a, C ABI in
include/nlfem.h); this package builds it, binds it with ctypes and exposes
:class:`Mesh`, :func:`assemble` and :class:`System` over torch CUDA tensors.
"""
from .api import BatchPlan, Mesh, System, assemble, assemble_batch, autotune, tune_set  # noqa: F401
from .binding import NlfemError, load, make_params  # noqa: F401
from .build import build as build_library  # noqa: F401
