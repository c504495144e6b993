"""GB300-native space-time finite-element heat-conduction solver (arXiv 2508.09589).

The compute path is the native library libst.so (hand-written CUDA for sm_103a behind
the C ABI in include/st.h).  This package only marshals arguments: importing it never
falls back to another implementation, and every call fails loudly if the library is
missing.
"""
from .api import (BDF1, MMA, Mesh, Server, TopOpt, footprint_bytes, mesh_desc, options, plan_hierarchy, solve_adjoint_batch,  # noqa: F401
                  solve_forward_batch, source)
from ._lib import STError, lib  # noqa: F401

__all__ = ["BDF1", "MMA", "Mesh", "Server", "TopOpt", "options", "source", "mesh_desc", "footprint_bytes", "plan_hierarchy", "STError", "lib",
           "solve_forward_batch", "solve_adjoint_batch"]
