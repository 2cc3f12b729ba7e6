"""GB300-native short-range molecular dynamics hot path.

Cut-off Lennard-Jones and Finnis-Sinclair EAM forces over cell-binned Verlet
neighbour lists, the list rebuild and velocity-Verlet NVE integration, as
hand-written CUDA for sm_103a behind the C ABI in include/md.h (libmd.so).
After Trott, Winterfeld & Crozier, "General-purpose molecular dynamics
simulations on GPU-based clusters" (LAMMPS_CUDA).
"""
from ._build import build as build_library  # noqa: F401
from ._lib import load as load_library  # noqa: F401
from .system import (EAMForces, LJForces, MDError, System, fp64_math, lj_params, pairs_to_matrix,  # noqa: F401
                     probe_ceilings)

__all__ = ["System", "LJForces", "EAMForces", "MDError", "lj_params", "pairs_to_matrix", "build_library", "load_library",
           "probe_ceilings", "fp64_math"]
