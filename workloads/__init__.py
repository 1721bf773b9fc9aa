"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds only input generation: mesh node coordinates, element
connectivity, boundary tags and seeded random draws.  It contains none of the
method's arithmetic (no geometry integrals, no basis, no fluxes), so that the
oracle and the CUDA path share nothing but their inputs.
"""
from .meshes import (BC_INTERIOR, BC_WALL, BC_FARFIELD, BC_SYMMETRY, BC_EXACT, MeshDesc,
                     ogrid, box, cubed_sphere_shell, half_mesh, named_config)
from .states import standard_normal_modes
from .requests import SolveRequest, request_stream

__all__ = ["BC_INTERIOR", "BC_WALL", "BC_FARFIELD", "BC_SYMMETRY", "BC_EXACT", "MeshDesc", "ogrid",
           "box", "cubed_sphere_shell", "half_mesh", "named_config", "standard_normal_modes",
           "SolveRequest", "request_stream"]
