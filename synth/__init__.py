"""Seeded synthetic inputs for the rotor-stator operator (meshes and field values).

This package holds input generation only: structured rotor-stator meshes (node
coordinates at the reference configuration, cell connectivity, side tags, wall
flags and the interface description) and pseudo-random field values drawn with
splitmix64.  It contains none of the discretisation's arithmetic (no basis,
quadrature, geometry derivatives, mortar mapping or operator terms).  Both the
CUDA library's tests/benchmark and the CPU oracle consume these inputs.
"""
from .mesh import RotorStatorMesh, rotor_stator_mesh
from .fields import splitmix64_uniform, random_nodal_field, smooth_nodal_field
from .configs import CONFIGS, make_config

__all__ = ["RotorStatorMesh", "rotor_stator_mesh", "splitmix64_uniform",
           "random_nodal_field", "smooth_nodal_field", "CONFIGS", "make_config"]
