"""Seeded synthetic inputs: perturbed all-hex meshes of boxes and loads.

This module is shared by the test oracle, the tests and the benchmark. It
holds no arithmetic of the spectral-element method itself: it only draws
vertex coordinates, hex connectivity, permutations, orientations and
right-hand sides from a seeded generator.
"""
from .mesh import (HexMesh, lattice_hex_mesh, split_triangle_hex_mesh, manufactured_u, manufactured_s,
                   gaussian_load, moving_source, PROPER_ROTATIONS, VTK_CORNER_BITS)

__all__ = ["HexMesh", "lattice_hex_mesh", "split_triangle_hex_mesh", "manufactured_u", "manufactured_s",
           "gaussian_load", "moving_source", "PROPER_ROTATIONS", "VTK_CORNER_BITS"]
