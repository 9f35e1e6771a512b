"""Seeded synthetic workloads shared by the CUDA path and the oracle.

This package only draws inputs: triangle meshes, per-triangle emission and
radiance-cache values, surface query points, pinhole cameras and per-point
material parameters, and captured-pixel radiance for emitter extraction.  It holds none of the method's arithmetic (no sampling,
no ray casting, no shading), so both sides of every parity test can consume
identical bytes without sharing any computation.
"""
from .scenes import (Mesh, cornell_box, procedural_room, building_floor, shading_tables,
                     surface_queries, pinhole_views, material_params, emitter_pixels)

__all__ = ["Mesh", "cornell_box", "procedural_room", "building_floor", "shading_tables",
           "surface_queries", "pinhole_views", "material_params", "emitter_pixels"]
