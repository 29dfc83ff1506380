"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package only draws meshes, tags, parameters and random numbers. It holds
none of the method's arithmetic (no assembly, no membrane model, no solver), so
that both sides that consume it stay independent of each other.
"""
from .mesh import StructuredMesh, structured_mesh, box_cells, tag_grid_boxes, snap_boxes  # noqa: F401
from .configs import CONFIGS, make_config, table2, Config  # noqa: F401
