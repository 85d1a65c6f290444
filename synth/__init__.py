"""Seeded synthetic inputs for the L2-projection transfer (Sec. 2.3, "Variational Transfer").

This package is shared by the CPU oracle, the tests and the benchmark. It only
*generates* inputs: solid meshes (P1 triangles / tetrahedra in the current
configuration), grid descriptions and fluid fields sampled at grid nodes. It
contains none of the transfer's arithmetic (no clipping, no quadrature, no
assembly, no solve).
"""
from .meshes import (  # noqa: F401
    Grid, disk_mesh, beam_mesh, leaflet_mesh, deformed_beam_mesh, random_rotation,
    place_body, grid_node_coords, taylor_green, sin_cos_2d, workload, batch_bodies,
    body_motion, combine_bodies, batch_workload, batch_coords, block_face_mask, BEAM_HEXES,
    stretched_axis, stretched_grid,
)
