"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

Nothing here computes any part of the eigensolver; see ``synth.workloads`` for
the named workloads (mesh family, sizes, p, levels, tolerance).
"""
from .meshes import (Mesh, bumpy_patch, bumpy_torus, displaced_geodesic_icosphere, displaced_icosphere,
                     flat_square, flat_torus, geodesic_icosphere, grid_patch_faces, grid_torus_faces, icosphere)
from .workloads import WORKLOADS, Workload, batch, make_workload

__all__ = ["Mesh", "bumpy_patch", "flat_square", "grid_patch_faces", "bumpy_torus", "displaced_geodesic_icosphere", "displaced_icosphere",
           "flat_torus", "geodesic_icosphere", "grid_torus_faces", "icosphere", "WORKLOADS",
           "Workload", "batch", "make_workload"]
