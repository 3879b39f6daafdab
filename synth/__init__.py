"""Seeded synthetic inputs shared by the FP64 oracle and the GB300 library tests.

This package produces plain input data only: polygonal meshes (vertex
coordinates and CCW vertex loops), polyhedral meshes (outward triangle
facets), element partitions, per-element
conductivity tensors, stimulus parameters and seeded vectors.  It holds none
of the discretisation's arithmetic (no basis, quadrature, assembly, solver or
ionic model).  Every generator takes an explicit seed and uses numpy's PCG64.
"""
from .meshes import (Mesh, PolyMesh3D, cartesian_square, voronoi_square, block_partition,
                     kmeans_partition, fibre_conductivity, isotropic_conductivity,
                     jittered_hex_cube, block_partition_3d)
from .workloads import (Workload, square16_p2, voronoi4096_p3, random_rhs,
                        stimulus_params, make_workload, voronoi_batch, hex_cube_p2)

__all__ = ["Mesh", "PolyMesh3D", "jittered_hex_cube", "block_partition_3d", "hex_cube_p2",
           "voronoi_batch", "cartesian_square", "voronoi_square", "block_partition",
           "kmeans_partition", "fibre_conductivity", "isotropic_conductivity", "Workload", "square16_p2", "voronoi4096_p3",
           "random_rhs", "stimulus_params", "make_workload"]
