"""Seeded synthetic inputs shared by the FP64 oracle and the GB300 library tests.

This package produces plain input data only: polygonal meshes (vertex
coordinates and CCW vertex loops), element partitions, per-element
conductivity tensors, stimulus parameters and seeded vectors.  It holds none
of the discretisation's arithmetic (no basis, quadrature, assembly, solver or
ionic model).  Every generator takes an explicit seed and uses numpy's PCG64.
"""
from .meshes import (Mesh, cartesian_square, voronoi_square, block_partition,
                     kmeans_partition, fibre_conductivity, isotropic_conductivity)
from .workloads import (Workload, square16_p2, voronoi4096_p3, random_rhs,
                        stimulus_params, make_workload, voronoi_batch)

__all__ = ["Mesh", "cartesian_square", "voronoi_square", "block_partition",
           "kmeans_partition", "fibre_conductivity", "isotropic_conductivity", "Workload", "square16_p2", "voronoi4096_p3",
           "random_rhs", "stimulus_params", "make_workload"]
