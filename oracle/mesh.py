"""Mesh connectivity and element geometry of a polygonal mesh (FP64).

Follows Sec. 3: T_h a mesh of disjoint polygons K with diameter h_K; faces are
split into interior faces F_h^I (shared by two elements) and boundary faces
F_h^N (homogeneous Neumann, contributing nothing to the forms).  An interior
face is an edge whose two vertex ids appear, in opposite orientation, in two
cells' CCW loops.  Face orientation: K+ is the lower cell id, and the unit
normal n points out of K+.

Pins (tests/test_oracle_mesh.py): face counts against Euler's formula for
the Cartesian mesh (2n(n-1) interior faces), areas summing to |Omega| = 1,
Cartesian diameters sqrt(2)/n, and outward normals summing (weighted by
length) to zero for every closed element.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Geometry:
    area: np.ndarray        # [nc]
    diameter: np.ndarray    # [nc] h_K = max vertex-vertex distance
    bbox: np.ndarray        # [nc, 4] (x0, x1, y0, y1)


@dataclass
class Faces:
    plus: np.ndarray        # [nf] K+ (lower id)
    minus: np.ndarray       # [nf] K-
    va: np.ndarray          # [nf] first vertex (in K+'s CCW order)
    vb: np.ndarray          # [nf] second vertex
    normal: np.ndarray      # [nf, 2] unit normal out of K+
    length: np.ndarray      # [nf]


def cell_polygon(mesh, k):
    return mesh.vertices[mesh.cell(k)]


def geometry(mesh) -> Geometry:
    nc = mesh.n_cells
    area = np.empty(nc)
    diam = np.empty(nc)
    bbox = np.empty((nc, 4))
    for k in range(nc):
        P = cell_polygon(mesh, k)
        Q = np.roll(P, -1, axis=0)
        area[k] = 0.5 * np.sum(P[:, 0] * Q[:, 1] - Q[:, 0] * P[:, 1])
        d = P[:, None, :] - P[None, :, :]
        diam[k] = np.sqrt((d ** 2).sum(-1)).max()
        bbox[k] = (P[:, 0].min(), P[:, 0].max(), P[:, 1].min(), P[:, 1].max())
    return Geometry(area, diam, bbox)


def interior_faces(mesh) -> Faces:
    """Interior edges matched by their sorted vertex-id pair, ordered by (K+, K-, va)."""
    owner = {}
    found = []
    for k in range(mesh.n_cells):
        c = mesh.cell(k)
        for a, b in zip(c, np.roll(c, -1)):
            key = (min(a, b), max(a, b))
            if key in owner:
                k0, a0, b0 = owner.pop(key)
                # K+ = lower id = k0 (cells visited in increasing order)
                found.append((k0, k, a0, b0))
            else:
                owner[key] = (k, int(a), int(b))
    found.sort()
    plus = np.array([f[0] for f in found], dtype=np.int64)
    minus = np.array([f[1] for f in found], dtype=np.int64)
    va = np.array([f[2] for f in found], dtype=np.int64)
    vb = np.array([f[3] for f in found], dtype=np.int64)
    e = mesh.vertices[vb] - mesh.vertices[va]
    length = np.sqrt((e ** 2).sum(1))
    # CCW loop of K+: outward normal of edge a->b is (dy, -dx)/|e|
    normal = np.stack([e[:, 1], -e[:, 0]], 1) / length[:, None]
    return Faces(plus, minus, va, vb, normal, length)
