"""Mesh connectivity and element geometry of polygonal and polyhedral meshes (FP64).

Follows Sec. 3: T_h a mesh of disjoint polytopes K with diameter h_K; faces are
split into interior faces F_h^I (shared by two elements) and boundary faces
F_h^N (homogeneous Neumann, contributing nothing to the forms).  In 2D an
interior face is an edge whose two vertex ids appear, in opposite orientation,
in two cells' CCW loops; in 3D it is a triangle facet whose three vertex ids
appear in two cells' outward facet lists.  Face orientation: K+ is the lower
cell id, and the unit normal n points out of K+.

Pins (tests/test_oracle_mesh.py, tests/test_oracle_3d.py): face counts against
Euler's formula for the Cartesian mesh (2n(n-1) interior faces) and against
the hex grid (2 * 3 n^2 (n-1) interior triangles), measures summing to
|Omega| = 1, Cartesian diameters sqrt(2)/n, and outward normals summing
(weighted by face measure) to zero for every closed element.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Geometry:
    area: np.ndarray        # [nc] area (2D) or volume (3D)
    diameter: np.ndarray    # [nc] h_K = max vertex-vertex distance
    bbox: np.ndarray        # [nc, 2 dim] (x0, x1, y0, y1[, z0, z1])


@dataclass
class Faces:
    plus: np.ndarray        # [nf] K+ (lower id)
    minus: np.ndarray       # [nf] K-
    va: np.ndarray          # [nf] first vertex (in K+'s CCW order)
    vb: np.ndarray          # [nf] second vertex
    normal: np.ndarray      # [nf, dim] unit normal out of K+
    length: np.ndarray      # [nf] length (2D) or area (3D)
    vc: np.ndarray = None   # [nf] third vertex of a 3D triangle face (K+'s orientation)


def cell_polygon(mesh, k):
    return mesh.vertices[mesh.cell(k)]


def geometry(mesh) -> Geometry:
    if mesh.dim == 3:
        return geometry3d(mesh)
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
    if mesh.dim == 3:
        return interior_faces3d(mesh)
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


def geometry3d(mesh) -> Geometry:
    """Volume by the divergence theorem (sum over outward facets of a.(b x c)/6),
    diameter and bounding box of each polyhedron."""
    nc = mesh.n_cells
    vol = np.empty(nc)
    diam = np.empty(nc)
    bbox = np.empty((nc, 6))
    for k in range(nc):
        F = mesh.vertices[mesh.facets(k)]                # [m, 3 vertices, 3]
        vol[k] = np.einsum("fi,fi->", F[:, 0], np.cross(F[:, 1], F[:, 2])) / 6.0
        P = mesh.vertices[mesh.cell(k)]
        d = P[:, None, :] - P[None, :, :]
        diam[k] = np.sqrt((d ** 2).sum(-1)).max()
        lo, hi = P.min(0), P.max(0)
        bbox[k] = (lo[0], hi[0], lo[1], hi[1], lo[2], hi[2])
    return Geometry(vol, diam, bbox)


def interior_faces3d(mesh) -> Faces:
    """Interior triangle facets matched by their sorted vertex-id triple, ordered by
    (K+, K-, va, vb, vc) with (va, vb, vc) in K+'s outward orientation."""
    owner = {}
    found = []
    for k in range(mesh.n_cells):
        for a, b, c in mesh.facets(k):
            key = tuple(sorted((int(a), int(b), int(c))))
            if key in owner:
                k0, f0 = owner.pop(key)
                found.append((k0, k) + f0)
            else:
                owner[key] = (k, (int(a), int(b), int(c)))
    found.sort()
    plus = np.array([f[0] for f in found], dtype=np.int64)
    minus = np.array([f[1] for f in found], dtype=np.int64)
    va = np.array([f[2] for f in found], dtype=np.int64)
    vb = np.array([f[3] for f in found], dtype=np.int64)
    vc = np.array([f[4] for f in found], dtype=np.int64)
    V = mesh.vertices
    cr = np.cross(V[vb] - V[va], V[vc] - V[va])
    nrm = np.sqrt((cr ** 2).sum(1))
    return Faces(plus, minus, va, vb, cr / nrm[:, None], 0.5 * nrm, vc)
