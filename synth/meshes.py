"""Seeded polygonal meshes of the unit square, partitions and conductivity fields.

A 2D mesh is a set of vertices (float64, shape [nv, 2]) and convex polygonal
cells given as counter-clockwise vertex loops in CSR form (``cell_ptr`` int64
[nc+1], ``cell_vtx`` int32).  Cells that share an edge share both vertex ids,
so connectivity can be recovered exactly from integer ids.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    vertices: np.ndarray      # [nv, dim] float64
    cell_ptr: np.ndarray      # [nc+1] int64
    cell_vtx: np.ndarray      # [cell_ptr[-1]] int32, CCW loops
    dim: int = 2

    @property
    def n_cells(self) -> int:
        return len(self.cell_ptr) - 1

    def cell(self, k: int) -> np.ndarray:
        return self.cell_vtx[self.cell_ptr[k]:self.cell_ptr[k + 1]]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def cartesian_square(n: int) -> Mesh:
    """n x n axis-aligned squares on [0,1]^2; cell (i, j) -> id j*n + i."""
    xs = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    cells = []
    for j in range(n):
        for i in range(n):
            v0 = j * (n + 1) + i
            cells.append([v0, v0 + 1, v0 + n + 2, v0 + n + 1])
    cell_vtx = np.asarray(cells, dtype=np.int32).ravel()
    cell_ptr = np.arange(0, 4 * n * n + 1, 4, dtype=np.int64)
    return Mesh(verts, cell_ptr, cell_vtx)


def _polygon_centroids(verts, cell_ptr, cell_vtx):
    """Area centroids of CCW polygons (used only to move Lloyd seeds)."""
    nc = len(cell_ptr) - 1
    out = np.empty((nc, 2))
    for k in range(nc):
        P = verts[cell_vtx[cell_ptr[k]:cell_ptr[k + 1]]]
        Q = np.roll(P, -1, axis=0)
        cr = P[:, 0] * Q[:, 1] - Q[:, 0] * P[:, 1]
        a = 0.5 * cr.sum()
        out[k, 0] = ((P[:, 0] + Q[:, 0]) * cr).sum() / (6.0 * a)
        out[k, 1] = ((P[:, 1] + Q[:, 1]) * cr).sum() / (6.0 * a)
    return out


def _voronoi_cells(seeds: np.ndarray):
    """Voronoi cells of ``seeds`` clipped to [0,1]^2 via mirrored seeds.

    The seeds are mirrored across the four sides of the square; each original
    seed's cell in the Voronoi diagram of the union is its cell clipped to the
    square.  Vertices are circumcentres of the Delaunay triangles; those that
    coincide (co-circular seeds, which mirroring always creates) are merged so
    that neighbouring cells share vertex ids.
    """
    from scipy.spatial import Delaunay, cKDTree

    n = len(seeds)
    x, y = seeds[:, 0], seeds[:, 1]
    allp = np.concatenate([
        seeds,
        np.stack([-x, y], 1), np.stack([2.0 - x, y], 1),
        np.stack([x, -y], 1), np.stack([x, 2.0 - y], 1)])
    tri = Delaunay(allp)
    S = tri.simplices
    A, B, C = allp[S[:, 0]], allp[S[:, 1]], allp[S[:, 2]]
    d = 2.0 * (A[:, 0] * (B[:, 1] - C[:, 1]) + B[:, 0] * (C[:, 1] - A[:, 1])
               + C[:, 0] * (A[:, 1] - B[:, 1]))
    a2, b2, c2 = (A ** 2).sum(1), (B ** 2).sum(1), (C ** 2).sum(1)
    ux = (a2 * (B[:, 1] - C[:, 1]) + b2 * (C[:, 1] - A[:, 1]) + c2 * (A[:, 1] - B[:, 1])) / d
    uy = (a2 * (C[:, 0] - B[:, 0]) + b2 * (A[:, 0] - C[:, 0]) + c2 * (B[:, 0] - A[:, 0])) / d
    cc = np.stack([ux, uy], 1)
    # snap to the square's sides (exact in exact arithmetic for mirrored pairs)
    for col in range(2):
        cc[np.abs(cc[:, col]) < 1e-10, col] = 0.0
        cc[np.abs(cc[:, col] - 1.0) < 1e-10, col] = 1.0

    # triangles incident to each original seed
    tri_of_pt = [[] for _ in range(n)]
    for t, s in enumerate(S):
        for v in s:
            if v < n:
                tri_of_pt[v].append(t)
    used = sorted({t for lst in tri_of_pt for t in lst})
    used = np.asarray(used, dtype=np.int64)
    # merge coincident circumcentres: union-find over pairs closer than 1e-11
    P = cc[used]
    tree = cKDTree(P)
    parent = np.arange(len(P))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for i, j in sorted(tree.query_pairs(1e-11)):
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)
    root = np.array([find(i) for i in range(len(P))])
    reps = np.unique(root)
    # deterministic vertex numbering: lexicographic in (y, x) of representatives
    order = np.lexsort((P[reps, 0], P[reps, 1]))
    new_id_of_rep = np.empty(len(P), dtype=np.int64)
    new_id_of_rep[reps[order]] = np.arange(len(reps))
    tri_to_vid = np.full(len(S), -1, dtype=np.int64)
    tri_to_vid[used] = new_id_of_rep[root]
    verts = P[reps[order]].copy()

    cell_ptr = [0]
    cell_vtx = []
    for i in range(n):
        ts = np.asarray(tri_of_pt[i])
        ang = np.arctan2(cc[ts, 1] - seeds[i, 1], cc[ts, 0] - seeds[i, 0])
        ts = ts[np.argsort(ang, kind="stable")]
        loop = [int(tri_to_vid[t]) for t in ts]
        # drop repeats created by merged (co-circular) circumcentres
        clean = []
        for v in loop:
            if not clean or clean[-1] != v:
                clean.append(v)
        while len(clean) > 1 and clean[0] == clean[-1]:
            clean.pop()
        if len(clean) < 3:
            raise RuntimeError("degenerate Voronoi cell")
        cell_vtx.extend(clean)
        cell_ptr.append(len(cell_vtx))
    return verts, np.asarray(cell_ptr, np.int64), np.asarray(cell_vtx, np.int32)


def _check_watertight(mesh: Mesh) -> None:
    """Every edge is used once (on the square's boundary) or twice, reversed."""
    edges = {}
    V = mesh.vertices
    for k in range(mesh.n_cells):
        c = mesh.cell(k)
        for a, b in zip(c, np.roll(c, -1)):
            edges[(int(a), int(b))] = edges.get((int(a), int(b)), 0) + 1
    for (a, b), m in edges.items():
        if m != 1:
            raise RuntimeError("edge used twice in one orientation")
        if (b, a) not in edges:
            pa, pb = V[a], V[b]
            on = any((pa[c] == s and pb[c] == s) for c in range(2) for s in (0.0, 1.0))
            if not on:
                raise RuntimeError("unmatched interior edge")


def voronoi_square(n_cells: int, seed: int, lloyd: int = 5) -> Mesh:
    """Voronoi mesh of ``n_cells`` uniform seeds in [0,1]^2, ``lloyd`` Lloyd steps."""
    seeds = _rng(seed).random((n_cells, 2))
    for it in range(lloyd + 1):
        verts, cp, cv = _voronoi_cells(seeds)
        if it < lloyd:
            seeds = _polygon_centroids(verts, cp, cv)
    mesh = Mesh(verts, cp, cv)
    _check_watertight(mesh)
    return mesh


def block_partition(n: int, b: int) -> np.ndarray:
    """Partition of the n x n Cartesian mesh into (n/b)^2 blocks of b x b cells."""
    m = n // b
    part = np.empty(n * n, dtype=np.int32)
    for j in range(n):
        for i in range(n):
            part[j * n + i] = (j // b) * m + (i // b)
    return part


def cell_points(mesh: Mesh) -> np.ndarray:
    """Vertex averages of the cells: a cheap interior point for seeding fields."""
    out = np.empty((mesh.n_cells, mesh.dim))
    for k in range(mesh.n_cells):
        out[k] = mesh.vertices[mesh.cell(k)].mean(axis=0)
    return out


def kmeans_partition(mesh: Mesh, k: int, seed: int, iters: int = 30) -> np.ndarray:
    """Seeded k-means of cell vertex-averages; ties go to the lowest cluster id."""
    return kmeans_points(cell_points(mesh), k, seed, iters)


def kmeans_points(pts: np.ndarray, k: int, seed: int, iters: int = 30) -> np.ndarray:
    """Seeded k-means labels of points [n, dim], dense ids by first appearance."""
    rng = _rng(seed)
    centres = pts[rng.choice(len(pts), size=k, replace=False)].copy()
    lab = np.zeros(len(pts), dtype=np.int32)
    for _ in range(iters):
        d2 = ((pts[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
        lab = np.argmin(d2, axis=1).astype(np.int32)
        for c in range(k):
            sel = lab == c
            if sel.any():
                centres[c] = pts[sel].mean(axis=0)
    # relabel clusters by first appearance so ids are dense and ordered
    uniq, first = np.unique(lab, return_index=True)
    remap = np.empty(k, dtype=np.int32)
    remap[uniq[np.argsort(first)]] = np.arange(len(uniq), dtype=np.int32)
    return remap[lab]


def isotropic_conductivity(n_cells: int, sigma: float, dim: int = 2) -> np.ndarray:
    return np.tile(sigma * np.eye(dim), (n_cells, 1, 1))


def fibre_conductivity(mesh: Mesh, sigma_l: float, sigma_t: float, seed: int,
                       kmax: int = 3) -> np.ndarray:
    """Piecewise-constant anisotropic conductivity along a seeded smooth fibre field.

    Fibre angle theta(x) = pi * sum_k b_k sin(pi k.x + phi_k) over integer
    wave vectors 0 < max|k_i| <= kmax, evaluated at each cell's vertex average;
    Sigma = sigma_t I + (sigma_l - sigma_t) l l^T with l = (cos theta, sin theta).
    """
    rng = _rng(seed)
    ks = [(a, b) for a in range(kmax + 1) for b in range(-kmax, kmax + 1)
          if (a, b) != (0, 0) and (a > 0 or b > 0)]
    ks = np.asarray(ks, dtype=np.float64)
    amp = rng.standard_normal(len(ks)) * 0.25 / (1.0 + (ks ** 2).sum(1))
    ph = rng.random(len(ks)) * 2.0 * np.pi
    pts = cell_points(mesh)
    theta = np.pi * (amp[None, :] * np.sin(np.pi * pts @ ks.T + ph[None, :])).sum(1)
    l = np.stack([np.cos(theta), np.sin(theta)], 1)
    S = sigma_t * np.eye(2)[None] + (sigma_l - sigma_t) * l[:, :, None] * l[:, None, :]
    return S


# ------------------------------------------------------------------ 3D meshes
@dataclass
class PolyMesh3D:
    """Polyhedral mesh: each cell is a closed surface of triangle facets.

    Facets are given per cell in CSR form (``cell_face_ptr`` int64 [nc+1] over
    ``face_vtx`` int32 [n_facets, 3]); every facet is oriented so that
    (b - a) x (c - a) points out of its cell.  Two cells share an interior face
    exactly when a facet's three vertex ids appear in both, in opposite
    orientation.
    """
    vertices: np.ndarray      # [nv, 3] float64
    cell_face_ptr: np.ndarray  # [nc+1] int64
    face_vtx: np.ndarray      # [n_facets, 3] int32
    dim: int = 3

    @property
    def n_cells(self) -> int:
        return len(self.cell_face_ptr) - 1

    def facets(self, k: int) -> np.ndarray:
        return self.face_vtx[self.cell_face_ptr[k]:self.cell_face_ptr[k + 1]]

    def cell(self, k: int) -> np.ndarray:
        """The cell's vertex ids, ascending."""
        return np.unique(self.facets(k))


# outward-oriented corner loops of the six faces of the unit hex, corners (di, dj, dk)
_HEX_FACES = (
    ((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)),   # x = 0
    ((1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)),   # x = 1
    ((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)),   # y = 0
    ((0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)),   # y = 1
    ((0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)),   # z = 0
    ((0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)),   # z = 1
)


def jittered_hex_cube(n: int, seed: int, jitter: float = 0.1) -> PolyMesh3D:
    """n^3 hexahedra on [0,1]^3 with seeded vertex jitter, as 12-facet polyhedra.

    Vertex (i, j, k) -> id (k (n+1) + j)(n+1) + i, moved by U[-jitter h, jitter h]
    (h = 1/n) along every axis in which it is not on the cube's boundary
    (boundary vertices move only tangentially; corners stay).  Each quadrilateral
    face is split into two triangles along the diagonal through its smallest
    vertex id, so both cells sharing a face split it the same way.  Cell (i, j, k)
    -> id (k n + j) n + i.
    """
    m = n + 1
    idx = np.arange(m)
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    grid = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)          # [nv, 3] ids along x, y, z
    h = 1.0 / n
    d = _rng(seed).uniform(-1.0, 1.0, grid.shape) * (jitter * h)
    d[(grid == 0) | (grid == n)] = 0.0
    verts = grid * h + d

    def vid(i, j, k):
        return (k * m + j) * m + i

    tris = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for quad in _HEX_FACES:
                    q = [vid(i + a, j + b, k + c) for a, b, c in quad]
                    s = int(np.argmin(q))
                    q = q[s:] + q[:s]
                    tris.append((q[0], q[1], q[2]))
                    tris.append((q[0], q[2], q[3]))
    face_vtx = np.asarray(tris, dtype=np.int32)
    cell_face_ptr = np.arange(0, 12 * n ** 3 + 1, 12, dtype=np.int64)
    return PolyMesh3D(verts, cell_face_ptr, face_vtx)


def block_partition_3d(n: int, b: int) -> np.ndarray:
    """Partition of the n^3 hex mesh into (n/b)^3 blocks of b^3 cells."""
    m = n // b
    c = np.arange(n)
    K, J, I = np.meshgrid(c, c, c, indexing="ij")
    return (((K // b) * m + J // b) * m + I // b).ravel().astype(np.int32)
