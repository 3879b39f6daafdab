"""Pins of oracle.mesh: connectivity and geometry (no GPU)."""
import numpy as np

from oracle import mesh as omesh
from synth.meshes import cartesian_square, voronoi_square


def test_cartesian_counts_and_geometry():
    n = 8
    m = cartesian_square(n)
    f = omesh.interior_faces(m)
    assert len(f.plus) == 2 * n * (n - 1)
    g = omesh.geometry(m)
    assert np.allclose(g.area, 1.0 / n ** 2)
    assert np.allclose(g.diameter, np.sqrt(2.0) / n)
    assert np.allclose(f.length, 1.0 / n)
    assert np.all(f.plus < f.minus)


def test_voronoi_areas_normals_orientation():
    m = voronoi_square(300, 5)
    g = omesh.geometry(m)
    assert np.isclose(g.area.sum(), 1.0, atol=1e-13)
    assert np.all(g.area > 0)
    f = omesh.interior_faces(m)
    # Euler: V - E + F = 1 for a planar subdivision of the square
    nb = sum(1 for k in range(m.n_cells) for _ in range(len(m.cell(k)))) - 2 * len(f.plus)
    E = len(f.plus) + nb
    assert len(m.vertices) - E + m.n_cells == 1
    # normals are unit, orthogonal to the edge and point from K+ towards K-
    V = m.vertices
    cen = np.array([V[m.cell(k)].mean(0) for k in range(m.n_cells)])
    assert np.allclose(np.linalg.norm(f.normal, axis=1), 1.0)
    assert np.allclose(((V[f.vb] - V[f.va]) * f.normal).sum(1), 0.0, atol=1e-15)
    assert np.all(((cen[f.minus] - cen[f.plus]) * f.normal).sum(1) > 0)
