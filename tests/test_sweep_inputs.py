"""Host-side inputs of the massively parallel sweep (no GPU): agglomerates aligned with
the grey/white interface, the conductivity tensors of the two regions, the initial
potential and the Table 1 layout of the report."""
import numpy as np

from paper_2512_19536_gb300 import schwarz_sweep as sw
from synth.meshes import voronoi_square, cell_points


def test_agglomerates_aligned_dense_and_sized():
    m = voronoi_square(512, 9)
    pts = cell_points(m)
    grey = pts[:, 1] >= 0.5
    for ratio in (2, 4, 8, 16):
        n_agg = max(2, round(512 / ratio ** 2))
        lab = sw.aligned_agglomerates(pts, n_agg, 5)
        ids = np.unique(lab)
        assert np.array_equal(ids, np.arange(len(ids)))          # dense ids, all used
        assert abs(len(ids) - n_agg) <= 1
        for J in ids:                                             # no agglomerate crosses y = 0.5
            assert grey[lab == J].all() or (~grey[lab == J]).all()


def test_grey_white_conductivity():
    pts = np.array([[0.3, 0.7], [0.6, 0.2]])
    s = sw.grey_white_conductivity(pts)
    assert np.allclose(s[0], 0.63 * np.eye(2))
    # white matter: sigma_l = 0.69 along e_y, sigma_n = 2.571 across it
    assert np.isclose(np.array([0, 1.0]) @ s[1] @ np.array([0, 1.0]), 0.69)
    assert np.isclose(np.array([1.0, 0]) @ s[1] @ np.array([1.0, 0]), 2.571)
    assert np.allclose(s[1], s[1].T)


def test_initial_potential_marks_the_imbalance_region():
    pts = np.array([[0.5, 0.95], [0.5, 0.5], [0.1, 0.99]])
    u = sw.initial_potential(pts, 3).reshape(3, 3)
    assert np.array_equal(u[:, 0], [-50.0, -67.0, -67.0])
    assert np.all(u[:, 1:] == 0.0)


def test_markdown_layout():
    rows = [{"p": 1, "n_h": 512, "H_over_h": 2, "kappa": 55.06, "its_per_step": 69.0},
            {"p": 1, "n_h": 512, "H_over_h": 4, "skipped": "big"},
            {"p": 1, "n_h": 512, "H_over_h": None, "kappa": 1.34e4, "its_per_step": 596.0}]
    md = sw.markdown(rows)
    assert "| 2h | 55.06 (69.0) |" in md and "| 4h | — |" in md and "| CG | 1.34e+04 (596.0) |" in md
