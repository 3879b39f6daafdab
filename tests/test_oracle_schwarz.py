"""Pins of oracle.schwarz (Eq. prec) (no GPU)."""
import numpy as np
import scipy.linalg as sla

from oracle import assembly, schwarz
from oracle.pcg import pcg
from synth.meshes import cartesian_square, block_partition, isotropic_conductivity


def small():
    m = cartesian_square(4)
    d = assembly.assemble(m, 2, isotropic_conductivity(16, 1.0), 10.0, 1.0, 0.1)
    return m, d


def test_symmetric(voronoi256):
    w, d = voronoi256
    S = schwarz.build(d, w.subdomain, w.coarse, 1)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal((2, d.n_dofs))
    assert np.isclose(x @ S.apply(y), y @ S.apply(x), rtol=1e-12)


def test_one_subdomain_one_level_is_exact_inverse():
    m, d = small()
    S = schwarz.build(d, np.zeros(m.n_cells, np.int32), None)
    b = np.random.default_rng(1).standard_normal(d.n_dofs)
    r = pcg(d.K, b, prec=S.apply, rtol=1e-12)
    assert r.iterations == 1


def test_one_subdomain_two_level_at_most_two_iterations():
    # B K = I + P_0 with P_0 a K-orthogonal projection: eigenvalues {1, 2}.
    m, d = small()
    zeros = np.zeros(m.n_cells, np.int32)
    S = schwarz.build(d, zeros, block_partition(4, 2), 1)
    BK = np.stack([S.apply(col) for col in d.K.toarray().T], 1)
    ev = np.sort(np.linalg.eigvals(BK).real)
    assert np.allclose(ev[(ev > 1.5)], 2.0) and np.allclose(ev[(ev < 1.5)], 1.0)
    b = np.random.default_rng(1).standard_normal(d.n_dofs)
    assert pcg(d.K, b, prec=S.apply, rtol=1e-12).iterations <= 2


def test_coarse_prolongation_reproduces_coarse_linear_function(voronoi256):
    w, d = voronoi256
    R0T, boxes = schwarz.coarse_prolongation(d, w.coarse, 1)
    # coarse function v0 = x on every agglomerate: slots (0,0) and (1,0) from J's box
    n_agg = len(boxes)
    c0 = np.zeros((n_agg, 3))
    for J, (X0, X1, _, _) in enumerate(boxes):
        c0[J, 0] = 0.5 * (X0 + X1); c0[J, 1] = 0.5 * (X1 - X0)
    fine = (R0T @ c0.ravel()).reshape(-1, d.n_p)
    bb = d.geom.bbox
    assert np.allclose(fine[:, 0], 0.5 * (bb[:, 0] + bb[:, 1]), atol=1e-13)
    assert np.allclose(fine[:, 1], 0.5 * (bb[:, 1] - bb[:, 0]), atol=1e-13)
    assert np.allclose(fine[:, 2:], 0.0, atol=1e-13)


def test_element_block_jacobi_special_case():
    # T_S = T_h and no coarse space: B is the inverse of the element-diagonal blocks of K.
    m, d = small()
    S = schwarz.build(d, np.arange(m.n_cells, dtype=np.int32), None)
    r = np.random.default_rng(2).standard_normal(d.n_dofs)
    Kd = d.K.toarray()
    n = d.n_p
    expect = np.concatenate([sla.solve(Kd[k * n:(k + 1) * n, k * n:(k + 1) * n], r[k * n:(k + 1) * n])
                             for k in range(m.n_cells)])
    assert np.allclose(S.apply(r), expect, rtol=1e-12, atol=1e-14)


def test_preconditioned_spectrum_real_positive():
    m, d = small()
    S = schwarz.build(d, block_partition(4, 2), block_partition(4, 2), 1)
    BK = np.stack([S.apply(col) for col in d.K.toarray().T], 1)
    ev = np.linalg.eigvals(BK)
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0
