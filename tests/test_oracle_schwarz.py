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


# ---- the massively parallel case of Sec. 4: every subdomain one fine element (T_S = T_h)

def test_massively_parallel_with_fine_coarse_space_closed_form():
    # T_S = T_h and the coarse cells are the fine elements with q = p: psi_J is the
    # fine modal basis on the same bounding box, so T_K = M_K^{-1} M_K = I, R_0^T = I,
    # K_0 = K and B_ad^{-1} = blockdiag(K_KK)^{-1} + K^{-1} (Eq. prec written out).
    m, d = small()
    cells = np.arange(m.n_cells, dtype=np.int32)
    S = schwarz.build(d, cells, cells, d.p)
    assert np.allclose(S.R0T.toarray(), np.eye(d.n_dofs), atol=1e-12)
    r = np.random.default_rng(11).standard_normal(d.n_dofs)
    Kd = d.K.toarray()
    n = d.n_p
    local = np.concatenate([sla.solve(Kd[k * n:(k + 1) * n, k * n:(k + 1) * n], r[k * n:(k + 1) * n])
                            for k in range(m.n_cells)])
    expect = local + np.linalg.solve(Kd, r)
    assert np.allclose(S.apply(r), expect, rtol=1e-10, atol=1e-13)


def test_massively_parallel_coarse_correction_is_k_orthogonal_projection(voronoi256):
    # Q = R_0^T K_0^{-1} R_0 K with K_0 = R_0 K R_0^T: Q^2 = Q and K Q symmetric, for a
    # coarse space of degree 1 and of degree q = p on the k-means agglomerates, with
    # every fine element its own subdomain.  A transposed R_0 or a wrong K_0 breaks both.
    w, d = voronoi256
    cells = np.arange(w.mesh.n_cells, dtype=np.int32)
    K = d.K.toarray()
    for q in (1, d.p):
        S = schwarz.build(d, cells, w.coarse, q)
        R0T = S.R0T.toarray()
        Q = R0T @ sla.cho_solve(S.K0_chol, R0T.T @ K)
        assert np.abs(Q @ Q - Q).max() <= 1e-8 * np.abs(Q).max()
        KQ = K @ Q
        assert np.abs(KQ - KQ.T).max() <= 1e-8 * np.abs(KQ).max()


def test_massively_parallel_spectrum_bounded_by_colouring():
    # Non-overlapping element subspaces on a Cartesian mesh are two-colourable (elements
    # of one colour share no face, so their K-projections are mutually K-orthogonal and
    # sum to a projection): lambda_max(B K) <= 2 + 1 (coarse projection).  The lower
    # end is positive (B SPD).  Block Jacobi alone is bounded by 2.
    m, d = small()
    cells = np.arange(m.n_cells, dtype=np.int32)
    K = d.K.toarray()
    for coarse, bound in ((None, 2.0), (block_partition(4, 2), 3.0)):
        S = schwarz.build(d, cells, coarse, d.p if coarse is not None else 1)
        BK = np.stack([S.apply(col) for col in K.T], 1)
        ev = np.linalg.eigvals(BK)
        assert np.abs(ev.imag).max() < 1e-8
        assert 0 < ev.real.min() and ev.real.max() <= bound + 1e-10
