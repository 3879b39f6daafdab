"""Pins of the shared-eigenbasis local solves (oracle/multirhs.py): the conductivity
scaling of the SIP stiffness, the eigen form against dense solves, and the whole
preconditioner against oracle.schwarz on the assembly with that conductivity."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, schwarz, multirhs


@pytest.fixture(scope="module")
def case():
    from synth.meshes import voronoi_square, kmeans_partition, isotropic_conductivity
    m = voronoi_square(60, 21)
    part = kmeans_partition(m, 4, 21)
    d1 = assembly.assemble(m, 2, isotropic_conductivity(m.n_cells, 1.0), 10.0, 1.0, 0.05)
    return m, part, d1


def test_stiffness_scales_with_scalar_conductivity(case):
    from synth.meshes import isotropic_conductivity
    m, part, d1 = case
    d7 = assembly.assemble(m, 2, isotropic_conductivity(m.n_cells, 0.7), 10.0, 1.0, 0.05)
    diff = abs(d7.A - 0.7 * d1.A).max()
    assert diff <= 1e-12 * abs(d1.A).max()
    assert abs(d7.M - d1.M).max() == 0.0


@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.9])
def test_eigen_form_equals_dense_solves(case, sigma):
    m, part, d1 = case
    dofs = multirhs.subdomain_dofs(part, d1.n_p)
    S = multirhs.build(d1.M, d1.A, dofs, d1.n_p)
    r = np.random.default_rng(3).standard_normal(d1.n_dofs)
    z = multirhs.apply_local(S, r, sigma, 1.0, 0.05)
    K = (d1.M + (0.5 * 0.05 * sigma) * d1.A).tocsr()
    ref = np.zeros_like(r)
    for dd in dofs:
        ref[dd] = np.linalg.solve(K[dd][:, dd].toarray(), r[dd])
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)
    for Q in S.Q:
        assert np.allclose(Q.T @ Q, np.eye(Q.shape[0]), atol=1e-12)


def test_preconditioner_equals_schwarz_on_that_conductivity(case):
    from synth.meshes import isotropic_conductivity
    m, part, d1 = case
    sigma = 1.6
    ds = assembly.assemble(m, 2, isotropic_conductivity(m.n_cells, sigma), 10.0, 1.0, 0.05)
    B = schwarz.build(ds, part, part, 1)
    S = multirhs.build(d1.M, d1.A, multirhs.subdomain_dofs(part, d1.n_p), d1.n_p)
    r = np.random.default_rng(4).standard_normal(d1.n_dofs)
    # local part: B minus its coarse correction
    r0 = B.R0T.T @ r
    import scipy.linalg as sla
    local_ref = B.apply(r) - B.R0T @ sla.cho_solve(B.K0_chol, r0)
    assert np.linalg.norm(multirhs.apply_local(S, r, sigma, 1.0, 0.05) - local_ref) <= \
        1e-10 * np.linalg.norm(local_ref)
