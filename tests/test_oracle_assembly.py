"""Pins of oracle.assembly: closed-form integrals, null spaces, SPD, convergence (no GPU)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, basis, quadrature
from oracle.assembly import element_rule
from synth.meshes import (cartesian_square, voronoi_square, isotropic_conductivity,
                          fibre_conductivity)


def linear_coeffs(disc, which):
    """Coefficients of u = 1, x or y in the modal basis, written from the affine map
    x = (x0 + x1)/2 + (x1 - x0)/2 * xi (modes (0,0), (1,0), (0,1) are slots 0, 1, 2)."""
    c = np.zeros((disc.mesh.n_cells, disc.n_p))
    bb = disc.geom.bbox
    if which == "1":
        c[:, 0] = 1.0
    elif which == "x":
        c[:, 0] = 0.5 * (bb[:, 0] + bb[:, 1]); c[:, 1] = 0.5 * (bb[:, 1] - bb[:, 0])
    else:
        c[:, 0] = 0.5 * (bb[:, 2] + bb[:, 3]); c[:, 2] = 0.5 * (bb[:, 3] - bb[:, 2])
    return c.ravel()


def test_mass_moments_unit_square(square16):
    _, d = square16
    one, X, Y = (linear_coeffs(d, s) for s in ("1", "x", "y"))
    assert abs(one @ d.M @ one - 1.0) < 1e-14
    assert abs(one @ d.M @ X - 0.5) < 1e-14
    assert abs(X @ d.M @ X - 1.0 / 3.0) < 1e-14
    assert abs(X @ d.M @ Y - 0.25) < 1e-14


def test_mass_moments_voronoi(voronoi256):
    _, d = voronoi256
    one, X, Y = (linear_coeffs(d, s) for s in ("1", "x", "y"))
    assert abs(one @ d.M @ one - 1.0) < 1e-13
    assert abs(X @ d.M @ X - 1.0 / 3.0) < 1e-13
    assert abs(X @ d.M @ Y - 0.25) < 1e-13


def test_stiffness_null_space_and_linear_energy(voronoi256):
    _, d = voronoi256
    one, X, Y = (linear_coeffs(d, s) for s in ("1", "x", "y"))
    scale = abs(d.A).max()
    assert np.abs(d.A @ one).max() < 1e-12 * scale
    # u = x, y are continuous: jumps and face terms vanish, A(u, v) = int Sigma grad u . grad v
    area = d.geom.area
    assert np.isclose(X @ d.A @ X, (area * d.sigma[:, 0, 0]).sum(), rtol=1e-12)
    assert np.isclose(X @ d.A @ Y, (area * d.sigma[:, 0, 1]).sum(), rtol=1e-10, atol=1e-12)
    assert np.isclose(Y @ d.A @ Y, (area * d.sigma[:, 1, 1]).sum(), rtol=1e-12)


def test_symmetric_positive_definite(square16):
    _, d = square16
    assert (d.K != d.K.T).nnz == 0
    ev = np.linalg.eigvalsh(d.K.toarray())
    assert ev[0] > 0
    np.linalg.cholesky(d.K.toarray())


def test_penalty_closed_form(square16):
    w, d = square16
    # sigma = 1, equal diameters sqrt(2)/16: eta = 10 * 1 * p^2 / h
    assert np.allclose(d.eta, 10.0 * 4 / (np.sqrt(2.0) / 16))


def test_penalty_uses_spectral_norm_and_averages():
    m = cartesian_square(2)
    S = np.array([np.diag([2.0, 1.0]), np.diag([1.0, 3.0]), np.eye(2), np.eye(2)])
    d = assembly.assemble(m, 1, S, 5.0, 1.0, 0.1)
    f = list(zip(d.faces.plus, d.faces.minus)).index((0, 1))
    assert np.isclose(d.eta[f], 5.0 * 0.5 * (2.0 + 3.0) * 1 / (np.sqrt(2.0) / 2))


def l2_error(d, U, u):
    err = 0.0
    for k in range(d.mesh.n_cells):
        x, w = quadrature.polygon_rule(d.mesh.vertices[d.mesh.cell(k)], d.p + 3)
        V, _ = basis.eval_basis(d.p, d.geom.bbox[k], x)
        err += np.sum(w * (V @ U.reshape(-1, d.n_p)[k] - u(x)) ** 2)
    return np.sqrt(err)


def manufactured(mesh, p, a, b, dt=2.0):
    """u = cos(pi x) cos(2 pi y) solves u - dt/2 div(Sigma grad u) = g with Sigma = diag(a, b)
    and homogeneous Neumann data on the unit square; g = (1 + dt/2 pi^2 (a + 4b)) u."""
    S = np.tile(np.diag([a, b]), (mesh.n_cells, 1, 1))
    d = assembly.assemble(mesh, p, S, 10.0, 1.0, dt)
    u = lambda x: np.cos(np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    c = 1.0 + 0.5 * dt * np.pi ** 2 * (a + 4 * b)
    rhs = assembly.load_vector(d, lambda x: c * u(x))
    U = spla.spsolve(d.K.tocsc(), rhs)
    return l2_error(d, U, u)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_rate_cartesian(p):
    errs = [manufactured(cartesian_square(n), p, 1.0, 0.4) for n in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.3, (errs, rates)


def test_convergence_rate_voronoi():
    p = 2
    errs, hs = [], []
    for n in (64, 256, 1024):
        m = voronoi_square(n, 11)
        errs.append(manufactured(m, p, 0.7, 1.3))
        hs.append(1.0 / np.sqrt(n))
    rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(np.array(hs[:-1]) / np.array(hs[1:]))
    assert rates[-1] > p + 1 - 0.5, (errs, rates)


def test_convergence_detects_swapped_conductivity():
    # Sensitivity: assembling with diag(b, a) instead of diag(a, b) must break the rate.
    m = cartesian_square(16)
    p = 2
    S = np.tile(np.diag([1.3, 0.7]), (m.n_cells, 1, 1))
    d = assembly.assemble(m, p, S, 10.0, 1.0, 2.0)
    u = lambda x: np.cos(np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    c = 1.0 + np.pi ** 2 * (0.7 + 4 * 1.3)
    U = spla.spsolve(d.K.tocsc(), assembly.load_vector(d, lambda x: c * u(x)))
    assert l2_error(d, U, u) > 1e-2
