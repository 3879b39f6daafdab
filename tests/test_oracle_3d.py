"""Pins of the oracle on polyhedral (3D) meshes (no GPU).

Closed forms that do not go through the oracle's own rules: simplex moments of
barycentric monomials, the divergence theorem facet by facet, Legendre
orthogonality on a box, the constant and linear functions of the SIP form, a
manufactured Neumann problem's h^(p+1) rate, and the Schwarz special cases.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, basis, quadrature, schwarz
from oracle.mesh import geometry, interior_faces
from oracle.pcg import pcg
from synth.meshes import jittered_hex_cube, block_partition_3d, isotropic_conductivity
from tests.conftest import cached


def random_spd(n_cells, seed):
    """Seeded per-cell SPD conductivities (input data for the anisotropic pins)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n_cells, 3, 3))
    return 0.3 * np.einsum("kij,klj->kil", B, B) + np.eye(3)[None]


def hex_disc(n, p, aniso=False, seed=3):
    def make():
        m = jittered_hex_cube(n, seed)
        S = random_spd(m.n_cells, 5) if aniso else isotropic_conductivity(m.n_cells, 1.0, dim=3)
        return m, assembly.assemble(m, p, S, 10.0, 1.0, 0.1)
    return cached(("hex", n, p, aniso, seed), make)


# ------------------------------------------------------------------- quadrature
def test_triangle_rule_in_space_barycentric_moments():
    # int_T l1^a l2^b l3^c dS = 2|T| a! b! c! / (a + b + c + 2)!
    rng = np.random.default_rng(0)
    A, B, C = rng.standard_normal((3, 3))
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    n = 3                                         # exact to degree 2n - 2 = 4
    x, w = quadrature.triangle_rule_3d(A, B, C, n)
    M = np.stack([A, B, C], 1)                    # columns: vertices; x = M l
    Lb = np.linalg.lstsq(np.vstack([M, np.ones(3)]), np.vstack([x.T, np.ones(len(x))]), rcond=None)[0]
    for a, b, c in [(0, 0, 0), (1, 0, 0), (2, 1, 0), (1, 1, 1), (0, 2, 2), (4, 0, 0)]:
        got = np.sum(w * Lb[0] ** a * Lb[1] ** b * Lb[2] ** c)
        want = 2 * area * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)
        assert np.isclose(got, want, rtol=1e-13), (a, b, c)


def test_gauss_jacobi_weights_and_exactness():
    # sum w = 1/(power+1); the rule integrates s^k s^power exactly for k <= 2n - 1
    for power in (1, 2):
        for n in (1, 2, 3, 4):
            s, w = quadrature.gauss_jacobi_01(n, power)
            for k in range(2 * n):
                assert np.isclose(np.sum(w * s ** k), 1.0 / (k + power + 1), rtol=1e-13), (power, n, k)
            assert not np.isclose(np.sum(w * s ** (2 * n)), 1.0 / (2 * n + power + 1), rtol=1e-9)


def test_tet_rule_barycentric_moments_to_degree_2n_minus_1():
    # int_T l1^a l2^b l3^c l4^d dV = 6|T| a! b! c! d! / (a + b + c + d + 3)!
    rng = np.random.default_rng(1)
    P = rng.standard_normal((4, 3))
    vol = abs(np.linalg.det(P[1:] - P[0])) / 6.0
    for n in (2, 3):
        x, w = quadrature.tet_rule(*P, n)
        assert len(w) == (14 if n == 3 else n ** 3)
        Lb = np.linalg.solve(np.vstack([P.T, np.ones(4)]), np.vstack([x.T, np.ones(len(x))]))
        for e in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 0, 0, 2), (1, 1, 0, 0), (0, 1, 1, 1),
                  (2 * n - 1, 0, 0, 0), (0, 0, 0, 2 * n - 1), (0, n - 1, 0, n), (1, 1, 1, 2 * n - 4)]:
            if sum(e) > 2 * n - 1 or min(e) < 0:
                continue
            got = np.sum(w * np.prod([Lb[i] ** e[i] for i in range(4)], axis=0))
            want = 6 * vol * np.prod([math.factorial(k) for k in e]) / math.factorial(sum(e) + 3)
            assert np.isclose(got, want, rtol=1e-12), (n, e)


def test_symmetric_tet_rule_is_exact_to_degree_5_and_no_further():
    # every barycentric monomial of degree <= 5 on a random tetrahedron (126 of them),
    # against 6|T| a! b! c! d! / (a + b + c + d + 3)!; positive weights, interior points,
    # the point set closed under the vertex permutations; some degree-6 monomial is missed
    rng = np.random.default_rng(5)
    P = rng.standard_normal((4, 3))
    vol = abs(np.linalg.det(P[1:] - P[0])) / 6.0
    x, w = quadrature.tet_rule(*P, 3)
    L, wr = quadrature.tet_symmetric_deg5()
    assert len(w) == 14 and np.all(wr > 0) and np.all(L > 0) and np.allclose(L.sum(1), 1.0)
    assert np.isclose(w.sum(), vol, rtol=1e-14)
    for perm in itertools.permutations(range(4)):
        Lp = L[:, perm]
        for k in range(14):
            j = np.argmin(np.abs(L - Lp[k]).sum(1))
            assert np.abs(L[j] - Lp[k]).max() < 1e-15 and wr[j] == wr[k]
    Lb = np.linalg.solve(np.vstack([P.T, np.ones(4)]), np.vstack([x.T, np.ones(len(x))]))
    missed = 0
    for e in itertools.product(range(7), repeat=4):
        if sum(e) > 6:
            continue
        got = np.sum(w * np.prod([Lb[i] ** e[i] for i in range(4)], axis=0))
        want = 6 * vol * np.prod([math.factorial(k) for k in e]) / math.factorial(sum(e) + 3)
        if sum(e) <= 5:
            assert np.isclose(got, want, rtol=1e-12), e
        else:
            missed += not np.isclose(got, want, rtol=1e-6)
    assert missed > 0


@pytest.mark.parametrize("p", [1, 2])
def test_polyhedron_rule_matches_divergence_theorem(p):
    # int_K x^a y^b z^c = 1/(a+1) sum_F n_x int_F x^(a+1) y^b z^c, facet by facet
    m = jittered_hex_cube(2, 9)
    V = m.vertices
    for k in range(m.n_cells):
        x, w = quadrature.polyhedron_rule(V, m.facets(k), p + 1)
        for a, b, c in [(0, 0, 0), (1, 0, 0), (0, 1, 1), (2, 1, 1), (0, 0, 2 * p), (p, p, 0)]:
            if a + b + c > 2 * p:
                continue
            got = np.sum(w * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
            want = 0.0
            for fa, fb, fc in m.facets(k):
                cr = np.cross(V[fb] - V[fa], V[fc] - V[fa])
                nx = cr[0] / np.linalg.norm(cr)
                xs, ws = quadrature.triangle_rule_3d(V[fa], V[fb], V[fc], p + 2)
                want += nx * np.sum(ws * xs[:, 0] ** (a + 1) * xs[:, 1] ** b * xs[:, 2] ** c) / (a + 1)
            assert np.isclose(got, want, rtol=1e-12, atol=1e-15), (k, a, b, c)


# --------------------------------------------------------------------- mesh
def test_hex_mesh_connectivity_and_volumes():
    n = 3
    m = jittered_hex_cube(n, 4)
    f = interior_faces(m)
    assert len(f.plus) == 2 * 3 * n * n * (n - 1)       # two triangles per interior quad
    assert np.all(f.plus < f.minus)
    g = geometry(m)
    assert abs(g.area.sum() - 1.0) < 1e-14
    for k in range(m.n_cells):                          # closed surfaces: sum of area normals = 0
        F = m.vertices[m.facets(k)]
        s = np.cross(F[:, 1] - F[:, 0], F[:, 2] - F[:, 0]).sum(0)
        assert np.abs(s).max() < 1e-15
        x, w = quadrature.polyhedron_rule(m.vertices, m.facets(k), 2)
        assert np.isclose(w.sum(), g.area[k], rtol=1e-13)
    # unmatched facets lie on the cube's boundary
    keys = {}
    for t in m.face_vtx:
        keys[tuple(sorted(t))] = keys.get(tuple(sorted(t)), 0) + 1
    for key, cnt in keys.items():
        if cnt == 1:
            P = m.vertices[list(key)]
            assert any(np.all(P[:, d] == s) for d in range(3) for s in (0.0, 1.0))


# -------------------------------------------------------------------- basis
def test_basis_3d_dimension_order_and_orthogonality():
    for p in range(1, 5):
        ms = basis.modes(p, 3)
        assert len(ms) == math.comb(p + 3, 3)
        assert [mm[:2] for mm in ms if mm[2] == 0] == basis.modes(p, 2)
    box = (0.1, 0.4, -0.2, 0.3, 0.5, 0.6)
    t, wt = np.polynomial.legendre.leggauss(5)        # tensor Gauss on the box
    T = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    W = np.einsum("i,j,k->ijk", wt, wt, wt).ravel()
    lo, hi = np.array(box[0::2]), np.array(box[1::2])
    x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * T
    W = W * np.prod(0.5 * (hi - lo))
    V, G = basis.eval_basis(3, box, x)
    Mb = V.T @ (W[:, None] * V)
    want = np.diag([np.prod([2.0 / (2 * a + 1) for a in mm]) * np.prod(hi - lo) / 8 for mm in basis.modes(3, 3)])
    assert np.allclose(Mb, want, atol=1e-14)
    # gradients against central differences
    hstep = 1e-6
    for d in range(3):
        e = np.zeros(3); e[d] = hstep
        Vp, _ = basis.eval_basis(3, box, x + e)
        Vm, _ = basis.eval_basis(3, box, x - e)
        assert np.allclose(G[:, :, d], (Vp - Vm) / (2 * hstep), atol=1e-5)


# ----------------------------------------------------------------- assembly
def linear_coeffs3(d, which):
    """Coefficients of u = 1, x, y, z: slots 0 and 1 + axis from the box map."""
    c = np.zeros((d.mesh.n_cells, d.n_p))
    bb = d.geom.bbox
    if which == 0:
        c[:, 0] = 1.0
    else:
        ax = which - 1
        c[:, 0] = 0.5 * (bb[:, 2 * ax] + bb[:, 2 * ax + 1])
        c[:, 1 + ax] = 0.5 * (bb[:, 2 * ax + 1] - bb[:, 2 * ax])
    return c.ravel()


def test_mass_moments_hex():
    m, d = hex_disc(3, 2)
    one, X, Y, Z = (linear_coeffs3(d, i) for i in range(4))
    assert abs(one @ d.M @ one - 1.0) < 1e-14
    assert abs(one @ d.M @ X - 0.5) < 1e-14
    assert abs(X @ d.M @ X - 1.0 / 3.0) < 1e-14
    assert abs(X @ d.M @ Y - 0.25) < 1e-14
    # int x y z = 1/8: y z is in P2, its projection is exact
    YZ = assembly.l2_project(d, lambda x: x[:, 1] * x[:, 2])
    assert abs(X @ d.M @ YZ - 0.125) < 1e-13


def test_stiffness_null_space_and_linear_energy_anisotropic():
    m, d = hex_disc(3, 2, aniso=True)
    one, X, Y, Z = (linear_coeffs3(d, i) for i in range(4))
    scale = abs(d.A).max()
    assert np.abs(d.A @ one).max() < 1e-12 * scale
    vol = d.geom.area
    for i, U in enumerate((X, Y, Z)):
        for j, W in enumerate((X, Y, Z)):
            assert np.isclose(U @ d.A @ W, (vol * d.sigma[:, i, j]).sum(), rtol=1e-11, atol=1e-12)


def test_symmetric_positive_definite_hex():
    m, d = hex_disc(2, 2, aniso=True)
    assert (d.K != d.K.T).nnz == 0
    np.linalg.cholesky(d.K.toarray())
    # two triangles per quad face: the pair's blocks are summed into one neighbour block
    assert d.K.nnz == (m.n_cells + 2 * 3 * 2 * 2 * 1) * d.n_p ** 2


def l2_error3(d, U, u):
    err = 0.0
    for k in range(d.mesh.n_cells):
        x, w = quadrature.polyhedron_rule(d.mesh.vertices, d.mesh.facets(k), d.p + 3)
        V, _ = basis.eval_basis(d.p, d.geom.bbox[k], x)
        err += np.sum(w * (V @ U.reshape(-1, d.n_p)[k] - u(x)) ** 2)
    return np.sqrt(err)


@pytest.mark.slow
@pytest.mark.parametrize("p", [2])
def test_convergence_rate_hex(p):
    """u = cos(pi x) cos(pi y) cos(pi z) solves u - dt/2 div(grad u) = (1 + 3/2 dt pi^2) u
    with homogeneous Neumann data; the L2 error falls like h^(p+1)."""
    dt = 2.0
    u = lambda x: np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) * np.cos(np.pi * x[:, 2])
    errs = []
    ns = (3, 6)
    for n in ns:
        m = jittered_hex_cube(n, 6)
        d = assembly.assemble(m, p, isotropic_conductivity(m.n_cells, 1.0, dim=3), 10.0, 1.0, dt)
        rhs = assembly.load_vector(d, lambda x: (1.0 + 1.5 * dt * np.pi ** 2) * u(x))
        errs.append(l2_error3(d, spla.spsolve(d.K.tocsc(), rhs), u))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 1 - 0.5, (errs, rate)


@pytest.mark.parametrize("p", [2, 3])
def test_interior_face_consistency_hex(p):
    """For the continuous u = x^2 and a constant Sigma, the interior-face terms of Eq. coer
    reduce A(u, v) to int (-div Sigma grad u) v + int_{boundary} (Sigma grad u . n) v for
    every DG function v: here -2 Sigma_xx int v + sum over boundary facets of
    int 2 x (Sigma n)_x v.  A wrong normal, sign or average in the face blocks breaks it."""
    m = jittered_hex_cube(3, 8)
    S0 = random_spd(1, 11)[0]
    d = assembly.assemble(m, p, np.tile(S0, (m.n_cells, 1, 1)), 10.0, 1.0, 0.1)
    U = assembly.l2_project(d, lambda x: x[:, 0] ** 2)
    v = np.random.default_rng(4).standard_normal(d.n_dofs)
    lhs = v @ (d.A @ U)
    # int v over Omega: M-weighted against the constant function
    one = np.zeros((m.n_cells, d.n_p)); one[:, 0] = 1.0
    rhs = -2.0 * S0[0, 0] * (one.ravel() @ d.M @ v)
    owner = {}
    for k in range(m.n_cells):
        for t in m.facets(k):
            key = tuple(sorted(int(i) for i in t))
            owner[key] = None if key in owner else (k, t)
    V = m.vertices
    vv = v.reshape(-1, d.n_p)
    for val in owner.values():
        if val is None:
            continue
        k, (a, b, c) = val
        cr = np.cross(V[b] - V[a], V[c] - V[a])
        n = cr / np.linalg.norm(cr)
        xs, ws = quadrature.triangle_rule_3d(V[a], V[b], V[c], p + 2)
        Phi, _ = basis.eval_basis(p, d.geom.bbox[k], xs)
        rhs += np.sum(ws * 2.0 * xs[:, 0] * (S0 @ n)[0] * (Phi @ vv[k]))
    assert np.isclose(lhs, rhs, rtol=1e-11, atol=1e-11 * abs(lhs)), (lhs, rhs)


# ------------------------------------------------------------------ Schwarz
def test_schwarz_special_cases_hex():
    m, d = hex_disc(2, 2)
    b = np.random.default_rng(3).standard_normal(d.n_dofs)
    zeros = np.zeros(m.n_cells, np.int32)
    S1 = schwarz.build(d, zeros, None)
    assert pcg(d.K, b, prec=S1.apply, rtol=1e-12).iterations == 1
    S2 = schwarz.build(d, zeros, np.arange(m.n_cells, dtype=np.int32) // 4, 1)
    assert pcg(d.K, b, prec=S2.apply, rtol=1e-12).iterations <= 2


def test_coarse_prolongation_reproduces_p1_hex():
    m, d = hex_disc(4, 2)
    coarse = block_partition_3d(4, 2)
    R0T, boxes = schwarz.coarse_prolongation(d, coarse, 1)
    assert R0T.shape[1] == 8 * 4
    # coarse function v0 = z on every agglomerate (slot 3 of the P1 modes)
    c0 = np.zeros((len(boxes), 4))
    for J, bx in enumerate(boxes):
        c0[J, 0] = 0.5 * (bx[4] + bx[5]); c0[J, 3] = 0.5 * (bx[5] - bx[4])
    fine = (R0T @ c0.ravel()).reshape(-1, d.n_p)
    want = linear_coeffs3(d, 3).reshape(-1, d.n_p)
    assert np.allclose(fine, want, atol=1e-13)
