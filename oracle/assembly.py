"""Symmetric interior-penalty PolyDG assembly: M_h, A_h and K_h (FP64).

Sec. 3 of the paper:
  * Eq. eta: on an interior face F shared by K+ and K-,
        eta = eta0 * {Sigma_K}_A * p^2 / {h_K}_H,
    {.}_A the arithmetic and {.}_H the harmonic average.  Sigma_K is read as
    the spectral norm |sqrt(Sigma_K)|_2^2 = lambda_max(Sigma_K) of the
    element's constant conductivity (the printed L2(K) norm would carry an
    area factor; see the list of readings).
  * Eq. coer: A(u,v) = sum_K int_K Sigma grad u . grad v
        - sum_F int_F ({Sigma grad u}.[v] + [u].{Sigma grad v}) + sum_F int_F eta [u].[v]
    with the jump [v] = v+ n+ + v- n- and the average {q} = (q+ + q-)/2 of
    Arnold et al. (the paper's text swaps the two names).  Boundary faces
    carry no terms (homogeneous Neumann, Eq. monodomain).
  * K_h = chi_m C_m M_h + (dt/2) A_h.
Matrix convention: A[i, j] = A(phi_j, phi_i); DOF index = K * n_p + local.
Off-diagonal face blocks are stored as B and B^T and element-diagonal blocks
are symmetrised, so K_h is bit-symmetric.

Pins (tests/test_oracle_assembly.py): 1^T M 1 = |Omega| and the exact
moments of x, x^2, xy on the unit square; A c_1 = 0 for the constant
function; A(x, x) = |Omega| Sigma_xx for the continuous linear function;
symmetry and positive definiteness of K_h; h^{p+1} convergence of the
manufactured Neumann problem.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import basis, quadrature
from .mesh import geometry, interior_faces, cell_polygon


@dataclass
class Discretisation:
    mesh: object
    p: int
    n_p: int
    geom: object
    faces: object
    sigma: np.ndarray
    eta: np.ndarray            # [nf] penalty per interior face
    M_blocks: np.ndarray       # [nc, n_p, n_p]
    A_diag: np.ndarray         # [nc, n_p, n_p] volume + face self terms
    A_off: np.ndarray          # [nf, n_p, n_p] block (test on K+, trial on K-)
    M: sp.csr_matrix
    A: sp.csr_matrix
    K: sp.csr_matrix
    chi_cm: float
    dt: float

    @property
    def n_dofs(self):
        return self.mesh.n_cells * self.n_p


def element_rule(mesh, k, p):
    """Element quadrature: polygon fan (2D) or polyhedron cone (3D) with n = p + 1."""
    if mesh.dim == 3:
        return quadrature.polyhedron_rule(mesh.vertices, mesh.facets(k), p + 1)
    return quadrature.polygon_rule(cell_polygon(mesh, k), p + 1)


def face_rule(mesh, faces, f, p):
    """Interior face quadrature: Gauss-Legendre on the edge (2D) or the collapsed
    triangle rule (3D), n = p + 1."""
    if mesh.dim == 3:
        V = mesh.vertices
        return quadrature.triangle_rule_3d(V[faces.va[f]], V[faces.vb[f]], V[faces.vc[f]], p + 1)
    return quadrature.segment_rule(mesh.vertices[faces.va[f]], mesh.vertices[faces.vb[f]], p + 1)


def penalty(eta0, p, sigma, diameter, faces):
    """Eq. eta with Sigma_K = lambda_max(Sigma_K)."""
    lam = np.array([np.linalg.eigvalsh(S).max() for S in sigma])
    kp, km = faces.plus, faces.minus
    avg_sigma = 0.5 * (lam[kp] + lam[km])
    harm_h = 2.0 * diameter[kp] * diameter[km] / (diameter[kp] + diameter[km])
    return eta0 * avg_sigma * p * p / harm_h


def assemble(mesh, p, sigma, eta0, chi_cm, dt) -> Discretisation:
    nc = mesh.n_cells
    n_p = len(basis.modes(p, mesh.dim))
    geom = geometry(mesh)
    faces = interior_faces(mesh)
    eta = penalty(eta0, p, sigma, geom.diameter, faces)

    M_blocks = np.zeros((nc, n_p, n_p))
    A_diag = np.zeros((nc, n_p, n_p))
    for k in range(nc):
        x, w = element_rule(mesh, k, p)
        V, G = basis.eval_basis(p, geom.bbox[k], x)
        M_blocks[k] = V.T @ (w[:, None] * V)
        SG = G @ sigma[k]                               # [nq, n_p, dim] = Sigma grad phi
        A_diag[k] = np.einsum("q,qid,qjd->ij", w, G, SG)

    A_off = np.zeros((len(faces.plus), n_p, n_p))
    sgn = {0: 1.0, 1: -1.0}                             # side 0 = K+, side 1 = K-
    for f in range(len(faces.plus)):
        kp, km = faces.plus[f], faces.minus[f]
        n = faces.normal[f]
        x, w = face_rule(mesh, faces, f, p)
        Vs, Fs = [], []
        for k in (kp, km):
            V, G = basis.eval_basis(p, geom.bbox[k], x)
            Vs.append(V)
            Fs.append(G @ (sigma[k] @ n))               # (Sigma grad phi) . n
        blocks = {}
        for a in (0, 1):
            for b in (0, 1):
                sa, sb = sgn[a], sgn[b]
                blk = (-0.5 * sa * Vs[a].T @ (w[:, None] * Fs[b])
                       - 0.5 * sb * Fs[a].T @ (w[:, None] * Vs[b])
                       + eta[f] * sa * sb * Vs[a].T @ (w[:, None] * Vs[b]))
                blocks[(a, b)] = blk
        A_diag[kp] += blocks[(0, 0)]
        A_diag[km] += blocks[(1, 1)]
        A_off[f] = blocks[(0, 1)]

    # bit-symmetric diagonal blocks
    A_diag = 0.5 * (A_diag + np.transpose(A_diag, (0, 2, 1)))
    M_blocks = 0.5 * (M_blocks + np.transpose(M_blocks, (0, 2, 1)))

    M = _blockdiag(M_blocks)
    A = _assemble_sparse(A_diag, A_off, faces, n_p)
    K = (chi_cm * M + (0.5 * dt) * A).tocsr()
    return Discretisation(mesh, p, n_p, geom, faces, sigma, eta, M_blocks,
                          A_diag, A_off, M.tocsr(), A.tocsr(), K.tocsr(), chi_cm, dt)


def _blockdiag(blocks):
    nc, n_p, _ = blocks.shape
    rows = (np.arange(nc)[:, None, None] * n_p + np.arange(n_p)[None, :, None]).repeat(n_p, 2)
    cols = (np.arange(nc)[:, None, None] * n_p + np.arange(n_p)[None, None, :]).repeat(n_p, 1)
    return sp.csr_matrix((blocks.ravel(), (rows.ravel(), cols.ravel())),
                         shape=(nc * n_p, nc * n_p))


def _assemble_sparse(diag, off, faces, n_p):
    nc = diag.shape[0]
    r, c, v = [], [], []
    li = np.arange(n_p)
    I, J = np.meshgrid(li, li, indexing="ij")
    for k in range(nc):
        r.append(k * n_p + I.ravel()); c.append(k * n_p + J.ravel()); v.append(diag[k].ravel())
    for f in range(len(faces.plus)):
        kp, km = faces.plus[f], faces.minus[f]
        r.append(kp * n_p + I.ravel()); c.append(km * n_p + J.ravel()); v.append(off[f].ravel())
        r.append(km * n_p + I.ravel()); c.append(kp * n_p + J.ravel()); v.append(off[f].T.ravel())
    return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))),
                         shape=(nc * n_p, nc * n_p))


def load_vector(disc: Discretisation, g):
    """b_i = int_Omega g phi_i for a vectorised function g(x [nq, dim]) -> [nq]."""
    out = np.zeros((disc.mesh.n_cells, disc.n_p))
    for k in range(disc.mesh.n_cells):
        x, w = element_rule(disc.mesh, k, disc.p)
        V, _ = basis.eval_basis(disc.p, disc.geom.bbox[k], x)
        out[k] = V.T @ (w * g(x))
    return out.ravel()


def l2_project(disc: Discretisation, g):
    """Coefficients of the L2 projection of g onto V_h (element-wise M_K^{-1} b_K)."""
    b = load_vector(disc, g).reshape(disc.mesh.n_cells, disc.n_p)
    return np.stack([np.linalg.solve(disc.M_blocks[k], b[k])
                     for k in range(disc.mesh.n_cells)]).ravel()


def evaluate(disc: Discretisation, coeffs, k, x):
    """Value of the DG function with coefficients ``coeffs`` at points x of element k."""
    V, _ = basis.eval_basis(disc.p, disc.geom.bbox[k], x)
    return V @ coeffs.reshape(disc.mesh.n_cells, disc.n_p)[k]
