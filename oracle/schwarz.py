"""Two-level non-overlapping additive Schwarz preconditioner (FP64).

Sec. 4 of the paper:
  * subdomains Omega_i (i = 1..N) are unions of fine elements; R_i^T extends
    a subdomain vector by zero and R_i restricts (a row selection);
  * the coarse space V_0 = P^q on the agglomerates of T_H (every fine element
    lies in exactly one agglomerate); R_0^T is the L2 projection V_0 -> V_h,
    which, since V_0 is contained in V_h, is exact: per fine element K in
    agglomerate J, R_0^T restricted to K is T_K = M_K^{-1} int_K phi_K psi_J^T;
  * R_0 is read as the Euclidean transpose of the matrix of R_0^T (so that
    K_0 = R_0 K_h R_0^T is the Galerkin matrix and B_ad is symmetric);
  * K_i = R_i K_h R_i^T for i = 0..N and, Eq. prec,
        B_ad^{-1} = sum_{i=0}^{N} R_i^T K_i^{-1} R_i.
The coarse basis psi_J is the modal Legendre basis of degree q on the
agglomerate's bounding box (the same construction as the fine basis).
Local and coarse solves use a dense Cholesky factorisation (library routine).

Pins (tests/test_oracle_schwarz.py): B_ad symmetric; one subdomain without
coarse space gives B_ad = K^{-1} (PCG converges in one iteration); one
subdomain with coarse space gives eigenvalues {1, 2} of B_ad K (at most two
iterations); R_0^T reproduces coarse polynomials exactly; element-block
Jacobi (T_S = T_h, no coarse) equals the textbook block-Jacobi operator.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import basis
from .assembly import element_rule


@dataclass
class Schwarz:
    sub_dofs: list            # per subdomain: global DOF indices (ascending)
    sub_chol: list            # per subdomain: cho_factor of K_i
    R0T: sp.csr_matrix        # [N, n0] or None
    K0: np.ndarray            # [n0, n0] or None
    K0_chol: object

    def apply(self, r):
        """z = B_ad^{-1} r (Eq. prec)."""
        z = np.zeros_like(r)
        for dofs, ch in zip(self.sub_dofs, self.sub_chol):
            z[dofs] += sla.cho_solve(ch, r[dofs])
        if self.R0T is not None:
            r0 = self.R0T.T @ r
            z += self.R0T @ sla.cho_solve(self.K0_chol, r0)
        return z


def agglomerate_bbox(mesh, cells):
    V = mesh.vertices[np.concatenate([mesh.cell(k) for k in cells])]
    lo, hi = V.min(0), V.max(0)
    return tuple(v for d in range(mesh.dim) for v in (lo[d], hi[d]))


def coarse_prolongation(disc, coarse, q):
    """Matrix of R_0^T: block (K, J(K)) = T_K = M_K^{-1} int_K phi_K psi_J^T."""
    mesh, p, n_p = disc.mesh, disc.p, disc.n_p
    n_q = len(basis.modes(q, mesh.dim))
    n_agg = int(coarse.max()) + 1
    boxes = [agglomerate_bbox(mesh, np.flatnonzero(coarse == J)) for J in range(n_agg)]
    rows, cols, vals = [], [], []
    for k in range(mesh.n_cells):
        J = int(coarse[k])
        x, w = element_rule(mesh, k, p)
        V, _ = basis.eval_basis(p, disc.geom.bbox[k], x)
        Psi, _ = basis.eval_basis(q, boxes[J], x)
        T = np.linalg.solve(disc.M_blocks[k], V.T @ (w[:, None] * Psi))   # [n_p, n_q]
        I, Jj = np.meshgrid(np.arange(n_p), np.arange(n_q), indexing="ij")
        rows.append(k * n_p + I.ravel())
        cols.append(J * n_q + Jj.ravel())
        vals.append(T.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(disc.n_dofs, n_agg * n_q)), boxes


def build(disc, subdomain, coarse=None, q=1) -> Schwarz:
    n_p = disc.n_p
    K = disc.K.tocsr()
    sub_dofs, sub_chol = [], []
    for i in range(int(subdomain.max()) + 1):
        cells = np.flatnonzero(subdomain == i)
        dofs = (cells[:, None] * n_p + np.arange(n_p)[None, :]).ravel()
        Ki = K[dofs][:, dofs].toarray()
        sub_dofs.append(dofs)
        sub_chol.append(sla.cho_factor(Ki, lower=True))
    R0T = K0 = K0_chol = None
    if coarse is not None:
        R0T, _ = coarse_prolongation(disc, coarse, q)
        K0 = (R0T.T @ (K @ R0T)).toarray()
        K0 = 0.5 * (K0 + K0.T)
        K0_chol = sla.cho_factor(K0, lower=True)
    return Schwarz(sub_dofs, sub_chol, R0T, K0, K0_chol)
