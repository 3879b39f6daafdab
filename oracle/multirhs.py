"""Local solves shared by simulations that differ only in a scalar conductivity (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Simulations on one mesh, partition and degree whose conductivity is a scalar multiple of
the identity, Sigma_K = sigma I, share the structure of their local matrices.  The
penalty of Eq. eta uses lambda_max(Sigma_K) = sigma and every term of the SIP form
(Eq. coer) is linear in Sigma, so A(sigma) = sigma A(1) and, with K = chi_cm M + dt/2 A
(Eq. fully-discrete-1),
    K_i(sigma) = chi_cm M_i + c A_i,   c = dt sigma / 2,   A_i = A_i(1).
With M_i = L_i L_i^T (block diagonal: one n_p x n_p Cholesky factor per element) and the
symmetric eigendecomposition L_i^{-1} A_i L_i^{-T} = Q_i diag(lam_i) Q_i^T,
    K_i(sigma)^{-1} = L_i^{-T} Q_i diag(1 / (chi_cm + c lam_i)) Q_i^T L_i^{-1},
so one factorisation serves every sigma, and R right-hand sides of R simulations are two
products with Q_i (n_i x n_i times n_i x R) per subdomain.

Pins (tests/test_oracle_multirhs.py): A assembled with sigma I equals sigma times A
assembled with I; the eigen form equals a dense solve with K_i(sigma) for several sigma;
the whole two-level preconditioner built with it equals oracle.schwarz's on the
assembly with that sigma.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class SharedLocal:
    sub_dofs: list        # per subdomain: global DOF indices (ascending, cell-major)
    L: list               # per subdomain: [n_cells_i, n_p, n_p] lower Cholesky factors of M_K
    Q: list               # per subdomain: n_i x n_i orthogonal
    lam: list             # per subdomain: eigenvalues of L^{-1} A_i L^{-T}
    n_p: int


def subdomain_dofs(subdomain_of_cell, n_p):
    sub = np.asarray(subdomain_of_cell)
    out = []
    for s in range(int(sub.max()) + 1):
        cells = np.flatnonzero(sub == s)
        out.append((cells[:, None] * n_p + np.arange(n_p)[None, :]).ravel())
    return out


def build(M, A1, sub_dofs, n_p) -> SharedLocal:
    """Factors of the shared local solves from the mass matrix M and the sigma = 1
    stiffness A1 (sparse, whole mesh) for the given subdomain DOF sets."""
    Ls, Qs, lams = [], [], []
    M = M.tocsr()
    A1 = A1.tocsr()
    for dofs in sub_dofs:
        Mi = M[dofs][:, dofs].toarray()
        Ai = A1[dofs][:, dofs].toarray()
        nc = len(dofs) // n_p
        L = np.stack([np.linalg.cholesky(Mi[k * n_p:(k + 1) * n_p, k * n_p:(k + 1) * n_p])
                      for k in range(nc)])
        Lfull = sla.block_diag(*L)
        Linv = sla.solve_triangular(Lfull, np.eye(len(dofs)), lower=True)
        C = Linv @ Ai @ Linv.T
        lam, Q = np.linalg.eigh(0.5 * (C + C.T))
        Ls.append(L)
        Qs.append(Q)
        lams.append(lam)
    return SharedLocal(sub_dofs, Ls, Qs, lams, n_p)


def apply_local(S: SharedLocal, r, sigma, chi_cm, dt):
    """z = sum_i R_i^T K_i(sigma)^{-1} R_i r through the eigen form."""
    z = np.zeros_like(r)
    c = 0.5 * dt * sigma
    for dofs, L, Q, lam in zip(S.sub_dofs, S.L, S.Q, S.lam):
        Lfull = sla.block_diag(*L)
        x = sla.solve_triangular(Lfull, r[dofs], lower=True)            # L^{-1} r
        y = (Q.T @ x) / (chi_cm + c * lam)
        z[dofs] = sla.solve_triangular(Lfull.T, Q @ y, lower=False)     # L^{-T} Q y
    return z
