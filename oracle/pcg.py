"""Preconditioned conjugate gradients (FP64), standard and flexible.

Sec. 4 and Sec. 5: the system of Eq. fully-discrete-1 is solved by PCG with
B_ad^{-1} (Eq. prec) as preconditioner, stopping when the Euclidean norm of
the relative residual |r_k| / |b| falls below a tolerance.  The iteration is
the textbook one (Saad, Iterative Methods, Alg. 9.1):
    r0 = b - K x0, z0 = B r0, p0 = z0;
    alpha = (r, z) / (K p, p); x += alpha p; r -= alpha K p;
    z = B r; beta = (r_new, z_new) / (r, z); p = z + beta p.
The flexible variant (for an inexact, e.g. reduced-precision, preconditioner)
replaces beta by (z_new, r_new - r) / (r, z).  The recorded alpha_k, beta_k
define the Lanczos tridiagonal used for condition-number estimates (Sec. 5).
If b = 0 the solution is x = 0 and no iteration is taken.

Pins (tests/test_oracle_pcg.py): agreement with a dense direct solve on small
SPD systems; the identity preconditioner reproduces unpreconditioned CG; an
exact inverse as preconditioner converges in one iteration; in exact
arithmetic CG terminates in at most (number of distinct eigenvalues) steps.
pcg_pipelined (the one-reduction rearrangement of the same iteration): its
coefficients and iterates equal the textbook PCG's up to rounding, it reaches the
direct solution, and its recurrence residual stays within rounding of b - K x.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    relres: float
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)


def pcg(K, b, x0=None, prec=None, rtol=1e-8, maxit=10000, flexible=False) -> PCGResult:
    apply_K = K if callable(K) else (lambda v: K @ v)
    apply_B = prec if prec is not None else (lambda v: v.copy())
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return PCGResult(np.zeros_like(b), 0, True, 0.0)
    r = b - apply_K(x)
    rel = np.linalg.norm(r) / bnorm
    if rel <= rtol:
        return PCGResult(x, 0, True, rel)
    z = apply_B(r)
    p = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for k in range(1, maxit + 1):
        q = apply_K(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        alphas.append(alpha)
        rel = np.linalg.norm(r_new) / bnorm
        if rel <= rtol:
            return PCGResult(x, k, True, rel, alphas, betas)
        z = apply_B(r_new)
        rz_new = r_new @ z
        beta = (z @ (r_new - r)) / rz if flexible else rz_new / rz
        betas.append(beta)
        p = z + beta * p
        r, rz = r_new, rz_new
    return PCGResult(x, maxit, False, rel, alphas, betas)


def lanczos_extremes(alphas, betas):
    """Extreme eigenvalues of the Lanczos tridiagonal T built from the PCG
    coefficients: T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1},
    T_{k,k+1} = sqrt(beta_k)/alpha_k (Saad, Sec. 6.7.3)."""
    m = len(alphas)
    if m == 0:
        return 1.0, 1.0
    d = np.empty(m)
    e = np.empty(max(m - 1, 0))
    for k in range(m):
        d[k] = 1.0 / alphas[k] + (betas[k - 1] / alphas[k - 1] if k > 0 else 0.0)
        if k < m - 1:
            e[k] = np.sqrt(betas[k]) / alphas[k]
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


def pcg_pipelined(K, b, x0=None, prec=None, rtol=1e-8, maxit=10000) -> PCGResult:
    """Pipelined PCG (Ghysels and Vanroose, "Hiding global synchronization latency in the
    preconditioned conjugate gradient algorithm", Parallel Computing 40, 2014): the same
    Krylov iterates as the textbook PCG in exact arithmetic, rearranged so that an
    iteration needs one global reduction (gamma = (r, u) and delta = (w, u) together),
    which a GPU form overlaps with the next preconditioner application and matvec.
    Auxiliary recurrences: u = B r, w = K u, m = B w, n = K m; the search direction p
    and its images s = K p, q = B s, z = K q follow the same beta.  Here the stopping
    test reads |r| directly (a GPU form would fuse it into the next reduction).  Records
    alpha_k, beta_k with the textbook meaning (the Lanczos tridiagonal is the same).
    """
    apply_K = K if callable(K) else (lambda v: K @ v)
    apply_B = prec if prec is not None else (lambda v: v.copy())
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return PCGResult(np.zeros_like(b), 0, True, 0.0)
    r = b - apply_K(x)
    rel = np.linalg.norm(r) / bnorm
    if rel <= rtol:
        return PCGResult(x, 0, True, rel)
    u = apply_B(r)
    w = apply_K(u)
    p, s, q, z = (np.zeros_like(b) for _ in range(4))
    alphas, betas = [], []
    gamma_old = alpha_old = None
    for k in range(1, maxit + 1):
        gamma, delta = r @ u, w @ u           # the iteration's one reduction
        m = apply_B(w)
        n = apply_K(m)
        if k == 1:
            beta, alpha = 0.0, gamma / delta
        else:
            beta = gamma / gamma_old
            alpha = gamma / (delta - beta * gamma / alpha_old)
            betas.append(beta)
        z = n + beta * z
        q = m + beta * q
        s = w + beta * s
        p = u + beta * p
        x = x + alpha * p
        r = r - alpha * s
        u = u - alpha * q
        w = w - alpha * z
        alphas.append(alpha)
        rel = np.linalg.norm(r) / bnorm
        if rel <= rtol:
            return PCGResult(x, k, True, rel, alphas, betas)
        gamma_old, alpha_old = gamma, alpha
    return PCGResult(x, maxit, False, rel, alphas, betas)
