"""Pins of oracle.pcg (no GPU)."""
import numpy as np

from oracle.pcg import pcg, lanczos_extremes


def spd_with_spectrum(ev, seed=0):
    n = len(ev)
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return (Q * ev) @ Q.T


def test_matches_dense_solve():
    A = spd_with_spectrum(np.linspace(1, 100, 60))
    b = np.random.default_rng(1).standard_normal(60)
    r = pcg(A, b, rtol=1e-13)
    assert r.converged
    assert np.allclose(r.x, np.linalg.solve(A, b), rtol=1e-9)


def test_distinct_eigenvalue_termination():
    # CG terminates in at most m steps for m distinct eigenvalues (exact arithmetic).
    ev = np.repeat([1.0, 2.0, 5.0, 9.0, 30.0], 12)
    A = spd_with_spectrum(ev, 3)
    b = np.random.default_rng(4).standard_normal(len(ev))
    assert pcg(A, b, rtol=1e-10).iterations <= 5


def test_exact_inverse_preconditioner_one_iteration():
    A = spd_with_spectrum(np.geomspace(1, 1e4, 40))
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(5).standard_normal(40)
    assert pcg(A, b, prec=lambda v: Ainv @ v, rtol=1e-10).iterations == 1
    assert pcg(A, b, prec=lambda v: Ainv @ v, rtol=1e-10, flexible=True).iterations == 1


def test_lanczos_extremes_recover_spectrum():
    ev = np.linspace(0.5, 40.0, 80)
    A = spd_with_spectrum(ev, 6)
    b = np.random.default_rng(7).standard_normal(80)
    r = pcg(A, b, rtol=1e-12)
    lo, hi = lanczos_extremes(r.alphas, r.betas)
    assert np.isclose(lo, 0.5, rtol=1e-6) and np.isclose(hi, 40.0, rtol=1e-6)


def test_zero_rhs_and_initial_guess():
    A = spd_with_spectrum(np.linspace(1, 10, 10))
    r = pcg(A, np.zeros(10))
    assert r.iterations == 0 and np.all(r.x == 0)
    b = np.random.default_rng(8).standard_normal(10)
    x = np.linalg.solve(A, b)
    assert pcg(A, b, x0=x, rtol=1e-8).iterations == 0


def test_flexible_equals_standard_with_fixed_spd_preconditioner():
    A = spd_with_spectrum(np.geomspace(1, 1e3, 50), 9)
    D = np.diag(1.0 / np.diag(A))
    b = np.random.default_rng(10).standard_normal(50)
    r1 = pcg(A, b, prec=lambda v: D @ v, rtol=1e-10)
    r2 = pcg(A, b, prec=lambda v: D @ v, rtol=1e-10, flexible=True)
    assert abs(r1.iterations - r2.iterations) <= 1
    assert np.allclose(r1.x, r2.x, rtol=1e-7)


# ---- pipelined PCG: the same iteration with one reduction per step

def test_pipelined_matches_textbook_coefficients_and_iterates():
    # exact arithmetic gives identical alpha_k, beta_k and x_k; rounding separates them
    # slowly on a well-conditioned system, so the first iterations agree closely
    from oracle.pcg import pcg_pipelined
    A = spd_with_spectrum(np.linspace(1, 50, 40), 5)
    Dinv = 1.0 / np.diag(A)
    b = np.random.default_rng(6).standard_normal(40)
    prec = lambda v: Dinv * v
    ref = pcg(A, b, prec=prec, rtol=1e-300, maxit=10)
    got = pcg_pipelined(A, b, prec=prec, rtol=1e-300, maxit=10)
    assert np.allclose(got.alphas, ref.alphas, rtol=1e-10)
    # at maxit the textbook loop has already formed the next beta; the pipelined one
    # forms it at the start of the following iteration
    assert np.allclose(got.betas, ref.betas[:len(got.betas)], rtol=1e-10) and len(got.betas) == 9
    assert np.allclose(got.x, ref.x, rtol=1e-9, atol=1e-12)
    # the recurrence residual (the stopping test reads it) is the true residual: the
    # coefficients do not depend on r, so only this catches an error in its recurrence
    true_rel = np.linalg.norm(b - A @ got.x) / np.linalg.norm(b)
    assert abs(got.relres - true_rel) <= 1e-12 and abs(got.relres - ref.relres) <= 1e-12


def test_pipelined_reaches_direct_solution_with_schwarz(square16):
    # on the 16 x 16 P2 case with the two-level preconditioner: the direct solution,
    # iteration counts within 2 of the textbook PCG, recurrence residual near the true one
    import scipy.sparse.linalg as spla
    from oracle import schwarz
    from oracle.pcg import pcg_pipelined
    w, d = square16
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    b = np.random.default_rng(7).standard_normal(d.n_dofs)
    got = pcg_pipelined(d.K, b, prec=S.apply, rtol=1e-10)
    ref = pcg(d.K, b, prec=S.apply, rtol=1e-10)
    x = spla.spsolve(d.K.tocsc(), b)
    assert got.converged and abs(got.iterations - ref.iterations) <= 2
    assert np.linalg.norm(got.x - x) <= 1e-8 * np.linalg.norm(x)
    true_rel = np.linalg.norm(b - d.K @ got.x) / np.linalg.norm(b)
    assert true_rel <= 1e-9

