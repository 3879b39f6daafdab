"""The library's Lanczos extreme-eigenvalue estimate (host function, no GPU) against the
oracle's, both fed with the oracle's PCG coefficients; and the eigenvalues of a known
spectrum recovered through it."""
import numpy as np

from test_abi import ensure_built
from oracle.pcg import pcg, lanczos_extremes as oracle_extremes


def test_lanczos_extremes_match_oracle_and_spectrum():
    ensure_built()
    from paper_2512_19536_gb300._native import lanczos_extremes
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.linspace(0.5, 40.0, 60)
    A = (Q * lam) @ Q.T
    b = rng.standard_normal(60)
    r = pcg(A, b, rtol=1e-14, maxit=200)
    lo, hi = lanczos_extremes(r.alphas, r.betas)
    olo, ohi = oracle_extremes(r.alphas, r.betas)
    assert abs(lo - olo) <= 1e-10 * abs(olo) and abs(hi - ohi) <= 1e-10 * abs(ohi)
    assert abs(lo - 0.5) <= 1e-6 and abs(hi - 40.0) <= 1e-6


def test_lanczos_extremes_long_traces_match_tridiagonal_eigensolver():
    # traces of tens of thousands of iterations (unpreconditioned CG at p = 4): the
    # library's extremes against LAPACK's tridiagonal bisection on the same T
    import time
    import scipy.linalg as sla
    ensure_built()
    from paper_2512_19536_gb300._native import lanczos_extremes
    rng = np.random.default_rng(12)
    m = 40000
    al = rng.uniform(1e-6, 1.0, m)
    be = rng.uniform(0.0, 0.99, m - 1)
    d = 1.0 / al + np.concatenate([[0.0], be / al[:-1]])
    e = np.sqrt(be) / al[:-1]
    t0 = time.time()
    lo, hi = lanczos_extremes(al, be)
    assert time.time() - t0 < 5.0
    ref_lo = sla.eigvalsh_tridiagonal(d, e, select="i", select_range=(0, 0))[0]
    ref_hi = sla.eigvalsh_tridiagonal(d, e, select="i", select_range=(m - 1, m - 1))[0]
    assert abs(hi - ref_hi) <= 1e-12 * abs(ref_hi)
    assert abs(lo - ref_lo) <= 1e-12 * abs(ref_hi)        # absolute accuracy ~ eps |T|


def test_lanczos_extremes_closed_forms():
    # one step: T = [1/alpha_0]; zero betas: T diagonal with T_kk = 1/alpha_k; a
    # Toeplitz T (alpha_k = 1/2 for k >= 1 after alpha_0 = 1/2, beta_k = 1/4 gives
    # T_kk = 2 + 1/2 for k >= 1 and T_00 = 2): checked against numpy's dense solver
    ensure_built()
    from paper_2512_19536_gb300._native import lanczos_extremes
    lo, hi = lanczos_extremes(np.array([0.25]), np.array([]))
    assert lo == hi == 4.0
    al = np.array([0.5, 0.125, 1.0, 0.2])
    lo, hi = lanczos_extremes(al, np.zeros(3))
    assert abs(lo - 1.0) <= 1e-15 and abs(hi - 8.0) <= 8e-15
    m = 200
    al = np.full(m, 0.5)
    be = np.full(m - 1, 0.25)
    d = 1.0 / al + np.concatenate([[0.0], be / al[:-1]])
    e = np.sqrt(be) / al[:-1]
    ev = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))
    lo, hi = lanczos_extremes(al, be)
    assert abs(lo - ev[0]) <= 1e-13 * ev[-1] and abs(hi - ev[-1]) <= 1e-13 * ev[-1]


def test_lanczos_extremes_rejects_bad_coefficients():
    ensure_built()
    import paper_2512_19536_gb300 as pd
    from paper_2512_19536_gb300._native import lanczos_extremes
    for al, be in ((np.array([1.0, -0.5]), np.array([0.1])), (np.array([1.0, 1.0]), np.array([-0.1])),
                   (np.array([np.inf, 1.0]), np.array([0.1]))):
        try:
            lanczos_extremes(al, be)
        except pd.PolyDGError as err:
            assert err.status == pd.POLYDG_EINVAL
        else:
            raise AssertionError("invalid coefficients accepted")
