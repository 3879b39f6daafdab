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
