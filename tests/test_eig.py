"""The host symmetric eigensolver of the library (setup of the shared local solves):
closed-form spectra, agreement with LAPACK (numpy.linalg.eigh), orthogonality and the
eigen equation, on CPU."""
import numpy as np
import pytest

from test_abi import ensure_built


def check(a, w, Q, tol):
    n = a.shape[0]
    assert np.all(np.diff(w) >= 0)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=tol)
    assert np.linalg.norm(a @ Q - Q * w) <= tol * max(1.0, np.linalg.norm(a))


@pytest.mark.parametrize("n", [1, 2, 3, 17, 120])
def test_second_difference_closed_form(n):
    pd = ensure_built()
    from paper_2512_19536_gb300._native import sym_eig
    a = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, Q = sym_eig(a)
    exact = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.allclose(w, np.sort(exact), atol=1e-12)
    check(a, w, Q, 1e-12)


@pytest.mark.parametrize("n,seed", [(5, 0), (64, 1), (257, 2)])
def test_random_symmetric_against_lapack(n, seed):
    pd = ensure_built()
    from paper_2512_19536_gb300._native import sym_eig
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n))
    a = g + g.T
    w, Q = sym_eig(a)
    assert np.allclose(w, np.linalg.eigvalsh(a), atol=1e-11 * np.abs(w).max())
    check(a, w, Q, 1e-11)


def test_ill_conditioned_spd_and_repeated_eigenvalues():
    pd = ensure_built()
    from paper_2512_19536_gb300._native import sym_eig
    rng = np.random.default_rng(3)
    Q0, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.concatenate([np.logspace(-8, 4, 30), np.full(10, 3.0)])
    a = (Q0 * lam) @ Q0.T
    w, Q = sym_eig(a)
    assert np.allclose(w, np.sort(lam), rtol=0, atol=1e-10 * lam.max())
    check(a, w, Q, 1e-10)
