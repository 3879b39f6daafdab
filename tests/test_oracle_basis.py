"""Pins of oracle.basis against closed-form Legendre polynomials (no GPU)."""
import numpy as np

from oracle import basis

T = np.linspace(-1.0, 1.0, 11)
CLOSED = [
    (lambda t: np.ones_like(t), lambda t: np.zeros_like(t)),
    (lambda t: t, lambda t: np.ones_like(t)),
    (lambda t: 0.5 * (3 * t ** 2 - 1), lambda t: 3 * t),
    (lambda t: 0.5 * (5 * t ** 3 - 3 * t), lambda t: 0.5 * (15 * t ** 2 - 3)),
    (lambda t: (35 * t ** 4 - 30 * t ** 2 + 3) / 8, lambda t: (140 * t ** 3 - 60 * t) / 8),
]


def test_legendre_values_and_derivatives():
    L, D = basis.legendre_table(4, T)
    for n, (f, df) in enumerate(CLOSED):
        assert np.allclose(L[n], f(T), atol=1e-14)
        assert np.allclose(D[n], df(T), atol=1e-13)


def test_legendre_matches_numpy_legval_high_degree():
    L, _ = basis.legendre_table(8, T)
    for n in range(9):
        c = np.zeros(n + 1); c[n] = 1.0
        assert np.allclose(L[n], np.polynomial.legendre.legval(T, c), atol=1e-13)


def test_mode_count_and_order():
    for p in range(6):
        assert len(basis.modes(p)) == (p + 1) * (p + 2) // 2
    assert basis.modes(2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]


def test_eval_basis_affine_map_and_gradient():
    bbox = (0.2, 0.6, -0.1, 0.4)
    x = np.array([[0.2, -0.1], [0.6, 0.4], [0.4, 0.15], [0.31, 0.02]])
    V, G = basis.eval_basis(3, bbox, x)
    # corners map to xi, eta = -1, +1; centre to 0
    assert np.allclose(V[0], [(-1) ** (a + b) for a, b in basis.modes(3)])
    assert np.allclose(V[1], 1.0)
    # gradient vs central differences of the values
    h = 1e-6
    for d in range(2):
        e = np.zeros(2); e[d] = h
        Vp, _ = basis.eval_basis(3, bbox, x + e)
        Vm, _ = basis.eval_basis(3, bbox, x - e)
        assert np.allclose(G[:, :, d], (Vp - Vm) / (2 * h), atol=1e-7)
