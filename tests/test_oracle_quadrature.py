"""Pins of oracle.quadrature against closed forms (no GPU)."""
from math import comb

import numpy as np
import pytest

from oracle import quadrature
from synth.meshes import voronoi_square


def test_gauss_legendre_closed_forms():
    # n = 1, 2, 3 nodes/weights on [0, 1] from the closed forms of L_1, L_2, L_3.
    x, w = quadrature.gauss_legendre_01(1)
    assert np.allclose(x, [0.5]) and np.allclose(w, [1.0])
    x, w = quadrature.gauss_legendre_01(2)
    assert np.allclose(np.sort(x), [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], atol=1e-15)
    x, w = quadrature.gauss_legendre_01(3)
    o = np.argsort(x)
    assert np.allclose(x[o], [0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w[o], [5 / 18, 8 / 18, 5 / 18], atol=1e-15)


def _segment_monomial(P, Q, m, n):
    """int_0^1 x(t)^m y(t)^n dt on x(t) = P + t (Q - P), by binomial expansion."""
    px, py = P
    dx, dy = Q[0] - P[0], Q[1] - P[1]
    s = 0.0
    for i in range(m + 1):
        for j in range(n + 1):
            s += comb(m, i) * comb(n, j) * px ** (m - i) * dx ** i * py ** (n - j) * dy ** j / (i + j + 1)
    return s


def polygon_monomial_exact(P, a, b):
    """int_K x^a y^b = 1/(a+1) oint x^{a+1} y^b n_x ds (divergence theorem), CCW polygon."""
    total = 0.0
    for k in range(len(P)):
        A, B = P[k], P[(k + 1) % len(P)]
        total += (B[1] - A[1]) * _segment_monomial(A, B, a + 1, b)
    return total / (a + 1)


POLYS = [
    np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]]),
    np.array([[0.3, 0.1], [0.9, 0.25], [1.1, 0.7], [0.6, 1.2], [0.1, 0.8], [0.05, 0.4]]),
]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_polygon_rule_exact_to_degree_2p(p):
    mesh = voronoi_square(16, 3)
    polys = POLYS + [mesh.vertices[mesh.cell(k)] for k in range(3)]
    for P in polys:
        x, w = quadrature.polygon_rule(P, p + 1)
        for a in range(2 * p + 1):
            for b in range(2 * p + 1 - a):
                exact = polygon_monomial_exact(P, a, b)
                got = np.sum(w * x[:, 0] ** a * x[:, 1] ** b)
                assert abs(got - exact) <= 1e-13 * max(1.0, abs(exact)), (p, a, b)


def test_polygon_rule_not_exact_beyond_its_degree():
    # Sensitivity check: with n points the rule is not exact at total degree 2n.
    P = POLYS[1]
    x, w = quadrature.polygon_rule(P, 2)
    got = np.sum(w * x[:, 0] ** 4)
    assert abs(got - polygon_monomial_exact(P, 4, 0)) > 1e-8


def test_segment_rule_length_and_moments():
    x, w = quadrature.segment_rule([0.2, 0.1], [0.7, 0.9], 3)
    L = np.hypot(0.5, 0.8)
    assert np.isclose(w.sum(), L, atol=1e-15)
    # int over the segment of x ds = L * (0.2 + 0.7)/2
    assert np.isclose((w * x[:, 0]).sum(), L * 0.45, atol=1e-15)
