"""Quadrature rules on segments, triangles, convex polygons, tetrahedra and
star-shaped polyhedra (FP64).

The paper does not fix a quadrature (Sec. 3 only says the forms are integrated
on polytopal elements).  The rules here: Gauss-Legendre on segments; on a
triangle the collapsed (Duffy) tensor rule x(s,t) = A + s(B-A) + s t (C-B)
with Jacobian 2|T| s; on a convex polygon the fan of triangles
(v0, v_k, v_{k+1}).  With n points per direction a triangle rule integrates
polynomials of total degree 2n-2 exactly; n = p + 1 makes the mass, stiffness
and coarse-transfer integrands exact.

In 3D a tetrahedron ABCD takes x(s,t,u) = A + s(B-A) + s t(C-B) + s t u(D-C)
with Jacobian 6|T| s^2 t; a monomial of degree d becomes a polynomial of degree at
most d in each of s, t and u, and the Jacobian's s^2 t is taken as the weight of
Gauss-Jacobi rules in s (weight s^2) and t (weight t), with Gauss-Legendre in u:
n points per direction integrate total degree 2n-1 exactly (n = p + 1: 2p + 1).  A polyhedron given
by outward triangle facets is the cone of tetrahedra (apex, a, b, c) from the
average of its vertices (the jittered hexahedra are star-shaped about it); a
triangle facet in space takes the 2D collapsed rule with Jacobian |(B-A) x (C-A)| s.

Pins (tests/test_oracle_quadrature.py, tests/test_oracle_3d.py): exact monomial
integrals over polygons and polyhedra via the divergence theorem, and
Gauss-Legendre nodes against the closed forms for n = 1..3.
"""
import numpy as np


def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1] (library routine)."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def segment_rule(a, b, n: int):
    """Nodes [n, 2] and weights [n] on the segment from a to b (weights sum to |b-a|)."""
    s, w = gauss_legendre_01(n)
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    pts = a[None, :] + s[:, None] * (b - a)[None, :]
    return pts, w * np.linalg.norm(b - a)


def triangle_rule(A, B, C, n: int):
    """Collapsed tensor rule with n x n points on triangle ABC (any orientation)."""
    s, ws = gauss_legendre_01(n)
    A, B, C = (np.asarray(v, float) for v in (A, B, C))
    twice_area = abs((B[0] - A[0]) * (C[1] - A[1]) - (B[1] - A[1]) * (C[0] - A[0]))
    pts, wts = [], []
    for i in range(n):          # s: from A towards edge BC
        for j in range(n):      # t: along the edge at parameter s
            x = A + s[i] * (B - A) + s[i] * s[j] * (C - B)
            pts.append(x)
            wts.append(ws[i] * ws[j] * s[i] * twice_area)
    return np.asarray(pts), np.asarray(wts)


def polygon_rule(P, n: int):
    """Fan rule on the convex polygon with vertices P [m, 2] (triangles v0, v_k, v_{k+1})."""
    P = np.asarray(P, float)
    pts, wts = [], []
    for k in range(1, len(P) - 1):
        x, w = triangle_rule(P[0], P[k], P[k + 1], n)
        pts.append(x)
        wts.append(w)
    return np.concatenate(pts), np.concatenate(wts)


def triangle_rule_3d(A, B, C, n: int):
    """Collapsed rule with n x n points on a triangle ABC in space."""
    s, ws = gauss_legendre_01(n)
    A, B, C = (np.asarray(v, float) for v in (A, B, C))
    twice_area = np.linalg.norm(np.cross(B - A, C - A))
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            pts.append(A + s[i] * (B - A) + s[i] * s[j] * (C - B))
            wts.append(ws[i] * ws[j] * s[i] * twice_area)
    return np.asarray(pts), np.asarray(wts)


def gauss_jacobi_01(n: int, power: int):
    """n-point Gauss rule on [0, 1] for the weight s**power (library routine)."""
    from scipy.special import roots_jacobi
    x, w = roots_jacobi(n, 0.0, float(power))       # weight (1 + x)^power on [-1, 1]
    return 0.5 * (x + 1.0), w / 2.0 ** (power + 1)


def tet_rule(A, B, C, D, n: int):
    """Collapsed rule on tetrahedron ABCD: n Gauss-Jacobi points in s (weight s^2) and
    t (weight t), n Gauss-Legendre points in u."""
    s, ws = gauss_jacobi_01(n, 2)
    t, wt = gauss_jacobi_01(n, 1)
    u, wu = gauss_legendre_01(n)
    A, B, C, D = (np.asarray(v, float) for v in (A, B, C, D))
    six_vol = abs(np.linalg.det(np.stack([B - A, C - A, D - A])))
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                pts.append(A + s[i] * (B - A) + s[i] * t[j] * (C - B)
                           + s[i] * t[j] * u[k] * (D - C))
                wts.append(ws[i] * wt[j] * wu[k] * six_vol)
    return np.asarray(pts), np.asarray(wts)


def polyhedron_rule(vertices, facets, n: int):
    """Cone rule on a polyhedron with outward triangle facets [m, 3] (vertex ids)."""
    V = np.asarray(vertices, float)
    apex = V[np.unique(facets)].mean(axis=0)
    pts, wts = [], []
    for a, b, c in facets:
        x, w = tet_rule(apex, V[a], V[b], V[c], n)
        pts.append(x)
        wts.append(w)
    return np.concatenate(pts), np.concatenate(wts)
