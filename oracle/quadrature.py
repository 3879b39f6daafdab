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
n points per direction integrate total degree 2n-1 exactly (n = p + 1: 2p + 1).  For
n = 3 (degree 5, P2) a fully symmetric rule of 14 points reaches the same degree with about
half the 27 points of the collapsed one, and the tetrahedra take it instead
(tet_symmetric_deg5): the element quadrature nodes carry the ionic state, so their number
sets the cost of the ionic update.  A polyhedron given
by outward triangle facets is the cone of tetrahedra (apex, a, b, c) from the
average of its vertices (the jittered hexahedra are star-shaped about it); a
triangle facet in space takes the 2D collapsed rule with Jacobian |(B-A) x (C-A)| s.

Pins (tests/test_oracle_quadrature.py, tests/test_oracle_3d.py): exact monomial
integrals over polygons and polyhedra via the divergence theorem, barycentric monomial
integrals over tetrahedra (every monomial of degree <= 5 for the symmetric rule),
and Gauss-Legendre nodes against the closed forms for n = 1..3.
"""
import functools

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


@functools.lru_cache(maxsize=None)
def tet_symmetric_deg5():
    """Fully symmetric 14-point rule on a tetrahedron, exact for polynomials of degree 5:
    barycentric points [14, 4] and weights summing to 1 (multiply by the volume).

    Orbits under the vertex permutations, in this order: (a, a, a, 1 - 3a) and then
    (b, b, b, 1 - 3b), the odd coordinate at vertex 0, 1, 2, 3; (c, c, 1/2 - c, 1/2 - c),
    the two c's at vertex pairs (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).  A rule that is
    invariant under the permutations integrates a polynomial exactly when it integrates its
    average over the permutations exactly, so exactness to degree 5 reduces to the
    invariant polynomials of degree <= 5.  With P_k = sum_i l_i^k and l_1 + ... + l_4 = 1
    these are spanned by 1, P_2, P_3, P_4, P_2^2 and P_2 P_3 (P_5 and the other products
    are combinations of them by Newton's identities), whose means over the tetrahedron are
    1, 2/5, 1/5, 4/35, 6/35 and 13/140 (the mean of l^alpha is 3! alpha! / (|alpha| + 3)!).
    Six equations in (a, b, c) and the three orbit weights, solved by a library root
    finder from a nearby start."""
    from scipy.optimize import root
    import itertools
    pairs = list(itertools.combinations(range(4), 2))

    def points(a, b, c):
        L = []
        for o in (a, b):
            for i in range(4):
                l = np.full(4, o)
                l[i] = 1.0 - 3.0 * o
                L.append(l)
        for i, j in pairs:
            l = np.full(4, 0.5 - c)
            l[i] = l[j] = c
            L.append(l)
        return np.asarray(L)

    def weights(wa, wb, wc):
        return np.concatenate([np.full(4, wa), np.full(4, wb), np.full(6, wc)])

    mean = np.array([1.0, 2.0 / 5.0, 1.0 / 5.0, 4.0 / 35.0, 6.0 / 35.0, 13.0 / 140.0])

    def residual(v):
        L = points(*v[:3])
        P2, P3, P4 = (L ** 2).sum(1), (L ** 3).sum(1), (L ** 4).sum(1)
        G = np.stack([np.ones(len(L)), P2, P3, P4, P2 * P2, P2 * P3])
        return G @ weights(*v[3:]) - mean

    sol = root(residual, [0.09, 0.31, 0.045, 0.07, 0.11, 0.04], method="hybr", tol=1e-14)
    assert np.abs(residual(sol.x)).max() < 1e-14
    L, w = points(*sol.x[:3]), weights(*sol.x[3:])
    L.flags.writeable = False
    w.flags.writeable = False
    return L, w


def tet_rule(A, B, C, D, n: int):
    """Rule on tetrahedron ABCD exact to degree 2n - 1: for n = 3 the symmetric 14-point
    rule; otherwise the collapsed rule, n Gauss-Jacobi points in s (weight s^2) and t
    (weight t), n Gauss-Legendre points in u."""
    if n == 3:
        L, w = tet_symmetric_deg5()
        V = np.stack([np.asarray(v, float) for v in (A, B, C, D)])
        six_vol = abs(np.linalg.det(V[1:] - V[0]))
        return L @ V, w * (six_vol / 6.0)
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
