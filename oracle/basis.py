"""Modal total-degree basis of P^p on an element (FP64).

The paper fixes a basis of V_h = P^p(T_h) without naming it (Sec. 3, after
Eq. coer).  The reading used throughout: on element K with axis-aligned
bounding box [x0,x1] x [y0,y1] map x -> xi = (2x - x0 - x1)/(x1 - x0) (same
for y -> eta) and take phi_(a,b) = L_a(xi) L_b(eta) for a + b <= p, L_n the
Legendre polynomials (L_n(1) = 1).  Ordering: by total degree d = a + b, and
within a degree by increasing b: (0,0), (1,0), (0,1), (2,0), (1,1), (0,2), ...
In 3D (box [x0,x1] x [y0,y1] x [z0,z1]) phi_(a,b,c) = L_a(xi) L_b(eta) L_c(zeta),
a + b + c <= p, ordered by total degree d, then by increasing c, then by
increasing b: (0,0,0), (1,0,0), (0,1,0), (0,0,1), (2,0,0), (1,1,0), (0,2,0),
(1,0,1), (0,1,1), (0,0,2), ...  (the c = 0 modes of each degree come first, in
the 2D order).

Pins (tests/test_oracle_basis.py, tests/test_oracle_3d.py): Legendre values
against the closed forms for n <= 4 and numpy's legval; derivatives against
central differences of the closed forms; dimensions C(p+2, 2) and C(p+3, 3);
L2-orthogonality on a box against the closed form prod 2/(2n+1).
"""
import numpy as np


def modes(p: int, dim: int = 2):
    """List of exponent tuples (a, b) or (a, b, c) in basis order."""
    out = []
    for d in range(p + 1):
        if dim == 2:
            for b in range(d + 1):
                out.append((d - b, b))
        else:
            for c in range(d + 1):
                for b in range(d - c + 1):
                    out.append((d - b - c, b, c))
    return out


def legendre_table(nmax: int, t):
    """Values L_0..L_nmax and derivatives at points t, by the three-term recurrence
    (n+1) L_{n+1} = (2n+1) t L_n - n L_{n-1}, and L'_{n+1} = L'_{n-1} + (2n+1) L_n."""
    t = np.asarray(t, float)
    L = np.zeros((nmax + 1,) + t.shape)
    D = np.zeros_like(L)
    L[0] = 1.0
    if nmax >= 1:
        L[1] = t
        D[1] = 1.0
    for n in range(1, nmax):
        L[n + 1] = ((2 * n + 1) * t * L[n] - n * L[n - 1]) / (n + 1)
        D[n + 1] = D[n - 1] + (2 * n + 1) * L[n]
    return L, D


def eval_basis(p: int, bbox, x):
    """Basis values [nq, n_p] and physical gradients [nq, n_p, dim] at points x [nq, dim].

    bbox = (x0, x1, y0, y1) in 2D, (x0, x1, y0, y1, z0, z1) in 3D."""
    x = np.asarray(x, float)
    if x.shape[1] == 3:
        return _eval_basis3d(p, bbox, x)
    x0, x1, y0, y1 = bbox
    sx, sy = 2.0 / (x1 - x0), 2.0 / (y1 - y0)
    xi = sx * x[:, 0] - (x0 + x1) / (x1 - x0)
    eta = sy * x[:, 1] - (y0 + y1) / (y1 - y0)
    Lx, Dx = legendre_table(p, xi)
    Ly, Dy = legendre_table(p, eta)
    ms = modes(p)
    V = np.empty((len(x), len(ms)))
    G = np.empty((len(x), len(ms), 2))
    for j, (a, b) in enumerate(ms):
        V[:, j] = Lx[a] * Ly[b]
        G[:, j, 0] = sx * Dx[a] * Ly[b]
        G[:, j, 1] = sy * Lx[a] * Dy[b]
    return V, G


def _eval_basis3d(p, bbox, x):
    L, D, S = [], [], []
    for d in range(3):
        lo, hi = bbox[2 * d], bbox[2 * d + 1]
        s = 2.0 / (hi - lo)
        Ld, Dd = legendre_table(p, s * x[:, d] - (lo + hi) / (hi - lo))
        L.append(Ld); D.append(Dd); S.append(s)
    ms = modes(p, 3)
    V = np.empty((len(x), len(ms)))
    G = np.empty((len(x), len(ms), 3))
    for j, (a, b, c) in enumerate(ms):
        V[:, j] = L[0][a] * L[1][b] * L[2][c]
        G[:, j, 0] = S[0] * D[0][a] * L[1][b] * L[2][c]
        G[:, j, 1] = S[1] * L[0][a] * D[1][b] * L[2][c]
        G[:, j, 2] = S[2] * L[0][a] * L[1][b] * D[2][c]
    return V, G
