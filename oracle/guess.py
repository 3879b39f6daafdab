"""Learned PCG initial guess: per-element network, its training, and the safeguard (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper starts each time step's PCG from the previous solution U^k (Sec. 5).
The learned form proposes instead x0 = U^k + s_d * o, where o is the output of
a small network applied element by element, and keeps whichever of {x0, U^k}
has the smaller Euclidean residual |b - K x|_2, so the converged answer is the
PCG's and only the iteration count can change.

Features of element e (n_p coefficients per element, history U^k, U^{k-1}, U^{k-2}):
  own      a_e  = (U^k_e - u_rest e_0) / s_u        (e_0: the constant mode)
           d1_e = (U^k_e - U^{k-1}_e) / s_d
           d2_e = (U^{k-1}_e - U^{k-2}_e) / s_d
  pooled   elementwise mean and elementwise max of [a, d1, d2] over the face
           neighbours N(e) of e (zeros if e has none)
  scalars  h_e / h_ref, dt / dt_ref, |N(e)| / 10    (h_e: cell diameter)
  -> 9 n_p + 3 inputs, in the order [own a, d1, d2 | mean a, d1, d2 | max a, d1, d2 | scalars].
Network: z1 = W1 x + b1, h1 = relu(z1); z2 = W2 h1 + b2, h2 = relu(z2); o = W3 h2 + b3,
with W1 [H, 9 n_p + 3], W2 [H, H], W3 [n_p, H].  Flat parameter order (the
library's too): W1 (row-major), b1, W2, b2, W3, b3.
Target of a training sample (U^{k-2..k+1} of one element): t = (U^{k+1}_e - U^k_e) / s_d;
loss L = mean over samples and outputs of (o - t)^2.
Training: Adam (Kingma & Ba, 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pins (tests/test_oracle_guess.py): features on a hand-built three-cell strip against
values worked out by hand; a network wired to reproduce chosen inputs exactly
(relu(u) - relu(-u) = u) checks the layer order and orientation; central finite
differences check every gradient; Adam's first step is -lr sign(g) and its
first two steps on f = theta^2 / 2 match the update written out by hand; training
drives the loss of a learnable target down; the safeguard picks the smaller residual.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Scales:
    u_rest: float = -67.0
    s_u: float = 50.0
    s_d: float = 1.0
    h_ref: float = 1.0
    dt_ref: float = 0.05

    def as_array(self):
        return np.array([self.u_rest, self.s_u, self.s_d, self.h_ref, self.dt_ref])


def n_inputs(n_p: int) -> int:
    return 9 * n_p + 3


def face_neighbours(n_cells: int, plus, minus):
    """List of face-neighbour ids of every cell (from the interior face list)."""
    nb = [[] for _ in range(n_cells)]
    for a, b in zip(plus, minus):
        nb[int(a)].append(int(b))
        nb[int(b)].append(int(a))
    return [np.array(sorted(x), dtype=np.int64) for x in nb]


def features(nbrs, h, dt, Uk, Uk1, Uk2, n_p: int, sc: Scales):
    """Feature matrix [n_cells, 9 n_p + 3] from the last three solutions."""
    nc = len(nbrs)
    e0 = np.zeros(n_p)
    e0[0] = 1.0
    A = (Uk.reshape(nc, n_p) - sc.u_rest * e0) / sc.s_u
    D1 = (Uk.reshape(nc, n_p) - Uk1.reshape(nc, n_p)) / sc.s_d
    D2 = (Uk1.reshape(nc, n_p) - Uk2.reshape(nc, n_p)) / sc.s_d
    own = np.concatenate([A, D1, D2], axis=1)               # [nc, 3 n_p]
    X = np.zeros((nc, n_inputs(n_p)))
    for e in range(nc):
        X[e, :3 * n_p] = own[e]
        if len(nbrs[e]):
            X[e, 3 * n_p:6 * n_p] = own[nbrs[e]].mean(axis=0)
            X[e, 6 * n_p:9 * n_p] = own[nbrs[e]].max(axis=0)
        X[e, 9 * n_p] = h[e] / sc.h_ref
        X[e, 9 * n_p + 1] = dt / sc.dt_ref
        X[e, 9 * n_p + 2] = len(nbrs[e]) / 10.0
    return X


def targets(Uk, Uk_next, n_p: int, sc: Scales):
    nc = Uk.size // n_p
    return (Uk_next.reshape(nc, n_p) - Uk.reshape(nc, n_p)) / sc.s_d


# ------------------------------------------------------------------ parameters
def shapes(n_p: int, H: int):
    F = n_inputs(n_p)
    return [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (n_p, H)),
            ("b3", (n_p,))]


def unflatten(theta, n_p: int, H: int) -> dict:
    out, k = {}, 0
    for name, shp in shapes(n_p, H):
        size = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + size], dtype=np.float64).reshape(shp)
        k += size
    assert k == len(theta)
    return out


def flatten(P: dict) -> np.ndarray:
    return np.concatenate([P[name].reshape(-1) for name in ("W1", "b1", "W2", "b2", "W3", "b3")])


def n_params(n_p: int, H: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n_p, H))


# ------------------------------------------------------------------ network
def forward(P: dict, X):
    """Outputs o [m, n_p] and the intermediate values needed by backward."""
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ P["W3"].T + P["b3"]
    return o, (X, z1, h1, z2, h2)


def loss(P: dict, X, T) -> float:
    o, _ = forward(P, X)
    return float(np.mean((o - T) ** 2))


def loss_and_grads(P: dict, X, T):
    """L = mean (o - t)^2 and dL/dtheta for every parameter (chain rule by layer)."""
    o, (X, z1, h1, z2, h2) = forward(P, X)
    m, n_out = o.shape
    L = float(np.mean((o - T) ** 2))
    do = 2.0 * (o - T) / (m * n_out)
    g = {"W3": do.T @ h2, "b3": do.sum(axis=0)}
    dh2 = do @ P["W3"]
    dz2 = dh2 * (z2 > 0.0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0.0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, g


@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0


def adam_init(n: int) -> AdamState:
    return AdamState(np.zeros(n), np.zeros(n), 0)


def adam_step(theta, grad, st: AdamState, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the flat parameter vector (returns the new vector)."""
    st.t += 1
    st.m = b1 * st.m + (1.0 - b1) * grad
    st.v = b2 * st.v + (1.0 - b2) * grad * grad
    mhat = st.m / (1.0 - b1 ** st.t)
    vhat = st.v / (1.0 - b2 ** st.t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps)


# ------------------------------------------------------------------ guess + safeguard
def propose(P: dict, X, Uk, sc: Scales):
    """x0 = U^k + s_d o (flattened like U^k)."""
    o, _ = forward(P, X)
    return Uk + sc.s_d * o.reshape(-1)


def safeguard(K, b, x_guess, Uk):
    """Keep the candidate with the smaller |b - K x|_2 (ties keep U^k)."""
    rg = np.linalg.norm(b - K @ x_guess)
    r0 = np.linalg.norm(b - K @ Uk)
    return (x_guess, True) if rg < r0 else (Uk, False)


def subspace_guess(K, b, history, xg=None, m=16):
    """x0 = U^k + V theta over the directions v = xg - U^k (if a proposal is given) and the
    last min(m, len(history) - 1) increments U^{k-j+1} - U^{k-j}; history = [U^k, U^{k-1},
    ...].  theta is the Galerkin projection V^T K V theta = V^T (b - K U^k): the x0 of the
    span with the smallest K-norm error (library least squares for the small system).
    Returns (x0, theta)."""
    Uk = history[0]
    dirs = []
    if xg is not None:
        dirs.append(xg - Uk)
    for j in range(1, min(m, len(history) - 1) + 1):
        dirs.append(history[j - 1] - history[j])
    if not dirs:
        return Uk.copy(), np.zeros(0)
    V = np.stack(dirs, 1)
    H = V.T @ (K @ V)
    theta, *_ = np.linalg.lstsq(0.5 * (H + H.T), V.T @ (b - K @ Uk), rcond=None)
    return Uk + V @ theta, theta
