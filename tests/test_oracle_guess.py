"""Pins of the learned-initial-guess oracle (oracle/guess.py) against values and
identities that do not come from the oracle itself: features worked out by hand on a
three-cell strip, a network wired by hand to reproduce chosen inputs, central finite
differences for every gradient, Adam's update written out by hand, and properties of
training and of the safeguard."""
import numpy as np
import pytest

from oracle import guess as G


def strip_case():
    # three cells in a row: faces (0, 1) and (1, 2); n_p = 2 coefficients per cell
    nbrs = G.face_neighbours(3, [0, 1], [1, 2])
    h = np.full(3, np.sqrt(2.0))
    sc = G.Scales(u_rest=-60.0, s_u=10.0, s_d=2.0, h_ref=np.sqrt(2.0), dt_ref=0.05)
    Uk = np.array([-50.0, 1.0, -40.0, 2.0, -60.0, 0.0])
    Uk1 = np.array([-52.0, 1.0, -41.0, 1.0, -60.0, 0.0])
    Uk2 = np.array([-55.0, 0.0, -41.0, 1.0, -61.0, 0.0])
    return nbrs, h, sc, Uk, Uk1, Uk2


def test_features_by_hand():
    nbrs, h, sc, Uk, Uk1, Uk2 = strip_case()
    assert [list(x) for x in nbrs] == [[1], [0, 2], [1]]
    X = G.features(nbrs, h, 0.1, Uk, Uk1, Uk2, 2, sc)
    # own [a | d1 | d2] per cell, a = (U^k - u_rest e0)/s_u, d1 = (U^k - U^k-1)/s_d, d2 = (U^k-1 - U^k-2)/s_d
    own0 = [1.0, 0.1, 1.0, 0.0, 1.5, 0.5]
    own1 = [2.0, 0.2, 0.5, 0.5, 0.0, 0.0]
    own2 = [0.0, 0.0, 0.0, 0.0, 0.5, 0.0]
    expect = np.array([
        own0 + own1 + own1 + [1.0, 2.0, 0.1],
        own1 + [0.5, 0.05, 0.5, 0.0, 1.0, 0.25] + own0 + [1.0, 2.0, 0.2],
        own2 + own1 + own1 + [1.0, 2.0, 0.1],
    ])
    assert X.shape == (3, G.n_inputs(2)) == (3, 21)
    assert np.allclose(X, expect, rtol=0, atol=1e-15)


def test_isolated_cell_pools_zero():
    nbrs = G.face_neighbours(2, [], [])
    X = G.features(nbrs, np.ones(2), 0.05, np.ones(4), np.zeros(4), np.zeros(4), 2, G.Scales())
    assert np.all(X[:, 6:18] == 0.0) and np.all(X[:, 20] == 0.0)


def test_network_wired_to_copy_inputs():
    """relu(u) - relu(-u) = u: hidden pairs copy inputs 3 and 7; W2 = I passes them on;
    W3 recombines.  Any transposed or misplaced layer breaks the equality."""
    n_p, H = 2, 4
    F = G.n_inputs(n_p)
    W1 = np.zeros((H, F))
    W1[0, 3], W1[1, 3], W1[2, 7], W1[3, 7] = 1.0, -1.0, 1.0, -1.0
    P = {"W1": W1, "b1": np.zeros(H), "W2": np.eye(H), "b2": np.zeros(H),
         "W3": np.array([[1.0, -1.0, 0.0, 0.0], [0.0, 0.0, 1.0, -1.0]]),
         "b3": np.array([0.5, -0.25])}
    X = np.random.default_rng(0).standard_normal((9, F))
    o, _ = G.forward(P, X)
    assert np.array_equal(o, np.stack([X[:, 3] + 0.5, X[:, 7] - 0.25], axis=1))
    # the flat layout round-trips
    th = G.flatten(P)
    assert th.size == G.n_params(n_p, H) == H * F + H + H * H + H + n_p * H + n_p
    Q = G.unflatten(th, n_p, H)
    assert all(np.array_equal(P[k], Q[k]) for k in P)


def test_gradients_against_central_differences():
    rng = np.random.default_rng(1)
    n_p, H, m = 3, 5, 7
    F = G.n_inputs(n_p)
    th = rng.standard_normal(G.n_params(n_p, H)) * 0.5
    X = rng.standard_normal((m, F))
    T = rng.standard_normal((m, n_p))
    L, g = G.loss_and_grads(G.unflatten(th, n_p, H), X, T)
    gflat = G.flatten(g)
    eps = 1e-6
    fd = np.empty_like(th)
    for k in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[k] += eps
        tm[k] -= eps
        fd[k] = (G.loss(G.unflatten(tp, n_p, H), X, T) - G.loss(G.unflatten(tm, n_p, H), X, T)) / (2 * eps)
    assert np.isclose(L, G.loss(G.unflatten(th, n_p, H), X, T))
    assert np.max(np.abs(fd - gflat)) <= 1e-7 * max(1.0, np.max(np.abs(gflat)))


def test_adam_first_step_is_lr_times_sign():
    th = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    st = G.adam_init(3)
    new = G.adam_step(th, g, st, lr=0.01)
    expect = np.array([1.0 - 0.01 * 0.5 / (0.5 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8),
                       3.0 - 0.01 * 1e-3 / (1e-3 + 1e-8)])
    assert np.allclose(new, expect, rtol=0, atol=1e-15)


def test_adam_two_steps_on_quadratic_by_hand():
    # f = theta^2 / 2, g = theta, theta0 = 1, lr 0.1, b1 0.9, b2 0.999, eps 1e-8
    st = G.adam_init(1)
    t1 = G.adam_step(np.array([1.0]), np.array([1.0]), st, lr=0.1)
    th1 = 1.0 - 0.1 * 1.0 / (1.0 + 1e-8)
    t2 = G.adam_step(t1, t1.copy(), st, lr=0.1)
    m2 = 0.9 * 0.1 + 0.1 * th1
    v2 = 0.999 * 0.001 + 0.001 * th1 * th1
    th2 = th1 - 0.1 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.998001)) + 1e-8)
    assert abs(t1[0] - th1) <= 1e-15 and abs(t2[0] - th2) <= 1e-14


def test_training_fits_a_learnable_target():
    rng = np.random.default_rng(2)
    n_p, H, m = 2, 16, 256
    F = G.n_inputs(n_p)
    X = rng.standard_normal((m, F))
    T = X @ (0.3 * rng.standard_normal((F, n_p)))
    th = rng.standard_normal(G.n_params(n_p, H)) * 0.2
    st = G.adam_init(th.size)
    L0 = G.loss(G.unflatten(th, n_p, H), X, T)
    for _ in range(400):
        _, g = G.loss_and_grads(G.unflatten(th, n_p, H), X, T)
        th = G.adam_step(th, G.flatten(g), st, lr=1e-2)
    assert G.loss(G.unflatten(th, n_p, H), X, T) <= 0.05 * L0


def test_safeguard_keeps_the_smaller_residual():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 6))
    K = A @ A.T + 6 * np.eye(6)
    x = rng.standard_normal(6)
    b = K @ x
    near, far = x + 1e-3, x + 1.0
    assert G.safeguard(K, b, near, far)[1] is True
    assert G.safeguard(K, b, far, near)[1] is False
    assert G.safeguard(K, b, near, near)[1] is False      # ties keep U^k
    # a network with zero output layer proposes U^k itself
    n_p, H = 2, 3
    P = G.unflatten(rng.standard_normal(G.n_params(n_p, H)), n_p, H)
    P["W3"][:] = 0.0
    P["b3"][:] = 0.0
    Uk = rng.standard_normal(6)
    X = rng.standard_normal((3, G.n_inputs(n_p)))
    assert np.array_equal(G.propose(P, X, Uk, G.Scales(s_d=3.0)), Uk)


# ------------------------------------------------------------ subspace initial guess
def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return B @ B.T + n * np.eye(n)


def test_subspace_guess_recovers_a_solution_in_the_span():
    # x* = U^k + 0.7 (U^k - U^{k-1}) - 0.2 (U^{k-2} - U^{k-3}): the residual vanishes
    from oracle.guess import subspace_guess
    K = _spd(40, 1)
    rng = np.random.default_rng(2)
    H = [rng.standard_normal(40) for _ in range(5)]
    xs = H[0] + 0.7 * (H[0] - H[1]) - 0.2 * (H[2] - H[3])
    x0, th = subspace_guess(K, K @ xs, H, m=4)
    assert np.allclose(x0, xs, atol=1e-10)
    assert np.allclose(th, [0.7, 0.0, -0.2, 0.0], atol=1e-10)


def test_subspace_guess_single_direction_closed_form_and_never_worse():
    # one direction: theta = v.r0 / v.Kv; more directions never raise the K-norm error
    from oracle.guess import subspace_guess
    K = _spd(30, 3)
    rng = np.random.default_rng(4)
    H = [rng.standard_normal(30) for _ in range(9)]
    b = rng.standard_normal(30)
    xs = np.linalg.solve(K, b)
    knorm = lambda e: np.sqrt(e @ (K @ e))
    x1, th = subspace_guess(K, b, H[:2], m=1)
    r0, v = b - K @ H[0], H[0] - H[1]
    assert np.isclose(th[0], (v @ r0) / (v @ (K @ v)), rtol=1e-12)
    err = [knorm(xs - H[0])]
    for m in range(1, 9):
        x0, _ = subspace_guess(K, b, H, m=m)
        err.append(knorm(xs - x0))
    assert all(err[i + 1] <= err[i] * (1 + 1e-12) for i in range(8))
    # the error is K-orthogonal to the span (Galerkin)
    x0, _ = subspace_guess(K, b, H, m=8)
    V = np.stack([H[j - 1] - H[j] for j in range(1, 9)], 1)
    assert np.abs(V.T @ (K @ (xs - x0))).max() < 1e-9 * np.abs(V.T @ (K @ xs)).max()
    # with a proposal as well
    xg = rng.standard_normal(30)
    x0g, thg = subspace_guess(K, b, H, xg=xg, m=8)
    assert len(thg) == 9 and knorm(xs - x0g) <= err[-1] * (1 + 1e-12)
