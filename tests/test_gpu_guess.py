"""Learned PCG initial guess on the GPU against the oracle (oracle/guess.py).

- proposal (features + network on the tensor cores: fp16 weights, features and
  activations as fp16 operands, fp32 accumulation) against the oracle's fp64 forward
  with the same fp16-rounded weights, with and without the three fp16 roundings of the
  layer inputs (5e-4 and 5e-3 of the largest output, times s_d);
- one training step: loss (fp32 vs fp64, 1e-5 relative) and the gradient read back
  from Adam's first moment (m = (1 - beta1) g after one step), within 1e-4 of the
  oracle's gradient in the 2-norm;
- coupled steps with a model attached reach the same answers as without (the safeguard
  and the FP64 stopping test decide), and a model whose output is zero is never taken.
"""
import numpy as np
import pytest

from conftest import cached

pytestmark = pytest.mark.gpu


def lib():
    import os
    import paper_2512_19536_gb300 as pd
    if not os.path.exists(pd.LIB_PATH):
        from paper_2512_19536_gb300.build import build
        build()
    return pd


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def mnorm_rel(d, got, ref):
    e = got - ref
    return np.sqrt(e @ (d.M @ e)) / np.sqrt(ref @ (d.M @ ref))


def init_params(n_p, seed, out_scale=1.0):
    """Seeded He-style initial parameters (the same arrays go to oracle and GPU)."""
    from oracle import guess as G
    rng = np.random.default_rng(seed)
    P = {}
    for name, shp in G.shapes(n_p, 128):
        if name.startswith("W"):
            P[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
        else:
            P[name] = 0.1 * rng.standard_normal(shp)
    P["W3"] *= out_scale
    return G.flatten(P)


def scales_for(d):
    from oracle import guess as G
    return G.Scales(u_rest=-67.0, s_u=50.0, s_d=0.3, h_ref=float(d.geom.diameter.mean()),
                    dt_ref=0.05)


def history(d, seed):
    rng = np.random.default_rng(seed)
    n = d.n_dofs
    Uk = np.zeros(n)
    Uk[::d.n_p] = -67.0
    Uk += rng.standard_normal(n)
    Uk1 = Uk - 0.2 * rng.standard_normal(n)
    Uk2 = Uk1 - 0.2 * rng.standard_normal(n)
    return Uk, Uk1, Uk2


def gpu_ctx(w):
    pd = lib()
    return pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                           w.subdomain, w.chi_cm, w.dt, w.eta0)


@pytest.fixture(scope="module")
def vor(voronoi256):
    w, d = voronoi256
    from oracle import guess as G
    nbrs = G.face_neighbours(d.mesh.n_cells, d.faces.plus, d.faces.minus)
    return w, d, gpu_ctx(w), nbrs


def test_proposal_matches_oracle(vor):
    from oracle import guess as G
    w, d, ctx, nbrs = vor
    pd = lib()
    theta = init_params(d.n_p, 11)
    sc = scales_for(d)
    model = pd.guess_create(d.n_p, theta, sc.as_array())
    Uk, Uk1, Uk2 = history(d, 12)
    x = dev(np.zeros(d.n_dofs))
    pd.guess_propose(model, ctx, dev(Uk), dev(Uk1), dev(Uk2), x)
    got = host(x)
    P16 = G.unflatten(theta.astype(np.float32).astype(np.float16).astype(np.float64), d.n_p, 128)
    X = G.features(nbrs, d.geom.diameter, w.dt, Uk, Uk1, Uk2, d.n_p, sc)
    o, _ = G.forward(P16, X)
    ref = G.propose(P16, X, Uk, sc)
    assert np.max(np.abs(o)) > 0.1                       # a non-trivial network output
    # the tensor-core kernel takes the features and both hidden layers' outputs as FP16
    # operands (FP32 accumulation): the same network with those three roundings, to the
    # FP32 sums' order (an activation whose FP32 and FP64 sums round to neighbouring FP16
    # values moves o by a weight times one FP16 ulp of it) ...
    h = lambda a: a.astype(np.float16).astype(np.float64)
    h1 = h(np.maximum(h(X) @ P16["W1"].T + P16["b1"], 0.0))
    h2 = h(np.maximum(h1 @ P16["W2"].T + P16["b2"], 0.0))
    ref16 = Uk + sc.s_d * (h2 @ P16["W3"].T + P16["b3"]).reshape(-1)
    assert np.max(np.abs(got - ref16)) <= 5e-4 * sc.s_d * np.max(np.abs(o))
    # ... and the FP64-activation network within the three roundings' bound (unit roundoff
    # 2^-11 each, through two layers of 128-term sums)
    assert np.max(np.abs(got - ref)) <= 5e-3 * sc.s_d * np.max(np.abs(o))


def trajectory(w, d, steps):
    """Caller-order solutions U^0..U^steps of the oracle's exactly solved run."""
    from oracle import monodomain

    def run():
        md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
        out = [md.state.U.copy()]
        for _ in range(steps):
            out.append(md.step().U.copy())
        return np.array(out)
    return cached(("traj", w.name, steps), run)


def test_train_step_matches_oracle(vor):
    from oracle import guess as G
    w, d, ctx, nbrs = vor
    pd = lib()
    traj = trajectory(w, d, 8)
    sc = scales_for(d)
    sc.s_d = float(np.sqrt(np.mean((traj[1:] - traj[:-1]) ** 2)))
    theta = init_params(d.n_p, 13)
    model = pd.guess_create(d.n_p, theta, sc.as_array())
    rng = np.random.default_rng(14)
    n = 300                                                # several tiles and a ragged tail
    samples = np.stack([rng.integers(2, 7, n), rng.integers(0, d.mesh.n_cells, n)], axis=1)
    lr = 1e-3
    loss = pd.guess_train_step(model, ctx, dev(traj), samples, lr)
    # oracle: the same samples, fp32-rounded initial parameters
    th32 = theta.astype(np.float32).astype(np.float64)
    Xs, Ts = [], []
    for k, c in samples:
        X = G.features(nbrs, d.geom.diameter, w.dt, traj[k], traj[k - 1], traj[k - 2], d.n_p, sc)
        Xs.append(X[c])
        Ts.append(G.targets(traj[k], traj[k + 1], d.n_p, sc)[c])
    X, T = np.array(Xs), np.array(Ts)
    L, g = G.loss_and_grads(G.unflatten(th32, d.n_p, 128), X, T)
    gref = G.flatten(g)
    p, m, v, t = model.params()
    assert t == 1
    assert abs(loss - L) <= 1e-5 * L
    ggpu = m / (1.0 - 0.9)
    assert np.linalg.norm(ggpu - gref) <= 1e-4 * np.linalg.norm(gref)
    st = G.adam_init(th32.size)
    new = G.adam_step(th32, ggpu, st, lr)                  # the update rule, from the GPU's gradient
    assert np.max(np.abs(p - new)) <= 1e-6 * lr + 1e-7 * np.max(np.abs(th32))


def test_training_reduces_loss_on_trajectories(vor):
    w, d, ctx, _ = vor
    pd = lib()
    traj = trajectory(w, d, 12)
    sc = scales_for(d)
    sc.s_d = float(np.sqrt(np.mean((traj[1:] - traj[:-1]) ** 2)))
    model = pd.guess_create(d.n_p, init_params(d.n_p, 15, out_scale=0.1), sc.as_array())
    rng = np.random.default_rng(16)
    T = dev(traj)
    losses = []
    for it in range(60):
        samples = np.stack([rng.integers(2, 11, 512), rng.integers(0, d.mesh.n_cells, 512)], axis=1)
        losses.append(pd.guess_train_step(model, ctx, T, samples, 3e-3))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5])


def run_sim(w, d, model, steps, rtol=1e-12, precision="fp64", flexible=False):
    pd = lib()
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=precision)
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=rtol, maxit=5000,
                        flexible=flexible)
    if model is not None:
        pd.sim_set_guess(sim, model)
    st = pd.monodomain_step(sim, steps)
    u = dev(np.zeros(d.n_dofs))
    pd.sim_get_state(sim, u)
    return st, host(u)


def test_zero_output_model_is_never_taken(vor):
    from oracle import guess as G
    w, d, _, _ = vor
    pd = lib()
    P = G.unflatten(init_params(d.n_p, 17), d.n_p, 128)
    P["W3"][:] = 0.0
    P["b3"][:] = 0.0
    model = pd.guess_create(d.n_p, G.flatten(P), scales_for(d).as_array())
    st_g, u_g = run_sim(w, d, model, 6, rtol=1e-8)
    st_0, u_0 = run_sim(w, d, None, 6, rtol=1e-8)
    assert st_g["guesses_taken"] == 0
    assert st_g["total_iterations"] == st_0["total_iterations"]
    assert np.array_equal(u_g, u_0)


def test_coupled_steps_with_trained_guess_match_oracle(vor):
    """A briefly trained model attached: the answer after 12 steps at rtol 1e-12 is the
    oracle's within the coupled-step bound; the guess is taken on some steps."""
    w, d, ctx, _ = vor
    pd = lib()
    traj = trajectory(w, d, 12)
    sc = scales_for(d)
    sc.s_d = float(np.sqrt(np.mean((traj[1:] - traj[:-1]) ** 2)))
    model = pd.guess_create(d.n_p, init_params(d.n_p, 18, out_scale=0.1), sc.as_array())
    rng = np.random.default_rng(19)
    T = dev(traj)
    for _ in range(80):
        samples = np.stack([rng.integers(2, 11, 512), rng.integers(0, d.mesh.n_cells, 512)], axis=1)
        pd.guess_train_step(model, ctx, T, samples, 3e-3)
    st, u = run_sim(w, d, model, 12)
    assert st["status"] == 0 and st["steps_done"] == 12
    assert 0 <= st["guesses_taken"] <= 10
    assert mnorm_rel(d, u, traj[12]) <= 1e-8


# ------------------------------------------------------------ subspace guess (policy 3)
def subspace_run(w, d, steps, model=None, rtol=1e-8, reset_history=False):
    """Per-step iteration counts and the final potential of a policy-3 run; with
    reset_history the simulation's own last solutions are restored through
    sim_set_history before every step, followed by the per-node functions its ionic update
    carries (sim_set_ionic_aux: setting the potentials invalidates them) -- a host-side
    state round trip."""
    import torch
    pd = lib()
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=rtol, maxit=5000)
    pd.sim_set_guess(sim, model, 3)
    its, hist = [], [dev(np.zeros(d.n_dofs))]
    pd.sim_get_state(sim, hist[0])
    for _ in range(steps):
        if reset_history:
            aux = torch.empty(6 * ctx.info.n_nodes, dtype=torch.float64, device="cuda")
            pd.sim_get_ionic_aux(sim, aux)
            pd.sim_set_history(sim, torch.stack(hist[::-1][:25]))
            pd.sim_set_ionic_aux(sim, aux)
        st = pd.monodomain_step(sim, 1)
        assert st["status"] == 0
        its.append(st["total_iterations"])
        u = dev(np.zeros(d.n_dofs))
        pd.sim_get_state(sim, u)
        hist.append(u)
    return its, host(hist[-1])


def test_subspace_guess_iterations_and_answer_match_oracle(vor):
    """Policy 3 without a model against the oracle running the same recipe
    (oracle.guess.subspace_guess + PCG with the same preconditioner): per-step
    iteration counts within 3, totals within 5 %, far fewer than from U^k, and the
    potential after the steps within the coupled-step bound of the direct solve."""
    from oracle import guess as G, monodomain, schwarz
    from oracle.pcg import pcg
    w, d, _, _ = vor
    steps = 40
    its, u = subspace_run(w, d, steps)
    S = cached(("schwarz", w.name), lambda: schwarz.build(d, w.subdomain, w.coarse, w.q))
    md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
    hist, ref_its, plain_its = [md.state.U.copy()], [], []
    for _ in range(steps):
        st = md.state
        b, y_new = md.rhs(st)
        x0, _ = G.subspace_guess(d.K, b, hist[::-1], m=24)
        r = pcg(d.K, b, x0=x0, prec=S.apply, rtol=1e-8)
        ref_its.append(r.iterations)
        plain_its.append(pcg(d.K, b, x0=st.U, prec=S.apply, rtol=1e-8).iterations)
        md.state = monodomain.State(r.x, st.U, y_new, st.k + 1)
        hist.append(r.x.copy())
    # the least squares are ill-conditioned (nearly parallel increments), so the two sides'
    # roundings pick slightly different guesses: a few iterations apart per step
    assert max(abs(a - b) for a, b in zip(its, ref_its)) <= 8, (list(its), list(ref_its))
    assert abs(sum(its) - sum(ref_its)) <= 0.05 * sum(ref_its), (sum(its), sum(ref_its))
    assert sum(its) < 0.8 * sum(plain_its), (sum(its), sum(plain_its))
    direct = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
    for _ in range(steps):
        ref = direct.step()
    assert mnorm_rel(d, u, ref.U) <= 1e-6


def test_subspace_guess_history_round_trip(vor):
    """Restoring the simulation's own last solutions before every step changes nothing."""
    w, d, _, _ = vor
    its_a, u_a = subspace_run(w, d, 14)
    its_b, u_b = subspace_run(w, d, 14, reset_history=True)
    assert its_a == its_b
    assert np.array_equal(u_a, u_b)


def test_subspace_guess_with_zero_model_drops_its_direction(vor):
    """A model whose output is zero gives K v_0 = 0: its direction is dropped by the
    pivoting and the steps match the model-free run; at rtol 1e-12 the answer is the
    oracle's."""
    from oracle import guess as G, monodomain
    w, d, _, _ = vor
    pd = lib()
    P = G.unflatten(init_params(d.n_p, 17), d.n_p, 128)
    P["W3"][:] = 0.0
    P["b3"][:] = 0.0
    model = pd.guess_create(d.n_p, G.flatten(P), scales_for(d).as_array())
    its_m, u_m = subspace_run(w, d, 10, model=model, rtol=1e-12)
    its_0, u_0 = subspace_run(w, d, 10, rtol=1e-12)
    assert its_m == its_0
    direct = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
    for _ in range(10):
        ref = direct.step()
    assert mnorm_rel(d, u_m, ref.U) <= 1e-8
