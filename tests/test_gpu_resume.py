"""Checkpoint / resume and bounded device waits, on a GB300 (through the C ABI).

* Resume: a simulation stepped k times, its state saved to the host (the last 25
  potentials, the ionic state -- with, for the per-node form, the functions of it that the
  update carries -- and the step index), then restored into a fresh simulation with
  sim_set_state + sim_set_history + sim_set_ionic_aux, continues bit for bit like one that
  was never interrupted -- per-node and modal ionic forms, with the subspace initial guess.
  Without the carried functions the resumed run agrees to rounding; the carried functions
  agree with their definitions evaluated from the state.
* Waits: with polydg_set_wait_limit(0) the grid barriers of the persistent kernel give
  up at once; the solve and the preconditioner application return POLYDG_ECUDA (no
  fault, no trap), and after restoring the default limit the same context solves again.
"""
import numpy as np
import pytest
import torch

from test_gpu_parity import lib, dev, host, mnorm_rel, gpu_ctx

pytestmark = pytest.mark.gpu

H = 25     # solutions the subspace initial guess reads


def make_sim(pd, ctx, pc, w, form):
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-10, maxit=5000,
                        flexible=True)
    if form == "modal":
        pd.sim_set_ionic_form(sim, "modal")
    pd.sim_set_guess(sim, None, 3)
    return sim


def snapshot(pd, sim, ctx, n_nodes, form):
    """U^k, the nodal states and, per form, the modal coefficients or the per-node functions
    the nodal update carries."""
    u = torch.empty(ctx.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.empty(5 * n_nodes, dtype=torch.float64, device="cuda")
    pd.sim_get_state(sim, u, y)
    if form == "modal":
        Y = torch.empty(5 * ctx.n_dofs, dtype=torch.float64, device="cuda")
        pd.sim_get_ionic_coeffs(sim, Y)
    else:
        Y = torch.empty(6 * n_nodes, dtype=torch.float64, device="cuda")
        pd.sim_get_ionic_aux(sim, Y)
    torch.cuda.synchronize()
    return u.cpu(), y.cpu(), Y.cpu()


@pytest.mark.parametrize("form", ["nodal", "modal"])
def test_resumed_run_is_bit_identical(voronoi256, form):
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    n_nodes = ctx.info.n_nodes
    k1, k2 = 20, 6            # the stimulus is on during both parts (t < 1 ms)

    ref = make_sim(pd, ctx, pc, w, form)
    pd.monodomain_step(ref, k1 + k2)
    u_ref, y_ref, Y_ref = snapshot(pd, ref, ctx, n_nodes, form)

    # the interrupted run: k1 steps, the state to the host (the potentials step by step)
    run = make_sim(pd, ctx, pc, w, form)
    hist = [snapshot(pd, run, ctx, n_nodes, form)[0]]           # U^0, then U^1 .. U^k1
    for _ in range(k1):
        pd.monodomain_step(run, 1)
        hist.append(snapshot(pd, run, ctx, n_nodes, form)[0])
    _, y_k, Y_k = snapshot(pd, run, ctx, n_nodes, form)
    assert run.step_index == k1
    run.close()

    # a fresh simulation resumes from the host copies (the carried functions last: setting
    # the potentials invalidates them)
    res = make_sim(pd, ctx, pc, w, form)
    pd.sim_set_state(res, k1, y=y_k.cuda(), Y=Y_k.cuda() if form == "modal" else None)
    assert res.step_index == k1
    last = torch.stack(hist[::-1][:H]).contiguous().cuda()        # U^k, U^{k-1}, ...
    pd.sim_set_history(res, last)
    if form == "nodal":
        pd.sim_set_ionic_aux(res, Y_k.cuda())
    pd.monodomain_step(res, k2)
    u_res, y_res, Y_res = snapshot(pd, res, ctx, n_nodes, form)
    assert res.step_index == k1 + k2
    assert torch.equal(u_res, u_ref)
    assert torch.equal(y_res, y_ref)
    assert torch.equal(Y_res, Y_ref)
    # and the run is a real one: the state moved during the resumed steps
    assert not torch.equal(y_res, y_k)


def carried_from_state(y):
    """E_Na, E_K, exp(-K_o/5), exp((25 - Na_i)/3) of nodal states y [5, n] (Sec. 2 model:
    K_i = 140 + (18 - Na_i), Na_o = 144 - 7 (Na_i - 18), E = 26.64 ln(c_out / c_in)); the
    carried u^{k-1} and exp(-u^{k-1}/720) are checked against each other."""
    Ko, Nai = y[2], y[3]
    Ki = 140.0 + (18.0 - Nai)
    Nao = 144.0 - 7.0 * (Nai - 18.0)
    return np.stack([26.64 * np.log(Nao / Nai), 26.64 * np.log(Ko / Ki), np.exp(-Ko / 5.0),
                     np.exp((25.0 - Nai) / 3.0)])


def test_carried_ionic_functions_track_the_state(voronoi256):
    """The nodal update carries functions of each node's state from step to step (updated
    from the step's increments, evaluated afresh every 256th step); after 255 carried steps
    -- the longest stretch, the stimulus on for the first 20 -- they agree with their
    definitions evaluated from the state to within a few hundred ulps, and the carried
    exp(-u^{k-1}/720) with the carried u^{k-1}."""
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    n_nodes = ctx.info.n_nodes
    sim = make_sim(pd, ctx, pc, w, "nodal")
    pd.monodomain_step(sim, 256)          # steps k = 0..255: evaluated at k = 0, then carried
    _, y, aux = snapshot(pd, sim, ctx, n_nodes, "nodal")
    y = y.numpy().reshape(5, -1)
    aux = aux.numpy().reshape(6, -1)
    ref = carried_from_state(y)
    rel = np.abs(aux[:4] - ref) / np.abs(ref).max(axis=1, keepdims=True)
    assert rel.max() <= 1e-12, rel.max(axis=1)
    B = np.exp(-aux[4] / 720.0)
    assert np.max(np.abs(aux[5] - B) / B) <= 1e-12
    assert np.max(np.abs(aux[4] - w.u_rest)) > 0.1   # the potential left its initial rest value
    assert np.ptp(y[2]) > 1e-6            # the concentrations did move


def test_resume_without_the_carried_functions_differs_by_rounding(voronoi256):
    """Restoring the state without sim_set_ionic_aux: the first resumed step evaluates the
    carried functions from the state, and the run stays within rounding of the
    uninterrupted one (relative difference of U far below the solver tolerance)."""
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    n_nodes = ctx.info.n_nodes
    k1, k2 = 20, 6
    ref = make_sim(pd, ctx, pc, w, "nodal")
    pd.monodomain_step(ref, k1 + k2)
    u_ref, _, _ = snapshot(pd, ref, ctx, n_nodes, "nodal")
    run = make_sim(pd, ctx, pc, w, "nodal")
    hist = [snapshot(pd, run, ctx, n_nodes, "nodal")[0]]        # U^0, then U^1 .. U^k1
    for _ in range(k1):
        pd.monodomain_step(run, 1)
        hist.append(snapshot(pd, run, ctx, n_nodes, "nodal")[0])
    _, y_k, _ = snapshot(pd, run, ctx, n_nodes, "nodal")
    res = make_sim(pd, ctx, pc, w, "nodal")
    pd.sim_set_state(res, k1, y=y_k.cuda())
    pd.sim_set_history(res, torch.stack(hist[::-1][:H]).contiguous().cuda())
    pd.monodomain_step(res, k2)
    u_res, _, _ = snapshot(pd, res, ctx, n_nodes, "nodal")
    assert float(torch.linalg.norm(u_res - u_ref) / torch.linalg.norm(u_ref)) <= 1e-8


def test_set_state_rejects_bad_arguments(voronoi256):
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    sim = make_sim(pd, ctx, pc, w, "nodal")
    y = torch.zeros(5 * ctx.info.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PolyDGError):
        pd.sim_set_state(sim, -1, y=y)                       # negative step index
    with pytest.raises(pd.PolyDGError):
        pd.sim_set_state(sim, 3)                             # the nodal form needs y
    Y = torch.zeros(5 * ctx.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PolyDGError):
        pd.sim_get_ionic_coeffs(sim, Y)                      # nodal form: no coefficients
    modal = make_sim(pd, ctx, pc, w, "modal")
    aux = torch.zeros(4 * ctx.info.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PolyDGError):
        pd.sim_get_ionic_aux(modal, aux)                     # modal form: nothing carried
    with pytest.raises(pd.PolyDGError):
        pd.sim_set_ionic_aux(modal, aux)


def test_device_wait_runs_out_and_the_context_recovers(voronoi256):
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    b = np.random.default_rng(61).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    z = dev(np.zeros(d.n_dofs))
    pd.set_wait_limit(0)              # a grid barrier gives up unless its CTA arrived last
    try:
        with pytest.raises(pd.PolyDGError) as e:
            pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-10, maxit=500, flexible=True)
        assert e.value.status == pd.POLYDG_ECUDA and "timed out" in str(e.value)
        with pytest.raises(pd.PolyDGError) as e:
            pd.asm_apply(pc, dev(b), z)
        assert e.value.status == pd.POLYDG_ECUDA
    finally:
        pd.set_wait_limit(-1)
    # the context is intact: the same solve now converges to the direct solution
    import scipy.sparse.linalg as spla
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000, flexible=True)
    assert st["status"] == 0
    assert mnorm_rel(d, host(x), spla.spsolve(d.K.tocsc(), b)) <= 1e-8
