"""Checkpoint / resume and bounded device waits, on a GB300 (through the C ABI).

* Resume: a simulation stepped k times, its state saved to the host (the last 17
  potentials, the ionic state, the step index), then restored into a fresh simulation
  with sim_set_state + sim_set_history, continues bit for bit like one that was never
  interrupted -- per-node and modal ionic forms, with the subspace initial guess.
* Waits: with polydg_set_wait_limit(0) the grid barriers of the persistent kernel give
  up at once; the solve and the preconditioner application return POLYDG_ECUDA (no
  fault, no trap), and after restoring the default limit the same context solves again.
"""
import numpy as np
import pytest
import torch

from test_gpu_parity import lib, dev, host, mnorm_rel, gpu_ctx

pytestmark = pytest.mark.gpu

H = 17     # solutions the subspace initial guess reads


def make_sim(pd, ctx, pc, w, form):
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-10, maxit=5000,
                        flexible=True)
    if form == "modal":
        pd.sim_set_ionic_form(sim, "modal")
    pd.sim_set_guess(sim, None, 3)
    return sim


def snapshot(pd, sim, ctx, n_nodes, form):
    u = torch.empty(ctx.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.empty(5 * n_nodes, dtype=torch.float64, device="cuda")
    pd.sim_get_state(sim, u, y)
    Y = None
    if form == "modal":
        Y = torch.empty(5 * ctx.n_dofs, dtype=torch.float64, device="cuda")
        pd.sim_get_ionic_coeffs(sim, Y)
    torch.cuda.synchronize()
    return u.cpu(), y.cpu(), (Y.cpu() if Y is not None else None)


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
    hist = []
    for _ in range(k1):
        pd.monodomain_step(run, 1)
        hist.append(snapshot(pd, run, ctx, n_nodes, form)[0])
    _, y_k, Y_k = snapshot(pd, run, ctx, n_nodes, form)
    assert run.step_index == k1
    run.close()

    # a fresh simulation resumes from the host copies
    res = make_sim(pd, ctx, pc, w, form)
    pd.sim_set_state(res, k1, y=y_k.cuda(), Y=Y_k.cuda() if Y_k is not None else None)
    assert res.step_index == k1
    last = torch.stack(hist[::-1][:H]).contiguous().cuda()        # U^k, U^{k-1}, ...
    pd.sim_set_history(res, last)
    pd.monodomain_step(res, k2)
    u_res, y_res, Y_res = snapshot(pd, res, ctx, n_nodes, form)
    assert res.step_index == k1 + k2
    assert torch.equal(u_res, u_ref)
    assert torch.equal(y_res, y_ref)
    if form == "modal":
        assert torch.equal(Y_res, Y_ref)
    # and the run is a real one: the state moved during the resumed steps
    assert not torch.equal(y_res, y_k)


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
