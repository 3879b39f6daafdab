"""The ionic state in the DG basis (Eq. fully-discrete-1, second line) on a GB300.

sim_set_ionic_form(sim, "modal") keeps, per cell and state, the n_p coefficients of the
DG basis and advances them by M_K^{-1} times the projected explicit increment; the ion
current then uses the states at the quadrature nodes.  Checked against the oracle's
modal form (oracle.monodomain, ionic_form="modal", direct solves) on the anisotropic
256-cell Voronoi P3 case with a Gaussian stimulus: after 20 coupled steps at rtol 1e-12
the potential within 1e-8 in the function L2 norm and the nodal states within 1e-9
relative, as for the per-node form in test_gpu_parity.py (the modal update adds one
n_p-term projection and one n_p x n_p product per state and step, in float64).  Also:
the form is fixed once stepping has started, a return to the per-node form before the
first step gives the per-node run bit for bit, and a batch that mixes both forms steps
each simulation as the oracle does.
"""
import numpy as np
import pytest

from conftest import cached
from test_gpu_parity import lib, dev, host, mnorm_rel, gpu_ctx, oracle_coupled

pytestmark = pytest.mark.gpu

STEPS = 20


def oracle_modal(w, d, steps):
    from oracle import monodomain

    def run():
        md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest, ionic_form="modal")
        return [md.step() for _ in range(steps)]
    return cached(("coupled_modal", w.name, steps), run)


def new_sim(pd, ctx, pc, w, form):
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-12, maxit=5000)
    pd.sim_set_ionic_form(sim, form)
    return sim


def state_of(pd, sim, d, w):
    from oracle import monodomain
    nodes = cached(("nodes", w.name), lambda: monodomain.quadrature_nodes(d))
    u = dev(np.zeros(d.n_dofs))
    y = dev(np.zeros(5 * len(nodes.w)))
    pd.sim_get_state(sim, u, y)
    return host(u), host(y).reshape(5, -1)


def test_modal_coupled_steps_parity(voronoi256):
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    sim = new_sim(pd, ctx, pc, w, "modal")
    st = pd.monodomain_step(sim, STEPS)
    u, y = state_of(pd, sim, d, w)
    ref = oracle_modal(w, d, STEPS)[-1]
    assert st["status"] == 0 and st["steps_done"] == STEPS
    assert mnorm_rel(d, u, ref.U) <= 1e-8
    assert np.allclose(y, ref.y, rtol=1e-9, atol=1e-12)
    # the modal states differ from the per-node ones (the forms are not the same update)
    nodal = oracle_coupled(w, d, STEPS)[-1]
    assert np.abs(ref.y - nodal.y).max() > 1e-9


def test_modal_form_is_chosen_before_the_first_step(voronoi256):
    pd = lib()
    w, d = voronoi256
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    sim = new_sim(pd, ctx, pc, w, "modal")
    pd.monodomain_step(sim, 1)
    with pytest.raises(pd.PolyDGError) as err:
        pd.sim_set_ionic_form(sim, "nodal")
    assert err.value.status == pd.POLYDG_EINVAL
    # modal then back to per-node before stepping: the per-node run, bit for bit
    a = new_sim(pd, ctx, pc, w, "modal")
    pd.sim_set_ionic_form(a, "nodal")
    b = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-12, maxit=5000)
    pd.monodomain_step(a, 3)
    pd.monodomain_step(b, 3)
    ua, ya = state_of(pd, a, d, w)
    ub, yb = state_of(pd, b, d, w)
    assert np.array_equal(ua, ub) and np.array_equal(ya, yb)


def test_batch_mixing_modal_and_nodal_forms(voronoi256):
    pd = lib()
    w, d = voronoi256
    sims, ctxs, pcs = [], [], []
    for form in ("modal", "nodal"):
        ctx = gpu_ctx(w)
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
        ctxs.append(ctx)
        pcs.append(pc)
        sims.append(new_sim(pd, ctx, pc, w, form))
    batch = pd.batch_create(sims)
    pd.batch_step(batch, STEPS)
    refs = (oracle_modal(w, d, STEPS)[-1], oracle_coupled(w, d, STEPS)[-1])
    for sim, ref in zip(sims, refs):
        u, y = state_of(pd, sim, d, w)
        assert mnorm_rel(d, u, ref.U) <= 1e-8
        assert np.allclose(y, ref.y, rtol=1e-9, atol=1e-12)
