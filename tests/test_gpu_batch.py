"""Batched multi-simulation steps: independent simulations of uneven sizes (different
meshes, conductivities and stimuli) advanced together, all PCG solves of a step in one
cooperative launch in which each simulation owns a group of CTAs.

Parity: every simulation of the batch against the FP64 oracle's exactly solved
trajectory (the same bounds as the single-simulation coupled test: u within 1e-8 in the
function L2 norm, ionic state within 1e-9 relative, both at rtol 1e-12), and against the
same simulation stepped alone by monodomain_step.  Also: failure of one simulation
leaves the others running; repeated calls replay the captured step deterministically.
"""
import numpy as np
import pytest

from conftest import cached

pytestmark = pytest.mark.gpu

STEPS = 10


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


@pytest.fixture(scope="module")
def small_batch():
    """Two Voronoi meshes (150-400 cells, P3) with two simulations each."""
    from synth import voronoi_batch
    from oracle import assembly

    def make():
        ws = voronoi_batch(n_meshes=2, sims_per_mesh=2, seed=5, cells=(150, 400),
                           cells_per_subdomain=40, n_steps=STEPS)
        ds = [assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt) for w in ws]
        return ws, ds
    return cached("small_batch", make)


def make_sims(ws, precision="fp64", flexible=False, rtol=1e-12, maxit=5000):
    pd = lib()
    out = []
    for w in ws:
        ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                              w.subdomain, w.chi_cm, w.dt, w.eta0)
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=precision)
        m = maxit[len(out)] if isinstance(maxit, (list, tuple)) else maxit
        out.append(pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=rtol,
                                 maxit=m, flexible=flexible))
    return out


def state(sim, d, with_y=False):
    pd = lib()
    u = dev(np.zeros(d.n_dofs))
    y = None
    if with_y:
        from oracle import monodomain
        nodes = cached(("nodes", id(d)), lambda: monodomain.quadrature_nodes(d))
        y = dev(np.zeros(5 * len(nodes.w)))
    pd.sim_get_state(sim, u, y)
    return host(u), (host(y).reshape(5, -1) if with_y else None)


def oracle_run(w, d, steps):
    from oracle import monodomain

    def run():
        md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
        for _ in range(steps):
            s = md.step()
        return s
    return cached(("coupled", w.name, steps), run)


def test_batch_matches_oracle(small_batch):
    import torch
    ws, ds = small_batch
    pd = lib()
    sims = make_sims(ws)
    bt = pd.batch_create(sims)
    groups = bt.groups()
    assert groups.sum() == torch.cuda.get_device_properties(0).multi_processor_count
    assert groups.min() >= 1
    big = int(np.argmax([w.mesh.n_cells for w in ws]))
    small = int(np.argmin([w.mesh.n_cells for w in ws]))
    assert groups[big] >= groups[small]
    stats, sec = pd.batch_step(bt, STEPS)
    assert sec > 0
    for sim, st, w, d in zip(sims, stats, ws, ds):
        assert st["status"] == 0 and st["steps_done"] == STEPS and sim.step_index == STEPS
        u, y = state(sim, d, with_y=True)
        ref = oracle_run(w, d, STEPS)
        assert mnorm_rel(d, u, ref.U) <= 1e-8
        assert np.allclose(y, ref.y, rtol=1e-9, atol=1e-12)


def test_batch_mixed_precision_matches_single_runs(small_batch):
    """fp32 local inverses, flexible PCG at the workload tolerance 1e-8: each simulation
    of the batch against the same simulation stepped alone (the two solves differ only
    in the CTA partition, hence in rounding; both stop at rtol 1e-8)."""
    ws, ds = small_batch
    pd = lib()
    batched = make_sims(ws, "fp32", True, 1e-8)
    alone = make_sims(ws, "fp32", True, 1e-8)
    bt = pd.batch_create(batched)
    stats, _ = pd.batch_step(bt, STEPS)
    for sb, sa, st, w, d in zip(batched, alone, stats, ws, ds):
        sa_st = pd.monodomain_step(sa, STEPS)
        ub, _ = state(sb, d)
        ua, _ = state(sa, d)
        assert st["status"] == 0
        assert mnorm_rel(d, ub, ua) <= 1e-6
        assert abs(st["total_iterations"] - sa_st["total_iterations"]) <= STEPS
        ref = oracle_run(w, d, STEPS)
        assert mnorm_rel(d, ub, ref.U) <= 1e-6


def test_batch_replays_deterministically(small_batch):
    """One call of 2k steps and two calls of k steps give bit-identical states (the
    captured step is replayed; the batched kernel's sums are order-fixed)."""
    ws, ds = small_batch
    pd = lib()
    a = make_sims(ws, "fp32", True, 1e-8)
    b = make_sims(ws, "fp32", True, 1e-8)
    ba, bb = pd.batch_create(a), pd.batch_create(b)
    sa, _ = pd.batch_step(ba, 4)
    sb1, _ = pd.batch_step(bb, 2)
    sb2, _ = pd.batch_step(bb, 2)
    for x, y, d, s1, t1, t2 in zip(a, b, ds, sa, sb1, sb2):
        ua, _ = state(x, d)
        ub, _ = state(y, d)
        assert np.array_equal(ua, ub)
        assert s1["total_iterations"] == t1["total_iterations"] + t2["total_iterations"]


def test_batch_failure_is_isolated(small_batch):
    """A simulation whose solve cannot converge (maxit = 2) stops with ENOTCONV after its
    first step; the other simulations complete every step."""
    ws, ds = small_batch
    pd = lib()
    sims = make_sims(ws, "fp64", False, 1e-12, maxit=[5000, 2, 5000, 5000])
    bt = pd.batch_create(sims)
    stats, _ = pd.batch_step(bt, 3, allow=(pd.POLYDG_ENOTCONV,))
    assert stats[1]["status"] == pd.POLYDG_ENOTCONV and stats[1]["steps_done"] == 1
    for i in (0, 2, 3):
        assert stats[i]["status"] == 0 and stats[i]["steps_done"] == 3


def test_batch_rejects_invalid_groups(small_batch):
    ws, _ = small_batch
    pd = lib()
    w = ws[0]
    ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                          w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    s1 = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus)
    s2 = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus)
    with pytest.raises(pd.PolyDGError) as e:      # two simulations on one preconditioner
        pd.batch_create([s1, s2])
    assert e.value.status == pd.POLYDG_EINVAL
    with pytest.raises(pd.PolyDGError) as e:      # the same simulation twice
        pd.batch_create([s1, s1])
    assert e.value.status == pd.POLYDG_EINVAL
    pc32 = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    s3 = pd.sim_create(ctx, pc32, u0=w.u_rest, stimulus=w.stimulus, flexible=True)
    with pytest.raises(pd.PolyDGError) as e:      # mixed local precisions
        pd.batch_create([s1, s3])
    assert e.value.status == pd.POLYDG_EINVAL


def test_batch_one_element_subdomains_match_oracle(small_batch):
    """The massively parallel case inside the batched launch: every simulation of the
    batch with one subdomain per cell (the small-subdomain P phase of pcg_batched_kernel)
    and its k-means agglomerates as the coarse space, fp64 and the fp32 store (flexible),
    each against the oracle's exactly solved trajectory."""
    import dataclasses
    ws, ds = small_batch
    pd = lib()
    wm = [dataclasses.replace(w, subdomain=np.arange(w.mesh.n_cells, dtype=np.int32)) for w in ws]
    for precision, flexible, tol in (("fp64", False, 1e-8), ("fp32", True, 1e-8)):
        sims = make_sims(wm, precision=precision, flexible=flexible)
        bt = pd.batch_create(sims)
        stats, _ = pd.batch_step(bt, STEPS)
        for sim, st, w, d in zip(sims, stats, ws, ds):
            assert st["status"] == 0 and st["steps_done"] == STEPS, (precision, st)
            u, _ = state(sim, d)
            ref = oracle_run(w, d, STEPS)
            assert mnorm_rel(d, u, ref.U) <= tol, precision
        bt.close()
