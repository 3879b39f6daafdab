"""Lockstep groups of simulations sharing their local solves (shared_local +
sim_set_shared_local + batch_step): every member against the oracle's exactly solved
coupled trajectory with its own conductivity.

Tolerances: fp32 eigenbasis at rtol 1e-12 (flexible PCG; the store only changes the
preconditioner): the coupled-step bound of the single-simulation tests, 1e-8 in the
function L2 norm; bf16 eigenbasis at the workload tolerance 1e-8: 1e-6, as for the
mixed form.  A batch may mix a group with simulations that have their own inverses;
a member that fails stops alone.
"""
import numpy as np
import pytest

from conftest import cached

pytestmark = pytest.mark.gpu

STEPS = 8
SIGMAS = [0.6, 1.0, 1.7]


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
def family():
    """Three workloads on one 150-cell Voronoi P3 mesh with 4 subdomains, scalar
    conductivities 0.6, 1.0, 1.7 and different stimulus sites."""
    from synth import Workload
    from synth.meshes import voronoi_square, kmeans_partition, isotropic_conductivity
    from oracle import assembly

    def make():
        m = voronoi_square(150, 31)
        part = kmeans_partition(m, 4, 31)
        out = []
        for k, sg in enumerate(SIGMAS):
            stim = {"x0": 0.3 + 0.2 * k, "y0": 0.6 - 0.1 * k, "amplitude": 250.0, "width": 0.08,
                    "duration": 1.0}
            w = Workload(f"group150_s{k}", m, 3, 1, isotropic_conductivity(m.n_cells, sg), part,
                         part.copy(), eta0=10.0, dt=0.05, rtol=1e-8, n_steps=STEPS, stimulus=stim)
            d = assembly.assemble(m, 3, w.sigma, w.eta0, w.chi_cm, w.dt)
            out.append((w, d))
        return out
    return cached("group_family", make)


def oracle_run(w, d, steps):
    from oracle import monodomain

    def run():
        md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
        for _ in range(steps):
            s = md.step()
        return s
    return cached(("coupled", w.name, steps), run)


def make_sim(w, rtol, maxit=5000):
    pd = lib()
    ctx = pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                          w.subdomain, w.chi_cm, w.dt, w.eta0)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    return ctx, pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=rtol, maxit=maxit,
                              flexible=True)


def state(sim, n):
    pd = lib()
    u = dev(np.zeros(n))
    pd.sim_get_state(sim, u)
    return host(u)


@pytest.mark.parametrize("precision,rtol,tol", [("fp32", 1e-12, 1e-8), ("bf16", 1e-8, 1e-6)])
def test_group_members_match_oracle(family, precision, rtol, tol):
    pd = lib()
    made = [make_sim(w, rtol) for w, _ in family]
    sl = pd.shared_local_setup(made[0][0], precision)
    for _, sim in made:
        pd.sim_set_shared_local(sim, sl)
    bt = pd.batch_create([sim for _, sim in made])
    assert len(set(bt.groups().tolist())) == 1          # one group: the same CTAs for all
    stats, _ = pd.batch_step(bt, STEPS)
    for (w, d), (_, sim), st in zip(family, made, stats):
        assert st["status"] == 0 and st["steps_done"] == STEPS
        assert mnorm_rel(d, state(sim, d.n_dofs), oracle_run(w, d, STEPS).U) <= tol


def test_group_next_to_a_solo_simulation(family, voronoi256):
    pd = lib()
    made = [make_sim(w, 1e-12) for w, _ in family[:2]]
    sl = pd.shared_local_setup(made[0][0], "fp32")
    for _, sim in made:
        pd.sim_set_shared_local(sim, sl)
    w2, d2 = voronoi256
    _, solo = make_sim(w2, 1e-12)
    bt = pd.batch_create([made[0][1], solo, made[1][1]])
    stats, _ = pd.batch_step(bt, STEPS)
    assert all(st["status"] == 0 for st in stats)
    for (w, d), (_, sim) in zip(family[:2], made):
        assert mnorm_rel(d, state(sim, d.n_dofs), oracle_run(w, d, STEPS).U) <= 1e-8
    assert mnorm_rel(d2, state(solo, d2.n_dofs), oracle_run(w2, d2, STEPS).U) <= 1e-8


def test_group_member_failure_is_isolated(family):
    pd = lib()
    made = [make_sim(w, 1e-12, maxit=(2 if k == 1 else 5000)) for k, (w, _) in enumerate(family)]
    sl = pd.shared_local_setup(made[0][0], "fp32")
    for _, sim in made:
        pd.sim_set_shared_local(sim, sl)
    bt = pd.batch_create([sim for _, sim in made])
    stats, _ = pd.batch_step(bt, 3, allow=(pd.POLYDG_ENOTCONV,))
    assert stats[1]["status"] == pd.POLYDG_ENOTCONV and stats[1]["steps_done"] == 1
    for k in (0, 2):
        assert stats[k]["status"] == 0 and stats[k]["steps_done"] == 3


def test_shared_local_checks(family):
    pd = lib()
    from synth.meshes import voronoi_square
    (w0, _), (w1, _) = family[0], family[1]
    c0, s0 = make_sim(w0, 1e-8)
    sl = pd.shared_local_setup(c0, "bf16")
    other = voronoi_square(150, 32)                  # another mesh
    from synth.meshes import kmeans_partition, isotropic_conductivity
    ctx = pd.polydg_setup(other.vertices, other.cell_ptr, other.cell_vtx,
                          isotropic_conductivity(other.n_cells, 1.0), 3,
                          kmeans_partition(other, 4, 32), 1.0, 0.05, 10.0)
    pc = pd.asm_setup(ctx, kmeans_partition(other, 4, 32), q=1, precision="fp32")
    sim = pd.sim_create(ctx, pc, u0=-67.0, flexible=True)
    with pytest.raises(pd.PolyDGError) as e:
        pd.sim_set_shared_local(sim, sl)
    assert e.value.status == pd.POLYDG_EINVAL
    pd.sim_set_shared_local(s0, sl)
    bt = pd.batch_create([s0])
    pd.sim_set_shared_local(s0, None)
    with pytest.raises(pd.PolyDGError) as e:             # membership changed after create
        pd.batch_step(bt, 1)
    assert e.value.status == pd.POLYDG_EINVAL
