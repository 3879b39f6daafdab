"""Parity of the CUDA path with the FP64 oracle on polyhedral (3D) meshes, on a GB300.

Jittered hexahedra split into 12-facet polyhedra, P2 (n_p = 10).  Two small cases
the oracle solves directly: a 4^3 mesh with anisotropic conductivity, 8 subdomains
and 8 coarse agglomerates (coarse inverse formed on the device), and a 10^3 mesh
whose coarse space has one agglomerate per cell (n_0 = 4000: the coarse inverse is
formed on the host and the persistent kernel distributes the coarse rows over its
CTAs behind an extra grid barrier).  Then the 48^3 workload (1,105,920 DOFs): rows
of K_h sampled against the oracle's assembly of each sampled cell's neighbourhood,
the true residual of fp64 and fp32 solves, and the fp32 form's coupled run against
the fp64 form's.  Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import cached
from test_gpu_parity import lib, dev, host, mnorm_rel

pytestmark = pytest.mark.gpu


def make_case(name):
    from synth import Workload, stimulus_params
    from synth.meshes import jittered_hex_cube, block_partition_3d, isotropic_conductivity
    from oracle import assembly
    from test_oracle_3d import random_spd

    def build():
        if name == "hex4":
            m = jittered_hex_cube(4, 13)
            sig = random_spd(m.n_cells, 21)
            sub = block_partition_3d(4, 2)
            coarse = sub.copy()
        else:
            m = jittered_hex_cube(10, 17)
            sig = isotropic_conductivity(m.n_cells, 1.0, dim=3)
            sub = block_partition_3d(10, 2)
            coarse = np.arange(m.n_cells, dtype=np.int32)
        w = Workload(name, m, 2, 1, sig, sub, coarse, eta0=10.0, dt=0.05, rtol=1e-8,
                     n_steps=10, stimulus=stimulus_params(23, dim=3))
        d = assembly.assemble(m, 2, sig, w.eta0, w.chi_cm, w.dt)
        return w, d
    return cached(("3d", name), build)


def ctx_of(w):
    return lib().setup_mesh(w.mesh, w.sigma, w.p, w.subdomain, w.chi_cm, w.dt, w.eta0)


@pytest.fixture(scope="module")
def hex4():
    w, d = make_case("hex4")
    return w, d, ctx_of(w)


@pytest.fixture(scope="module")
def hex10():
    w, d = make_case("hex10")
    return w, d, ctx_of(w)


@pytest.mark.parametrize("case", ["hex4", "hex10"])
def test_connectivity_bit_exact_3d(case, request):
    w, d, ctx = request.getfixturevalue(case)
    plus, minus = ctx.faces()
    assert np.array_equal(plus, d.faces.plus) and np.array_equal(minus, d.faces.minus)
    assert ctx.info.n_dofs == d.n_dofs and ctx.info.n_p == 10


@pytest.mark.parametrize("case", ["hex4", "hex10"])
def test_matvec_elementwise_3d(case, request):
    w, d, ctx = request.getfixturevalue(case)
    x = np.random.default_rng(31).standard_normal(d.n_dofs)
    y = dev(np.zeros(d.n_dofs))
    ctx.matvec(dev(x), y)
    bound = 64 * np.finfo(float).eps * (abs(d.K) @ np.abs(x))
    assert np.all(np.abs(host(y) - d.K @ x) <= bound)


@pytest.mark.parametrize("case", ["hex4", "hex10"])
def test_asm_apply_fp64_3d(case, request):
    from oracle import schwarz
    w, d, ctx = request.getfixturevalue(case)
    pd = lib()
    S = cached(("3d-schwarz", case), lambda: schwarz.build(d, w.subdomain, w.coarse, w.q))
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    assert pc.info()["n_coarse"] == 4 * (int(w.coarse.max()) + 1)
    r = np.random.default_rng(32).standard_normal(d.n_dofs)
    z = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(r), z)
    ref = S.apply(r)
    assert np.linalg.norm(host(z) - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("case", ["hex4", "hex10"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pcg_solution_3d(case, prec, request):
    from oracle import schwarz
    from oracle.pcg import pcg
    w, d, ctx = request.getfixturevalue(case)
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=prec)
    b = np.random.default_rng(33).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000, flexible=(prec != "fp64"))
    ref = cached(("3d-direct", case), lambda: spla.spsolve(d.K.tocsc(), b))
    assert st["status"] == 0 and st["relres"] <= 1e-12
    assert mnorm_rel(d, host(x), ref) <= 1e-8
    if prec == "fp64":
        S = cached(("3d-schwarz", case), lambda: schwarz.build(d, w.subdomain, w.coarse, w.q))
        st2 = pd.pcg_solve(ctx, pc, dev(b), dev(np.zeros(d.n_dofs)), rtol=w.rtol, maxit=5000)
        its = pcg(d.K, b, prec=S.apply, rtol=w.rtol).iterations
        assert abs(st2["iterations"] - its) <= 2, (st2, its)


def test_coupled_steps_3d(hex4):
    from oracle import monodomain
    w, d, _ = hex4
    pd = lib()
    steps = 10
    ctx = ctx_of(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-12, maxit=5000)
    st = pd.monodomain_step(sim, steps)
    assert st["status"] == 0 and st["steps_done"] == steps
    nodes = monodomain.quadrature_nodes(d)
    u, y = dev(np.zeros(d.n_dofs)), dev(np.zeros(5 * len(nodes.w)))
    pd.sim_get_state(sim, u, y)
    md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
    for _ in range(steps):
        ref = md.step()
    assert mnorm_rel(d, host(u), ref.U) <= 1e-8
    yg = host(y).reshape(5, -1)
    assert np.allclose(yg, ref.y, rtol=1e-9, atol=1e-12)
    # the stimulus is on and off-centre: the potential is not uniform any more
    assert np.ptp(ref.U[::d.n_p]) > 1e-3


def test_invalid_3d_mesh_rejected():
    from synth.meshes import jittered_hex_cube, isotropic_conductivity
    pd = lib()
    m = jittered_hex_cube(2, 1)
    sig = isotropic_conductivity(m.n_cells, 1.0, dim=3)
    zero = np.zeros(m.n_cells, np.int32)
    fv = m.face_vtx.copy()
    fv[0] = fv[0][::-1]                       # one inward facet
    with pytest.raises(pd.PolyDGError) as e:
        pd.polydg_setup3d(m.vertices, m.cell_face_ptr, fv, sig, 2, zero)
    assert e.value.status == pd.POLYDG_EINVAL
    with pytest.raises(pd.PolyDGError) as e:   # only P2 maps to the device kernels in 3D
        pd.polydg_setup3d(m.vertices, m.cell_face_ptr, m.face_vtx, sig, 1, zero)
    assert e.value.status == pd.POLYDG_EINVAL
    bad = sig.copy(); bad[0, 0, 1] = 0.5      # not symmetric
    with pytest.raises(pd.PolyDGError) as e:
        pd.polydg_setup3d(m.vertices, m.cell_face_ptr, m.face_vtx, bad, 2, zero)
    assert e.value.status == pd.POLYDG_EINVAL


# ------------------------------------------------------------- 48^3 workload
def neighbourhood_rows(mesh, sigma, p, eta0, chi_cm, dt, cells):
    """Oracle block rows of K_h for the given cells, each from the assembly of the
    sub-mesh made of the cell and its face neighbours (a row of K_h depends on that
    cell, its neighbours and the faces between them only)."""
    from synth.meshes import PolyMesh3D
    from oracle import assembly
    owner = {}
    for k in range(mesh.n_cells):
        for t in mesh.facets(k):
            owner.setdefault(tuple(sorted(int(v) for v in t)), []).append(k)
    out = {}
    for k in cells:
        nbr = sorted({c for t in mesh.facets(k) for c in owner[tuple(sorted(int(v) for v in t))]})
        fp = np.concatenate([[0], np.cumsum([len(mesh.facets(c)) for c in nbr])]).astype(np.int64)
        sub = PolyMesh3D(mesh.vertices, fp, np.concatenate([mesh.facets(c) for c in nbr]))
        d = assembly.assemble(sub, p, sigma[nbr], eta0, chi_cm, dt)
        i = nbr.index(k)
        K = d.K.toarray()
        n = d.n_p
        out[k] = {c: K[i * n:(i + 1) * n, j * n:(j + 1) * n] for j, c in enumerate(nbr)}
    return out


@pytest.fixture(scope="module")
def hex48():
    from synth import hex_cube_p2
    w = hex_cube_p2()
    return w, ctx_of(w)


def test_hex48_sampled_rows_of_matvec(hex48):
    w, ctx = hex48
    n_p = 10
    nd = ctx.info.n_dofs
    assert nd == 1105920
    rng = np.random.default_rng(41)
    cells = sorted(set(rng.choice(w.mesh.n_cells, 24, replace=False).tolist()) | {0, w.mesh.n_cells - 1})
    rows = neighbourhood_rows(w.mesh, w.sigma, w.p, w.eta0, w.chi_cm, w.dt, cells)
    x = rng.standard_normal(nd)
    y = dev(np.zeros(nd))
    ctx.matvec(dev(x), y)
    got = host(y).reshape(-1, n_p)
    X = x.reshape(-1, n_p)
    for k in cells:
        ref = sum(B @ X[c] for c, B in rows[k].items())
        absref = sum(np.abs(B) @ np.abs(X[c]) for c, B in rows[k].items())
        assert np.all(np.abs(got[k] - ref) <= 64 * np.finfo(float).eps * absref), k


def test_hex48_fp32_and_fp64_solves_and_coupled_run(hex48):
    w, ctx = hex48
    pd = lib()
    nd = ctx.info.n_dofs
    b = np.random.default_rng(42).standard_normal(nd)
    sols, its = {}, {}
    for prec in ("fp64", "fp32"):
        pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=prec)
        x = dev(np.zeros(nd))
        st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-8, maxit=2000, flexible=(prec == "fp32"))
        assert st["status"] == 0
        r = dev(np.zeros(nd))
        ctx.matvec(x, r)
        true_res = np.linalg.norm(b - host(r)) / np.linalg.norm(b)
        assert true_res <= 2e-8, (prec, true_res)
        sols[prec], its[prec] = host(x), st["iterations"]
        sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=w.rtol, maxit=2000,
                            flexible=(prec == "fp32"))
        sst = pd.monodomain_step(sim, w.n_steps)
        assert sst["status"] == 0 and sst["steps_done"] == w.n_steps
        u = dev(np.zeros(nd))
        pd.sim_get_state(sim, u, None)
        sols[prec + "_u"] = host(u)
        its[prec + "_steps"] = sst["total_iterations"] / w.n_steps
        sim.close()
        pc.close()
    print("hex48 iterations", its)
    e = np.linalg.norm(sols["fp32"] - sols["fp64"]) / np.linalg.norm(sols["fp64"])
    assert e <= 1e-6, e
    eu = np.linalg.norm(sols["fp32_u"] - sols["fp64_u"]) / np.linalg.norm(sols["fp64_u"])
    assert eu <= 1e-6, eu


def test_one_element_subdomains_3d(hex4):
    """T_S = T_h on a polyhedral mesh (one subdomain per cell, the small-subdomain P phase)
    with the 2^3-cell agglomerates as the coarse space: B_ad r and PCG against the oracle."""
    from oracle import schwarz
    import dataclasses
    w, d, _ = hex4
    pd = lib()
    wm = dataclasses.replace(w, subdomain=np.arange(w.mesh.n_cells, dtype=np.int32))
    ctx = ctx_of(wm)
    S = schwarz.build(d, wm.subdomain, wm.coarse, wm.q)
    r = np.random.default_rng(35).standard_normal(d.n_dofs)
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-4), ("bf16", 5e-2)):
        pc = pd.asm_setup(ctx, wm.coarse, q=wm.q, precision=prec)
        assert pc.info()["n_subdomains"] == w.mesh.n_cells
        z = dev(np.zeros(d.n_dofs))
        pd.asm_apply(pc, dev(r), z)
        ref = S.apply(r)
        assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref), prec
    pc = pd.asm_setup(ctx, wm.coarse, q=wm.q, precision="fp64")
    b = np.random.default_rng(36).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000)
    assert st["status"] == 0
    assert mnorm_rel(d, host(x), spla.spsolve(d.K.tocsc(), b)) <= 1e-8


@pytest.mark.slow
def test_hex12_coupled_run_in_the_measured_form_vs_oracle():
    """The 48^3 workload's recipe on a 12^3 mesh the oracle assembles (27 subdomains of 4^3
    cells = coarse agglomerates, coarse P1, isotropic sigma, the same stimulus recipe): 8
    coupled steps in the measured form -- fp32 local inverses, flexible PCG, the subspace
    initial guess -- at rtol 1e-12 against the oracle's exactly solved trajectory."""
    from oracle import monodomain
    from synth import hex_cube_p2
    from oracle import assembly
    w = hex_cube_p2(n=12)
    d = cached(("hex12", "disc"), lambda: assembly.assemble(w.mesh, w.p, w.sigma, w.eta0, w.chi_cm, w.dt))
    pd = lib()
    steps = 8
    ctx = ctx_of(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=1e-12, maxit=5000, flexible=True)
    pd.sim_set_guess(sim, None, 3)
    st = pd.monodomain_step(sim, steps)
    assert st["status"] == 0 and st["steps_done"] == steps
    nodes = monodomain.quadrature_nodes(d)
    u, y = dev(np.zeros(d.n_dofs)), dev(np.zeros(5 * len(nodes.w)))
    pd.sim_get_state(sim, u, y)
    md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
    for _ in range(steps):
        ref = md.step()
    assert mnorm_rel(d, host(u), ref.U) <= 1e-8
    assert np.allclose(host(y).reshape(5, -1), ref.y, rtol=1e-9, atol=1e-12)
