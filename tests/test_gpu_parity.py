"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on a GB300.

Tolerances, derived from the arithmetic:
  * connectivity: bit-exact (integer work);
  * K x: both sides sum the same 10-term products in float64 in different
    orders, so |Kx_gpu - Kx_oracle| <= 64 eps (|K| |x|) entry-wise;
  * B_ad r (fp64 store): the GPU applies explicit inverses formed by Cholesky,
    the oracle Cholesky solves; both are backward stable, so the difference is
    bounded by kappa(K_i) eps ~ 1e-11 relative for these kappa; we use 1e-9;
  * solutions: GPU PCG at rtol 1e-12 against the oracle's direct solve, error
    in the function L2 norm sqrt(e^T M e) / sqrt(u^T M u) <= 1e-8;
  * coupled steps: relative L2 error of u after the steps <= 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def gpu_ctx(w):
    pd = lib()
    return pd.polydg_setup(w.mesh.vertices, w.mesh.cell_ptr, w.mesh.cell_vtx, w.sigma, w.p,
                           w.subdomain, w.chi_cm, w.dt, w.eta0)


@pytest.fixture(scope="module")
def sq(square16):
    w, d = square16
    return w, d, gpu_ctx(w)


@pytest.fixture(scope="module")
def vor(voronoi256):
    w, d = voronoi256
    return w, d, gpu_ctx(w)


@pytest.mark.parametrize("case", ["sq", "vor"])
def test_connectivity_bit_exact(case, request):
    w, d, ctx = request.getfixturevalue(case)
    plus, minus = ctx.faces()
    assert np.array_equal(plus, d.faces.plus) and np.array_equal(minus, d.faces.minus)
    assert ctx.info.n_faces == len(d.faces.plus)
    assert ctx.info.n_dofs == d.n_dofs


@pytest.mark.parametrize("case", ["sq", "vor"])
def test_matvec_elementwise(case, request):
    w, d, ctx = request.getfixturevalue(case)
    x = np.random.default_rng(3).standard_normal(d.n_dofs)
    y = dev(np.zeros(d.n_dofs))
    ctx.matvec(dev(x), y)
    got = host(y)
    ref = d.K @ x
    bound = 64 * np.finfo(float).eps * (abs(d.K) @ np.abs(x))
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("case", ["sq", "vor"])
def test_asm_apply_fp64(case, request):
    from oracle import schwarz
    w, d, ctx = request.getfixturevalue(case)
    pd = lib()
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    r = np.random.default_rng(4).standard_normal(d.n_dofs)
    z = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(r), z)
    got, ref = host(z), S.apply(r)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()        # entry by entry


def test_asm_apply_one_level(vor):
    from oracle import schwarz
    w, d, ctx = vor
    pd = lib()
    S = schwarz.build(d, w.subdomain, None)
    pc = pd.asm_setup(ctx, None, precision="fp64")
    r = np.random.default_rng(5).standard_normal(d.n_dofs)
    z = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(r), z)
    ref = S.apply(r)
    assert np.linalg.norm(host(z) - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.abs(host(z) - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_asm_apply_reduced_precision_error_bound(vor, prec):
    # fp32/bf16 store of K_i^{-1}: relative error of B r bounded by the store's
    # unit roundoff times the inverse's row-sum growth; checked loosely.
    from oracle import schwarz
    w, d, ctx = vor
    pd = lib()
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=prec)
    r = np.random.default_rng(6).standard_normal(d.n_dofs)
    z = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(r), z)
    ref = S.apply(r)
    tol = 1e-4 if prec == "fp32" else 5e-2
    assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref)
    assert np.abs(host(z) - ref).max() <= tol * np.abs(ref).max()


def test_asm_apply_edge_cases(vor):
    # r = 0 gives z = 0 exactly; a NaN in r is reported, and the context stays usable
    w, d, ctx = vor
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    z = dev(np.full(d.n_dofs, 7.0))
    pd.asm_apply(pc, dev(np.zeros(d.n_dofs)), z)
    assert np.array_equal(host(z), np.zeros(d.n_dofs))
    r = np.random.default_rng(8).standard_normal(d.n_dofs)
    r[17] = np.nan
    with pytest.raises(pd.PolyDGError) as e:
        pd.asm_apply(pc, dev(r), z)
    assert e.value.status == pd.POLYDG_ENONFINITE
    r[17] = 0.5
    pd.asm_apply(pc, dev(r), z)
    assert np.all(np.isfinite(host(z)))
    # the application is linear and deterministic: B (2r) = 2 B r bit for bit (a power of
    # two scales every rounding exactly), and two calls agree bit for bit
    z2 = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(2.0 * r), z2)
    assert np.array_equal(host(z2), 2.0 * host(z))
    z3 = dev(np.zeros(d.n_dofs))
    pd.asm_apply(pc, dev(r), z3)
    assert np.array_equal(host(z3), host(z))


@pytest.mark.parametrize("case", ["sq", "vor"])
def test_pcg_solution_and_iterations(case, request):
    from oracle import schwarz
    from oracle.pcg import pcg
    w, d, ctx = request.getfixturevalue(case)
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    b = np.random.default_rng(7).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000)
    ref = spla.spsolve(d.K.tocsc(), b)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    assert mnorm_rel(d, host(x), ref) <= 1e-8
    # iteration counts at the workload tolerance agree with the oracle's PCG
    S = schwarz.build(d, w.subdomain, w.coarse, w.q)
    x2 = dev(np.zeros(d.n_dofs))
    st2 = pd.pcg_solve(ctx, pc, dev(b), x2, rtol=w.rtol, maxit=5000)
    its = pcg(d.K, b, prec=S.apply, rtol=w.rtol).iterations
    assert abs(st2["iterations"] - its) <= 2, (st2, its)


def test_plain_cg(sq):
    from oracle.pcg import pcg
    w, d, ctx = sq
    pd = lib()
    b = np.random.default_rng(8).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, None, dev(b), x, rtol=1e-10, maxit=20000)
    ref = spla.spsolve(d.K.tocsc(), b)
    assert st["status"] == 0
    assert mnorm_rel(d, host(x), ref) <= 1e-7
    its = pcg(d.K, b, rtol=1e-10).iterations
    assert abs(st["iterations"] - its) <= max(3, its // 50)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_flexible_pcg_mixed_precision_converges_to_fp64_answer(vor, prec):
    w, d, ctx = vor
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=prec)
    b = np.random.default_rng(9).standard_normal(d.n_dofs)
    x = dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000, flexible=True)
    ref = spla.spsolve(d.K.tocsc(), b)
    assert st["status"] == 0
    assert mnorm_rel(d, host(x), ref) <= 1e-8


def test_edge_cases(vor):
    pd = lib()
    w, d, ctx = vor
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    n = d.n_dofs
    # b = 0 -> x = 0 without iterations, whatever x0 was
    x = dev(np.ones(n))
    st = pd.pcg_solve(ctx, pc, dev(np.zeros(n)), x, rtol=1e-8)
    assert st["iterations"] == 0 and st["status"] == 0 and np.all(host(x) == 0)
    # x0 = exact solution -> zero iterations
    b = np.random.default_rng(10).standard_normal(n)
    ref = spla.spsolve(d.K.tocsc(), b)
    x = dev(ref)
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-8)
    assert st["iterations"] == 0
    # maxit reached -> ENOTCONV, x holds the last iterate (better than x0 = 0)
    x = dev(np.zeros(n))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-14, maxit=3)
    assert st["status"] == pd.POLYDG_ENOTCONV and st["iterations"] == 3
    assert 0 < st["relres"] < 1
    # non-finite right-hand side -> ENONFINITE
    bad = b.copy(); bad[5] = np.nan
    with pytest.raises(pd.PolyDGError) as e:
        pd.pcg_solve(ctx, pc, dev(bad), dev(np.zeros(n)), rtol=1e-8)
    assert e.value.status == pd.POLYDG_ENONFINITE
    # invalid arguments
    with pytest.raises(pd.PolyDGError) as e:
        pd.pcg_solve(ctx, pc, dev(b), dev(np.zeros(n)), rtol=-1.0)
    assert e.value.status == pd.POLYDG_EINVAL


def test_single_subdomain_one_level_converges_in_one_iteration():
    from synth.meshes import cartesian_square, isotropic_conductivity
    pd = lib()
    m = cartesian_square(6)
    zero = np.zeros(m.n_cells, np.int32)
    ctx = pd.polydg_setup(m.vertices, m.cell_ptr, m.cell_vtx, isotropic_conductivity(36, 1.0), 2,
                          zero, 1.0, 0.1, 10.0)
    pc = pd.asm_setup(ctx, None, precision="fp64")
    b = np.random.default_rng(11).standard_normal(ctx.n_dofs)
    st = pd.pcg_solve(ctx, pc, dev(b), dev(np.zeros(ctx.n_dofs)), rtol=1e-10)
    assert st["iterations"] == 1


def test_invalid_mesh_rejected():
    from synth.meshes import cartesian_square, isotropic_conductivity
    pd = lib()
    m = cartesian_square(2)
    cv = m.cell_vtx.copy()
    cv[:4] = cv[:4][::-1]                                  # clockwise first cell
    with pytest.raises(pd.PolyDGError) as e:
        pd.polydg_setup(m.vertices, m.cell_ptr, cv, isotropic_conductivity(4, 1.0), 1,
                        np.zeros(4, np.int32))
    assert e.value.status == pd.POLYDG_EINVAL
    with pytest.raises(pd.PolyDGError) as e:
        pd.polydg_setup(m.vertices, m.cell_ptr, m.cell_vtx, -isotropic_conductivity(4, 1.0), 1,
                        np.zeros(4, np.int32))
    assert e.value.status == pd.POLYDG_EINVAL


def run_coupled(w, d, steps, precision="fp64", flexible=False, rtol=1e-12):
    pd = lib()
    ctx = gpu_ctx(w)
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision=precision)
    sim = pd.sim_create(ctx, pc, u0=w.u_rest, stimulus=w.stimulus, rtol=rtol, maxit=5000,
                        flexible=flexible)
    st = pd.monodomain_step(sim, steps)
    u = dev(np.zeros(d.n_dofs))
    nodes = cached(("nodes", w.name), lambda: __import__("oracle.monodomain").monodomain.quadrature_nodes(d))
    y = dev(np.zeros(5 * len(nodes.w)))
    pd.sim_get_state(sim, u, y)
    return st, host(u), host(y).reshape(5, -1), sim


def oracle_coupled(w, d, steps):
    from oracle import monodomain
    def run():
        md = monodomain.Monodomain(d, w.stimulus, u0=w.u_rest)
        out = []
        for _ in range(steps):
            out.append(md.step())
        return out
    return cached(("coupled", w.name, steps), run)


def test_coupled_steps_parity(vor):
    w, d, _ = vor
    steps = 20
    st, u, y, sim = run_coupled(w, d, steps)
    ref = oracle_coupled(w, d, steps)[-1]
    assert st["status"] == 0 and st["steps_done"] == steps and sim.step_index == steps
    assert mnorm_rel(d, u, ref.U) <= 1e-8
    assert np.allclose(y, ref.y, rtol=1e-9, atol=1e-12)


def test_coupled_steps_mixed_precision(vor):
    w, d, _ = vor
    steps = 20
    st, u, _, _ = run_coupled(w, d, steps, precision="fp32", flexible=True)
    ref = oracle_coupled(w, d, steps)[-1]
    assert st["status"] == 0
    assert mnorm_rel(d, u, ref.U) <= 1e-8


def test_traced_pcg_coefficients_and_condition_estimate(sq):
    """alpha_k, beta_k of the GPU's plain fp64 PCG against the oracle's PCG with the
    same preconditioner (the first coefficients agree to rounding, which grows slowly
    along the iteration), and the Lanczos estimate of kappa(B_ad^{-1} K) from each."""
    from oracle import schwarz
    from oracle.pcg import pcg, lanczos_extremes
    w, d, ctx = sq
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    from synth import random_rhs
    b = random_rhs(d.n_dofs, 31)
    x = dev(np.zeros(d.n_dofs))
    st, al, be = pd.pcg_solve_trace(ctx, pc, dev(b), x, rtol=1e-10, maxit=500)
    S = cached(("schwarz", w.name), lambda: schwarz.build(d, w.subdomain, w.coarse, w.q))
    ref = pcg(d.K, b, prec=S.apply, rtol=1e-10, maxit=500)
    assert st["status"] == 0 and abs(st["iterations"] - ref.iterations) <= 1
    k = min(8, len(ref.alphas))
    assert np.allclose(al[:k], ref.alphas[:k], rtol=1e-8)
    assert np.allclose(be[:k - 1], ref.betas[:k - 1], rtol=1e-8)
    lo, hi = pd.lanczos_extremes(al, be)
    olo, ohi = lanczos_extremes(ref.alphas, ref.betas)
    assert abs(hi / lo - ohi / olo) <= 1e-6 * (ohi / olo)
