"""Local solves shared by simulations that differ in a scalar conductivity: the GPU's
two-pass eigenbasis application (one factorisation, several right-hand sides with their
own conductivities) against the oracle's (oracle/multirhs.py, fp64).

Tolerances: fp32 store of Q: fp32 rounding of Q, of L^{-1} r and of the sums over n_i
terms, amplified at most by the condition of the element mass factors on either side:
1e-4 relative in the 2-norm.  bf16 store: unit roundoff 2^-9 in every entry of Q instead:
3e-2.  Each right-hand side is compared with its own conductivity's exact local solve.
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


@pytest.fixture(scope="module")
def case():
    from synth.meshes import voronoi_square, kmeans_partition, isotropic_conductivity
    from oracle import assembly, multirhs

    def make():
        m = voronoi_square(150, 31)
        part = kmeans_partition(m, 4, 31)
        d1 = assembly.assemble(m, 3, isotropic_conductivity(m.n_cells, 1.0), 10.0, 1.0, 0.05)
        S = multirhs.build(d1.M, d1.A, multirhs.subdomain_dofs(part, d1.n_p), d1.n_p)
        return m, part, d1, S
    return cached("shared_local_case", make)


def gpu_ctx(m, part, sigma):
    from synth.meshes import isotropic_conductivity
    pd = lib()
    return pd.polydg_setup(m.vertices, m.cell_ptr, m.cell_vtx, isotropic_conductivity(m.n_cells, sigma),
                           3, part, 1.0, 0.05, 10.0)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 3e-2)])
def test_shared_local_solves_match_oracle(case, precision, tol):
    from oracle import multirhs
    m, part, d1, S = case
    pd = lib()
    ctx = gpu_ctx(m, part, 1.3)                   # any member's context: sigma_ref = 1.3
    sl = pd.shared_local_setup(ctx, precision)
    assert sl.info()["sigma_ref"] == 1.3
    sigmas = [0.6, 1.3, 1.9, 0.5]
    rng = np.random.default_rng(5)
    rs = [rng.standard_normal(d1.n_dofs) for _ in sigmas]
    zs = [dev(np.zeros(d1.n_dofs)) for _ in sigmas]
    pd.shared_local_apply(sl, [dev(r) for r in rs], zs, sigmas)
    for r, z, sg in zip(rs, zs, sigmas):
        ref = multirhs.apply_local(S, r, sg, 1.0, 0.05)
        got = host(z)
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (precision, sg)


def test_fewer_right_hand_sides_and_store_size(case):
    from oracle import multirhs
    m, part, d1, S = case
    pd = lib()
    ctx = gpu_ctx(m, part, 0.8)
    sl = pd.shared_local_setup(ctx, "bf16")
    n_i = [len(x) for x in multirhs.subdomain_dofs(part, d1.n_p)]
    assert sl.info()["store_bytes"] == sum(2 * n * ((n + 7) // 8 * 8) * 2 for n in n_i)
    r = np.random.default_rng(6).standard_normal(d1.n_dofs)
    z = dev(np.zeros(d1.n_dofs))
    pd.shared_local_apply(sl, [dev(r)], [z], [1.1])
    ref = multirhs.apply_local(S, r, 1.1, 1.0, 0.05)
    assert np.linalg.norm(host(z) - ref) <= 3e-2 * np.linalg.norm(ref)


def test_anisotropic_conductivity_is_rejected(case):
    from synth.meshes import fibre_conductivity
    m, part, d1, S = case
    pd = lib()
    ctx = pd.polydg_setup(m.vertices, m.cell_ptr, m.cell_vtx, fibre_conductivity(m, 1.3, 0.2, 3),
                          3, part, 1.0, 0.05, 10.0)
    with pytest.raises(pd.PolyDGError) as e:
        pd.shared_local_setup(ctx, "fp32")
    assert e.value.status == pd.POLYDG_EINVAL


@pytest.mark.parametrize("nrhs", [5, 16])
def test_tensor_core_passes_for_many_right_hand_sides(case, nrhs):
    """BF16 store: both passes run as tcgen05 BF16 GEMMs (FP32 accumulate) for up to 16
    right-hand sides at once; each one against the oracle's exact local solve with its own
    conductivity (3e-2, the BF16 bound above), and against the FP32-eigenbasis form in
    groups of four (the two differ by the BF16 rounding of Q alone: 3e-2).  The subdomains
    here have ~375 DOFs: three 128-row tiles, the last one ragged, six 64-column tiles."""
    from oracle import multirhs
    m, part, d1, S = case
    pd = lib()
    ctx = gpu_ctx(m, part, 1.0)
    sl = pd.shared_local_setup(ctx, "bf16")
    sl32 = pd.shared_local_setup(ctx, "fp32")
    rng = np.random.default_rng(40 + nrhs)
    sigmas = list(rng.uniform(0.5, 2.0, nrhs))
    rs = [rng.standard_normal(d1.n_dofs) for _ in range(nrhs)]
    zs = [dev(np.zeros(d1.n_dofs)) for _ in range(nrhs)]
    pd.shared_local_apply(sl, [dev(r) for r in rs], zs, sigmas)
    z32 = [dev(np.zeros(d1.n_dofs)) for _ in range(nrhs)]
    for k0 in range(0, nrhs, 4):
        k1 = min(nrhs, k0 + 4)
        pd.shared_local_apply(sl32, [dev(r) for r in rs[k0:k1]], z32[k0:k1], sigmas[k0:k1])
    for r, z, zf, sg in zip(rs, zs, z32, sigmas):
        ref = multirhs.apply_local(S, r, sg, 1.0, 0.05)
        got = host(z)
        assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref), sg
        assert np.linalg.norm(got - host(zf)) <= 3e-2 * np.linalg.norm(ref), sg
    # the same right-hand side in two slots gives the same result (columns are independent)
    z1, z2 = dev(np.zeros(d1.n_dofs)), dev(np.zeros(d1.n_dofs))
    pd.shared_local_apply(sl, [dev(rs[0]), dev(rs[0])], [z1, z2], [sigmas[0], sigmas[0]])
    assert np.array_equal(host(z1), host(z2))


def test_tensor_core_rhs_limit(case):
    m, part, d1, S = case
    pd = lib()
    ctx = gpu_ctx(m, part, 1.0)
    sl = pd.shared_local_setup(ctx, "bf16")
    r = [dev(np.zeros(d1.n_dofs)) for _ in range(17)]
    with pytest.raises(pd.PolyDGError) as e:
        pd.shared_local_apply(sl, r, r, [1.0] * 17)
    assert e.value.status == pd.POLYDG_EINVAL
