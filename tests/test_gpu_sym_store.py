"""The symmetric pair-row store of the fp32 local inverses, on a GB300 (through the C ABI).

With an fp32 store and at least four subdomains per CTA, the persistent PCG kernel streams
only the lower triangle of each K_i^{-1} (two triangle rows per bulk copy, rows m and
n - 1 - m) and adds the upper triangle's share of every row from the column sums it keeps
per warp (Sec. 4, Eq. prec: the local solves K_i^{-1} R_i r).  A 3200-cell Voronoi P3 mesh
cut into 800 k-means subdomains of about 40 DOFs takes that form; the checks are those of
the full-row store:
  * asm_info reports two rows per copy (the form is taken) for fp32 and one for fp64;
  * B_ad r against the oracle's Cholesky solves, relative 1e-4 in norm and entry by entry
    (the fp32 store's bound), and against the fp64 store on the GPU;
  * two applications are bit-identical (the column sums are added in a fixed order);
  * flexible PCG with the fp32 store reaches the direct solution to 1e-8 in the M-norm,
    and a second solve repeats it bit for bit.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import cached
from test_gpu_parity import lib, dev, host, mnorm_rel, gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def many():
    from synth.meshes import voronoi_square, kmeans_partition, fibre_conductivity
    from synth import Workload, stimulus_params
    from oracle import assembly, schwarz

    def make():
        m = voronoi_square(3200, 11)
        part = kmeans_partition(m, 800, 11)
        w = Workload("voronoi3200_p3_800", m, 3, 1, fibre_conductivity(m, 1.3, 0.2, 11), part,
                     part.copy(), eta0=10.0, dt=0.05, rtol=1e-8, n_steps=1,
                     stimulus=stimulus_params(11))
        d = assembly.assemble(m, w.p, w.sigma, w.eta0, w.chi_cm, w.dt)
        S = schwarz.build(d, w.subdomain, w.coarse, w.q)
        return w, d, S
    w, d, S = cached("voronoi3200_800", make)
    return w, d, S, gpu_ctx(w)


def test_sym_store_is_taken_for_fp32_only(many):
    w, d, S, ctx = many
    pd = lib()
    sizes = np.bincount(w.subdomain)
    assert sizes.max() * d.n_p > 32 and len(sizes) >= 4 * 152
    pc32 = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    pc64 = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    i32, i64 = pc32.info(), pc64.info()
    assert i32["rows_per_tile"] == 2 and i64["rows_per_tile"] == 1
    # the triangle rows: about half the bytes of the full rows
    n = sizes * d.n_p
    assert i32["local_store_bytes"] < 0.62 * 4 * np.sum(n * ((n + 7) // 8 * 8))


def test_sym_store_apply_matches_oracle_and_fp64(many):
    w, d, S, ctx = many
    pd = lib()
    pc32 = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    pc64 = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp64")
    r = np.random.default_rng(21).standard_normal(d.n_dofs)
    z32, z32b, z64 = (dev(np.zeros(d.n_dofs)) for _ in range(3))
    pd.asm_apply(pc32, dev(r), z32)
    pd.asm_apply(pc32, dev(r), z32b)
    pd.asm_apply(pc64, dev(r), z64)
    got, again, g64, ref = host(z32), host(z32b), host(z64), S.apply(r)
    assert np.array_equal(got, again)
    for other in (ref, g64):
        assert np.linalg.norm(got - other) <= 1e-4 * np.linalg.norm(other)
        assert np.abs(got - other).max() <= 1e-4 * np.abs(other).max()
    assert np.linalg.norm(g64 - ref) <= 1e-9 * np.linalg.norm(ref)


def test_sym_store_pcg_reaches_direct_solution(many):
    # flexible PCG (the fp32 store's preconditioner is not exactly linear, so the
    # pipelined recurrences, which assume a fixed one, are not used with it)
    w, d, S, ctx = many
    pd = lib()
    pc = pd.asm_setup(ctx, w.coarse, q=w.q, precision="fp32")
    b = np.random.default_rng(22).standard_normal(d.n_dofs)
    x, x2 = dev(np.zeros(d.n_dofs)), dev(np.zeros(d.n_dofs))
    st = pd.pcg_solve(ctx, pc, dev(b), x, rtol=1e-12, maxit=5000, flexible=True)
    st2 = pd.pcg_solve(ctx, pc, dev(b), x2, rtol=1e-12, maxit=5000, flexible=True)
    assert st["status"] == 0 and st2["iterations"] == st["iterations"]
    assert np.array_equal(host(x), host(x2))
    ref = cached("voronoi3200_800_direct", lambda: spla.spsolve(d.K.tocsc(), b))
    assert mnorm_rel(d, host(x), ref) <= 1e-8
