"""polydg_spd_inverse_static: batched SPD inversion that allocates no device memory.

Some callers of this library cannot call cudaMalloc: processes whose device memory
belongs to another allocator (a caching allocator, a fixed arena reserved up front),
and code that must not fail on allocation mid-step.  This entry point keeps its workspace in one fixed
static device array.  Its output is checked, on two calls in a row, against the
library's existing inverse path: with one subdomain and no coarse space, asm_apply
applies K^{-1} (formed by asm_setup), so asm_apply on the unit vectors returns the
columns of K^{-1}.  Since both run the same Cholesky kernel, every result is also
checked against an independent float64 inverse on the host (numpy) and through the
residual K X - I; a third call at an order that is not a multiple of 32, after the
larger ones, would read the earlier calls' workspace if it were not cleared.  This file
is collected last.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def lib():
    import paper_2512_19536_gb300 as pd
    if not os.path.exists(pd.LIB_PATH):
        from paper_2512_19536_gb300.build import build
        build()
    return pd


def test_static_inverse_matches_asm_inverse_on_two_calls():
    import torch
    from synth.meshes import cartesian_square, isotropic_conductivity
    pd = lib()
    m = cartesian_square(4)
    ctx = pd.polydg_setup(m.vertices, m.cell_ptr, m.cell_vtx, isotropic_conductivity(16, 1.0), 2,
                          np.zeros(16, np.int32), 1.0, 0.1, 10.0)
    pc = pd.asm_setup(ctx, None, precision="fp64")       # one level, one subdomain: B = K^{-1}
    n = ctx.n_dofs
    K = torch.empty((n, n), dtype=torch.float64, device="cuda")
    Kinv_ref = torch.empty((n, n), dtype=torch.float64, device="cuda")
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    col = torch.empty(n, dtype=torch.float64, device="cuda")
    for j in range(n):
        e.zero_()
        e[j] = 1.0
        ctx.matvec(e, col)
        K[:, j] = col
        pd.asm_apply(pc, e, col)
        Kinv_ref[:, j] = col
    torch.cuda.synchronize()
    scale = Kinv_ref.abs().max().item()
    tol = 1e-12 * scale
    K_host = K.cpu().numpy()
    inv_host = np.linalg.inv(K_host)
    cond = np.linalg.cond(K_host)
    assert np.abs(Kinv_ref.cpu().numpy() - inv_host).max() <= 1e-12 * cond * np.abs(inv_host).max()

    # first call: a batch of K and 2K (inverses K^{-1} and K^{-1}/2)
    mats = torch.stack([K, 2.0 * K]).contiguous()
    pd.spd_inverse_static(mats, n, n, 2)
    torch.cuda.synchronize()
    assert (mats[0] - Kinv_ref).abs().max().item() <= tol
    assert (mats[1] - 0.5 * Kinv_ref).abs().max().item() <= 0.5 * tol

    # second call on fresh input, with a padded leading dimension: the shared static
    # workspace must not leak the first call's contents
    ld = n + 8
    padded = torch.zeros((1, n, ld), dtype=torch.float64, device="cuda")
    padded[0, :, :n] = K
    pd.spd_inverse_static(padded, n, ld, 1)
    torch.cuda.synchronize()
    assert (padded[0, :, :n] - Kinv_ref).abs().max().item() <= tol
    for X, A in ((mats[0], K_host), (mats[1], 2.0 * K_host), (padded[0, :, :n], K_host)):
        Xh = X.cpu().numpy()
        assert np.abs(A @ Xh - np.eye(n)).max() <= 1e-12 * cond
        assert np.abs(Xh - np.linalg.inv(A)).max() <= 1e-12 * cond * np.abs(np.linalg.inv(A)).max()

    # third call: the leading 40 x 40 block (40 is not a multiple of 32, so the workspace
    # stride differs from the calls before and their contents would show if not cleared)
    m40 = 40
    blk = K[:m40, :m40].contiguous().reshape(1, m40, m40).clone()
    pd.spd_inverse_static(blk, m40, m40, 1)
    torch.cuda.synchronize()
    A40 = K_host[:m40, :m40]
    X40 = blk[0].cpu().numpy()
    c40 = np.linalg.cond(A40)
    assert np.abs(A40 @ X40 - np.eye(m40)).max() <= 1e-12 * c40
    assert np.abs(X40 - np.linalg.inv(A40)).max() <= 1e-12 * c40 * np.abs(np.linalg.inv(A40)).max()


def test_static_inverse_rejects_oversize_and_indefinite():
    import torch
    pd = lib()
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PolyDGError) as err:
        pd._native._check(pd.load().polydg_spd_inverse_static(big.data_ptr(), 2048, 2048, 1, None))
    assert err.value.status == pd.POLYDG_EINVAL
    A = -torch.eye(8, dtype=torch.float64, device="cuda").reshape(1, 8, 8).contiguous()
    with pytest.raises(pd.PolyDGError) as err:
        pd.spd_inverse_static(A, 8, 8, 1)
    assert err.value.status == pd.POLYDG_ENOTSPD
    # host memory is refused before any launch
    host = torch.eye(8, dtype=torch.float64).reshape(1, 8, 8).contiguous()
    with pytest.raises(pd.PolyDGError) as err:
        pd._native._check(pd.load().polydg_spd_inverse_static(host.data_ptr(), 8, 8, 1, None))
    assert err.value.status == pd.POLYDG_EINVAL
