"""Pins of oracle.monodomain and oracle.ionic (no GPU)."""
import numpy as np
import scipy.linalg as sla

from oracle import assembly, ionic, monodomain
from synth.meshes import cartesian_square, isotropic_conductivity


def small(dt=0.05):
    m = cartesian_square(4)
    return assembly.assemble(m, 2, isotropic_conductivity(16, 1.0), 10.0, 1.0, dt)


def test_linear_scheme_conserves_mean():
    # f = 0, no stimulus, Neumann: 1^T M U is invariant under Crank-Nicolson.
    d = small()
    md = monodomain.Monodomain(d, None, ion=False)
    U = np.random.default_rng(0).standard_normal(d.n_dofs)
    md.state = monodomain.State(U, U.copy(), md.state.y, 0)
    one = np.zeros(d.n_dofs); one[::d.n_p] = 1.0
    m0 = one @ d.M @ U
    for _ in range(5):
        st = md.step()
    assert abs(one @ d.M @ st.U - m0) < 1e-12 * np.abs(U).max()


def test_eigenmode_amplification_factor():
    # A v = lam M v:  K v' = (M - dt/2 A) v  =>  v' = (1 - dt lam/2)/(1 + dt lam/2) v.
    dt = 0.05
    d = small(dt)
    lam, vecs = sla.eigh(d.A.toarray(), d.M.toarray())
    j = len(lam) // 2
    v = vecs[:, j]
    md = monodomain.Monodomain(d, None, ion=False)
    md.state = monodomain.State(v.copy(), v.copy(), md.state.y, 0)
    st = md.step()
    g = (1 - dt * lam[j] / 2) / (1 + dt * lam[j] / 2)
    assert np.allclose(st.U, g * v, atol=1e-10 * np.abs(v).max())


def test_first_step_uses_initial_state_for_extrapolation():
    d = small()
    md = monodomain.Monodomain(d, None)
    U0 = md.state.U.copy()
    md.state.U_prev[:] = 1e6                               # must be ignored on step 0
    b0, _ = md.rhs(md.state)
    md.state.U_prev[:] = U0
    b1, _ = md.rhs(md.state)
    assert np.array_equal(b0, b1)


# ---- the ionic state in the DG basis (Eq. fully-discrete-1, second line)

def test_modal_ionic_state_equals_nodal_on_uniform_fields():
    # A spatially uniform potential and state stay uniform (no stimulus, Neumann), and a
    # constant lies in every P^p(K): the projection M_K^{-1} sum_q w_q d_q phi(x_q) of a
    # uniform increment d is d times the constant mode, so the modal and the per-node
    # forms produce the same states.  A missing M_K^{-1}, weight or dt breaks it.
    d = small()
    runs = {}
    for form in ("nodal", "modal"):
        md = monodomain.Monodomain(d, None, u0=-50.0, ionic_form=form)
        for _ in range(5):
            st = md.step()
        runs[form] = st
    yn, ym = runs["nodal"].y, runs["modal"].y
    assert np.allclose(ym, yn, rtol=1e-12, atol=1e-14)
    assert np.allclose(runs["modal"].U, runs["nodal"].U, rtol=1e-12, atol=1e-12)
    Y = runs["modal"].Y.reshape(5, -1, d.n_p)
    assert np.allclose(Y[:, :, 1:], 0.0, atol=1e-13)          # still constants


def test_modal_ionic_update_balances_cell_integrals():
    # Under a Gaussian stimulus the fields vary in space.  Since 1 is in P^p(K), the
    # projected update keeps every cell's integral balance exactly:
    #   int_K y_h^{k+1} - int_K y_h^k = sum_{q in K} w_q dt y'(u^k(x_q), y_h^k(x_q)),
    # with the integrals of the degree-p fields taken by the (exact) element rule.
    from synth import stimulus_params
    d = small()
    md = monodomain.Monodomain(d, stimulus_params(3), ionic_form="modal")
    nodes, nc, n_p = md.nodes, d.mesh.n_cells, d.n_p
    for _ in range(3):
        before = md.state
        after = md.step()
        u_nodes = monodomain.nodal_values(nodes, before.U, n_p)
        yq = np.stack([monodomain.nodal_values(nodes, before.Y[l], n_p) for l in range(5)])
        incr = d.dt * ionic.dydt(u_nodes, yq)
        for l in range(5):
            cell_int = lambda v: np.bincount(nodes.cell, weights=nodes.w * v, minlength=nc)
            lhs = cell_int(after.y[l]) - cell_int(yq[l])
            rhs = cell_int(incr[l])
            assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-13 * np.abs(yq[l]).max())
    # the fields really vary: the modal form differs from the per-node one
    nodal = monodomain.Monodomain(d, stimulus_params(3))
    for _ in range(3):
        ref = nodal.step()
    assert np.abs(after.y - ref.y).max() > 1e-12
