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


def test_rest_state_is_near_equilibrium():
    y0 = ionic.rest_state(-67.0)
    assert 0 < y0[0] < 1 and 0 < y0[1] < 1
    f = ionic.f_ion(np.array([-67.0]), y0[:, None])[0]
    assert abs(f) < 0.01                                   # uA/cm^2
    dy = ionic.dydt(np.array([-67.0]), y0[:, None])[:, 0]
    assert abs(dy[0]) < 1e-12 and abs(dy[1]) < 1e-12       # gates at steady state
    assert abs(dy[2]) < 1e-3 and abs(dy[3]) < 1e-3         # slow concentration drift


def test_rate_singularities_are_continuous():
    for v0 in (-30.0, -34.0):                              # removable points of alpha_m, alpha_n
        V = np.array([v0 - 1e-4, v0, v0 + 1e-4])
        am, _, an, _, _, _ = ionic.gating_rates(V)
        a = am if v0 == -30.0 else an
        assert np.all(np.isfinite(a))
        assert abs(a[1] - 0.5 * (a[0] + a[2])) < 1e-6


def test_first_step_uses_initial_state_for_extrapolation():
    d = small()
    md = monodomain.Monodomain(d, None)
    U0 = md.state.U.copy()
    md.state.U_prev[:] = 1e6                               # must be ignored on step 0
    b0, _ = md.rhs(md.state)
    md.state.U_prev[:] = U0
    b1, _ = md.rhs(md.state)
    assert np.array_equal(b0, b1)
