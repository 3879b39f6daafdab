"""Pins of the ionic model and of its coupling into the Crank-Nicolson step (no GPU).

Eq. fully-discrete-1: K_h U^{k+1} = (chi_m C_m M - dt/2 A) U^k - chi_m dt I^{k+1} + dt F,
with I^{k+1}_i = sum_q w_q f(u~(x_q), y^{k+1}_q) phi_i(x_q), u~ = 3/2 U^k - 1/2 U^{k-1}
(U^0 on the first step) and y^{k+1} = y^k - dt m(u^k, y^k) at the nodes.

The coupling tests replace the Barreto-Cressman current by currents whose discrete
solution has a closed form, so a wrong sign or coefficient of the ion term, a wrong
extrapolation, a dropped chi_m or an ion current taken from the old state fails them:
  * a linear current g u on a generalised eigenmode A v = lam M v gives the two-step
    recurrence (chi + dt lam/2) a_{k+1} = (chi - dt lam/2) a_k - chi dt g u~_k;
  * an affine current g (u - E) on the constant mode (A 1 = 0) gives
    a_{k+1} = a_k - dt g (u~_k - E);
  * with a nonlinear current and the state frozen, a spatially uniform field follows
    u' = -f(u) (chi_m C_m = chi_m, C_m = 1) to second order in dt (the midpoint
    extrapolation); the exact solution of w' = -g w - c w^3 is a Bernoulli closed form;
  * with the model's own explicit Euler state update the coupled scheme is first order
    (the state is advanced to t^{k+1} with the slope at t^k).
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import erf

from oracle import assembly, ionic, monodomain
from synth.meshes import cartesian_square, isotropic_conductivity


def disc(n=4, p=2, chi=0.7, dt=0.05):
    m = cartesian_square(n)
    return assembly.assemble(m, p, isotropic_conductivity(n * n, 1.0), 10.0, chi, dt)


def const_mode(d):
    one = np.zeros(d.n_dofs)
    one[::d.n_p] = 1.0                       # phi_0 = 1 on every cell
    return one


def frozen(monkeypatch, f):
    """Current f(V, y) and a state update that leaves y unchanged."""
    monkeypatch.setattr(ionic, "f_ion", f)
    monkeypatch.setattr(ionic, "euler_step", lambda V, y, dt: y)


def eigen_run(monkeypatch, cls=monodomain.Monodomain, current=None):
    """Largest deviation, over two eigenmodes and six steps, of the oracle's U^k from the
    closed-form recurrence of a linear current g u."""
    chi, dt, g = 0.7, 0.05, 3.0
    d = disc(chi=chi, dt=dt)
    lam, vecs = sla.eigh(d.A.toarray(), d.M.toarray())
    worst = 0.0
    for j in (5, len(lam) // 2):
        v = vecs[:, j]
        frozen(monkeypatch, current or (lambda V, y: g * V))
        md = cls(d, None)
        md.state = monodomain.State(v.copy(), v.copy(), md.state.y, 0)
        a = [1.0]
        for k in range(6):
            u_ext = a[k] if k == 0 else 1.5 * a[k] - 0.5 * a[k - 1]
            a.append(((chi - 0.5 * dt * lam[j]) * a[k] - chi * dt * g * u_ext)
                     / (chi + 0.5 * dt * lam[j]))
            st = md.step()
            worst = max(worst, np.abs(st.U - a[-1] * v).max() / np.abs(v).max())
        # the ion term is visible: without it the amplitude differs by far more
        plain = ((chi - 0.5 * dt * lam[j]) / (chi + 0.5 * dt * lam[j])) ** 6
        assert abs(a[-1] - plain) > 1e-3 * abs(plain) + 1e-6
    return worst


def test_linear_current_on_an_eigenmode_follows_the_two_step_recurrence(monkeypatch):
    assert eigen_run(monkeypatch) < 1e-11


class _ExtrapolatedToTheEnd(monodomain.Monodomain):
    """Planted mistake: u~ = 2 U^k - U^{k-1} (extrapolation to t^{k+1})."""

    def rhs(self, st):
        if st.k > 0:
            st = monodomain.State(st.U, 2.0 * st.U_prev - st.U, st.y, st.k, st.Y)
        return super().rhs(st)


@pytest.mark.parametrize("mistake", ["sign", "extrapolation", "chi"])
def test_planted_mistakes_in_the_ion_term_fail_the_recurrence(monkeypatch, mistake):
    g, chi = 3.0, 0.7
    if mistake == "sign":              # + chi dt I
        dev = eigen_run(monkeypatch, current=lambda V, y: -g * V)
    elif mistake == "chi":             # - dt I (chi_m dropped)
        dev = eigen_run(monkeypatch, current=lambda V, y: g * V / chi)
    else:
        dev = eigen_run(monkeypatch, cls=_ExtrapolatedToTheEnd)
    assert dev > 1e-6


def test_affine_current_on_the_constant_mode(monkeypatch):
    chi, dt, g, E = 0.7, 0.05, 2.0, -60.0
    d = disc(chi=chi, dt=dt)
    one = const_mode(d)
    frozen(monkeypatch, lambda V, y: g * (V - E))
    md = monodomain.Monodomain(d, None, u0=-67.0)
    a = [-67.0]
    for k in range(8):
        u_ext = a[k] if k == 0 else 1.5 * a[k] - 0.5 * a[k - 1]
        a.append(a[k] - dt * g * (u_ext - E))
        st = md.step()
        assert np.allclose(st.U, a[-1] * one, rtol=0, atol=1e-11 * 67.0), k


def test_the_current_sees_u_tilde_and_the_updated_state(monkeypatch):
    # spies: the state update receives u^k at the nodes, the current receives u~ and
    # the state the update returned
    d = disc()
    rng = np.random.default_rng(3)
    seen = {}

    def upd(V, y, dt):
        seen["V_update"] = V.copy()
        return y + 0.25                       # any change of the state

    def cur(V, y):
        seen["V_current"] = V.copy()
        seen["y_current"] = y.copy()
        return np.zeros_like(V)

    monkeypatch.setattr(ionic, "euler_step", upd)
    monkeypatch.setattr(ionic, "f_ion", cur)
    md = monodomain.Monodomain(d, None)
    U1, U0 = rng.standard_normal(d.n_dofs), rng.standard_normal(d.n_dofs)
    y0 = md.state.y.copy()
    for k, (Uk, Uprev) in enumerate([(U0, U0), (U1, U0)]):
        md.state = monodomain.State(Uk, Uprev, y0, k)
        md.rhs(md.state)
        nodes = md.nodes
        assert np.allclose(seen["V_update"], monodomain.nodal_values(nodes, Uk, d.n_p), atol=1e-13)
        ext = Uk if k == 0 else 1.5 * Uk - 0.5 * Uprev
        assert np.allclose(seen["V_current"], monodomain.nodal_values(nodes, ext, d.n_p), atol=1e-13)
        assert np.array_equal(seen["y_current"], y0 + 0.25)


def test_a_state_dependent_current_uses_y_k_plus_1(monkeypatch):
    # f = c y_0 with y_0 growing by s dt per step: on the constant mode
    # a_{k+1} = a_k - dt c (y0 + (k + 1) s dt).  The old state gives a_k - dt c (y0 + k s dt).
    chi, dt, c, s = 0.7, 0.05, 1.5, 4.0
    d = disc(chi=chi, dt=dt)
    one = const_mode(d)
    monkeypatch.setattr(ionic, "f_ion", lambda V, y: c * y[0])
    monkeypatch.setattr(ionic, "euler_step", lambda V, y, dt_: y + s * dt_)
    md = monodomain.Monodomain(d, None, u0=-67.0)
    y00 = md.state.y[0, 0]
    a = -67.0
    for k in range(5):
        a = a - dt * c * (y00 + (k + 1) * s * dt)
        st = md.step()
        assert np.allclose(st.U, a * one, rtol=0, atol=1e-11 * 67.0), k


def bernoulli(w0, g, c, t):
    """Exact solution of w' = -g w - c w^3, w(0) = w0."""
    e = np.exp(-g * t)
    return w0 * e / np.sqrt(1.0 + (c * w0 * w0 / g) * (1.0 - e * e))


def uniform_run(monkeypatch, dt, T, f, u0, update=None):
    d = disc(n=2, p=1, chi=0.7, dt=dt)
    if update is None:
        frozen(monkeypatch, f)
    else:
        monkeypatch.setattr(ionic, "f_ion", f)
        monkeypatch.setattr(ionic, "euler_step", update)
    md = monodomain.Monodomain(d, None, u0=u0)
    for _ in range(int(round(T / dt))):
        st = md.step()
    vals = st.U[::d.n_p]
    assert np.ptp(vals) < 1e-9 * abs(vals).max()      # the field stays uniform
    assert np.abs(st.U.reshape(-1, d.n_p)[:, 1:]).max() < 1e-9 * abs(vals).max()
    return vals[0]


def test_uniform_field_is_second_order_with_a_frozen_state(monkeypatch):
    g, c, E, u0, T = 1.0, 0.001, -60.0, -50.0, 1.0
    f = lambda V, y: g * (V - E) + c * (V - E) ** 3
    exact = E + bernoulli(u0 - E, g, c, T)
    errs = [abs(uniform_run(monkeypatch, dt, T, f, u0) - exact) for dt in (0.05, 0.025, 0.0125, 0.00625)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.6 for r in ratios), (errs, ratios)


def test_extrapolation_to_the_step_end_is_only_first_order(monkeypatch):
    # the same run with the planted u~ = 2 U^k - U^{k-1}: the order test above fails
    g, c, E, u0, T = 1.0, 0.001, -60.0, -50.0, 1.0
    f = lambda V, y: g * (V - E) + c * (V - E) ** 3
    exact = E + bernoulli(u0 - E, g, c, T)
    errs = []
    for dt in (0.05, 0.025, 0.0125, 0.00625):
        d = disc(n=2, p=1, chi=0.7, dt=dt)
        frozen(monkeypatch, f)
        md = _ExtrapolatedToTheEnd(d, None, u0=u0)
        for _ in range(int(round(T / dt))):
            st = md.step()
        errs.append(abs(st.U[0] - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert not all(3.6 < r < 4.6 for r in ratios), (errs, ratios)


def test_real_model_uniform_field_is_first_order(monkeypatch):
    # the model's explicit Euler update of the state (first order) bounds the scheme
    u0, T = -55.0, 2.0
    runs = {dt: uniform_run(monkeypatch, dt, T, ionic.f_ion, u0, update=ionic.euler_step)
            for dt in (0.1, 0.05, 0.025, 0.0125, 0.003125)}
    ref = runs[0.003125]
    errs = [abs(runs[dt] - ref) for dt in (0.1, 0.05, 0.025, 0.0125)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.6 < r < 2.6 for r in ratios), (errs, ratios)


def test_stimulus_enters_with_dt_at_the_midpoint():
    # b(stimulus) - b(none) = dt F while t^{k+1/2} < duration and 0 afterwards, and the
    # constant-mode sum of F is the Gaussian's integral over the unit square (erf form)
    dt = 0.05
    d = disc(n=16, p=2, chi=1.0, dt=dt)
    stim = {"x0": 0.45, "y0": 0.55, "amplitude": 7.0, "width": 0.12, "duration": 0.1}
    on = monodomain.Monodomain(d, stim)
    off = monodomain.Monodomain(d, None)
    w = stim["width"]
    s = w * np.sqrt(np.pi / 2.0)
    ix = s * (erf((1 - stim["x0"]) / (np.sqrt(2) * w)) + erf(stim["x0"] / (np.sqrt(2) * w)))
    iy = s * (erf((1 - stim["y0"]) / (np.sqrt(2) * w)) + erf(stim["y0"] / (np.sqrt(2) * w)))
    total = stim["amplitude"] * ix * iy
    for k, active in ((0, True), (1, True), (2, False), (3, False)):   # t_half = 0.025, 0.075, ...
        st = monodomain.State(off.state.U, off.state.U, off.state.y, k)
        b_on, _ = on.rhs(st)
        b_off, _ = off.rhs(st)
        diff = b_on - b_off
        if active:
            assert abs(diff[::d.n_p].sum() / dt - total) < 1e-5 * total
            assert np.allclose(diff, dt * on.F, rtol=0, atol=1e-15 * total)
        else:
            assert np.array_equal(diff, np.zeros_like(diff))


# ---- the model itself

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


def test_nernst_potentials_and_current_reversal():
    # each current vanishes at its own reversal potential: with every conductance but
    # one channel's dropped, f(E_X) = 0, and E = 26.64 ln(c_out / c_in)
    y = ionic.rest_state(-67.0)[:, None].copy()
    Ki = 140.0 + (18.0 - y[3, 0])
    E_K = 26.64 * np.log(y[2, 0] / Ki)
    _, I_K, _ = ionic.currents(np.array([E_K]), y)
    assert abs(I_K[0]) < 1e-12
    Nao = 144.0 - 7.0 * (y[3, 0] - 18.0)
    E_Na = 26.64 * np.log(Nao / y[3, 0])
    I_Na, _, _ = ionic.currents(np.array([E_Na]), y)
    assert abs(I_Na[0]) < 1e-12
    E_Cl = 26.64 * np.log(6.0 / 130.0)
    _, _, I_Cl = ionic.currents(np.array([E_Cl]), y)
    assert abs(I_Cl[0]) < 1e-12
