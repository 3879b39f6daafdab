"""Barreto-Cressman ionic model, pointwise (FP64).

The paper (Sec. 2) couples the monodomain equation to the Barreto-Cressman
model: a Hodgkin-Huxley-type membrane with intracellular sodium,
extracellular potassium and intracellular calcium concentrations and their
gating variables, and defers the equations to the cited publications.  This
module restates that model (Cressman et al. 2009; Barreto and Cressman 2011)
in outward-current convention:

    state y = (n, h, K_o, Na_i, Ca_i); V in mV, t in ms, concentrations in mM.
    f(V, y)  = I_Na + I_K + I_Cl                               (uA/cm^2, outward)
    I_Na     = (g_Na m_inf^3 h + g_NaL) (V - E_Na)
    I_K      = (g_K n^4 + g_AHP Ca_i/(1 + Ca_i) + g_KL) (V - E_K)
    I_Cl     = g_ClL (V - E_Cl)
    dn/dt    = phi (alpha_n (1 - n) - beta_n n),   dh/dt likewise
    dK_o/dt  = (gamma beta I_K - 2 beta I_pump - I_glia - I_diff) / tau
    dNa_i/dt = (-gamma I_Na - 3 I_pump) / tau
    dCa_i/dt = -0.002 g_Ca (V - E_Ca) / (1 + exp(-(V + 25)/2.5)) - Ca_i / 80
with K_i = 140 + (18 - Na_i), Na_o = 144 - beta (Na_i - 18), Nernst
potentials E = 26.64 ln(c_out / c_in) (E_Cl with Cl_i = 6, Cl_o = 130), and
the pump, glial buffering and bath diffusion terms below.  The paper's
m(u, y) of Eq. monodomain is -dy/dt.

PARITY UNPINNED as physics: the cited publications are not available to
check these constants against.  What is pinned (tests/test_oracle_ionic.py):
the rest state at the paper's u0 = -67 mV is close to equilibrium, gating
steady states lie in (0, 1), the rate functions' removable singularities are
evaluated by their limits, and each current vanishes at its Nernst reversal
potential.  The coupling of f and of the state update into the time step is
pinned there too, with currents whose discrete solution has a closed form.
"""
import numpy as np

G_NA, G_K, G_AHP, G_KL, G_NAL, G_CLL = 100.0, 40.0, 0.01, 0.05, 0.0175, 0.05
PHI, RHO, G_GLIA, EPS, K_BATH = 3.0, 1.25, 66.0, 1.2, 4.0
GAMMA, BETA, TAU = 0.0445, 7.0, 1000.0
CL_I, CL_O, G_CA, E_CA = 6.0, 130.0, 0.1, 120.0
NERNST = 26.64
N_STATE = 5


def _vtrap(x, y):
    """x / (1 - exp(-x / y)), with the limit y at x = 0."""
    x = np.asarray(x, float)
    small = np.abs(x / y) < 1e-6
    safe = np.where(small, 1.0, x)
    return np.where(small, y * (1.0 + 0.5 * x / y), safe / (1.0 - np.exp(-safe / y)))


def gating_rates(V):
    V = np.asarray(V, float)
    alpha_m = 0.1 * _vtrap(V + 30.0, 10.0)
    beta_m = 4.0 * np.exp(-(V + 55.0) / 18.0)
    alpha_n = 0.01 * _vtrap(V + 34.0, 10.0)
    beta_n = 0.125 * np.exp(-(V + 44.0) / 80.0)
    alpha_h = 0.07 * np.exp(-(V + 44.0) / 20.0)
    beta_h = 1.0 / (1.0 + np.exp(-(V + 14.0) / 10.0))
    return alpha_m, beta_m, alpha_n, beta_n, alpha_h, beta_h


def currents(V, y):
    """(I_Na, I_K, I_Cl) outward, for potentials V [m] and states y [5, m]."""
    n, h, Ko, Nai, Cai = y
    am, bm, _, _, _, _ = gating_rates(V)
    m_inf = am / (am + bm)
    Ki = 140.0 + (18.0 - Nai)
    Nao = 144.0 - BETA * (Nai - 18.0)
    E_Na = NERNST * np.log(Nao / Nai)
    E_K = NERNST * np.log(Ko / Ki)
    E_Cl = NERNST * np.log(CL_I / CL_O)
    I_Na = (G_NA * m_inf ** 3 * h + G_NAL) * (V - E_Na)
    I_K = (G_K * n ** 4 + G_AHP * Cai / (1.0 + Cai) + G_KL) * (V - E_K)
    I_Cl = G_CLL * (V - E_Cl)
    return I_Na, I_K, I_Cl


def f_ion(V, y):
    """Total outward ionic current f(u, y) of Eq. monodomain."""
    I_Na, I_K, I_Cl = currents(V, y)
    return I_Na + I_K + I_Cl


def dydt(V, y):
    """Right-hand side dy/dt = -m(u, y), shape [5, m]."""
    n, h, Ko, Nai, Cai = y
    _, _, an, bn, ah, bh = gating_rates(V)
    I_Na, I_K, _ = currents(V, y)
    I_pump = RHO / (1.0 + np.exp((25.0 - Nai) / 3.0)) / (1.0 + np.exp(5.5 - Ko))
    I_glia = G_GLIA / (1.0 + np.exp((18.0 - Ko) / 2.5))
    I_diff = EPS * (Ko - K_BATH)
    dn = PHI * (an * (1.0 - n) - bn * n)
    dh = PHI * (ah * (1.0 - h) - bh * h)
    dKo = (GAMMA * BETA * I_K - 2.0 * BETA * I_pump - I_glia - I_diff) / TAU
    dNai = (-GAMMA * I_Na - 3.0 * I_pump) / TAU
    dCai = (-0.002 * G_CA * (V - E_CA) / (1.0 + np.exp(-(V + 25.0) / 2.5)) - Cai / 80.0)
    return np.stack([dn, dh, dKo, dNai, dCai])


def rest_state(V0=-67.0):
    """Gating variables at their steady state for V0; K_o = 4, Na_i = 18, Ca_i = 0."""
    _, _, an, bn, ah, bh = gating_rates(np.array([V0]))
    return np.array([an[0] / (an[0] + bn[0]), ah[0] / (ah[0] + bh[0]), 4.0, 18.0, 0.0])


def euler_step(V, y, dt):
    """Explicit update y^{k+1} = y^k - dt m(u^k, y^k) (Eq. fully-discrete-1, second line,
    taken per quadrature node)."""
    return y + dt * dydt(V, y)
