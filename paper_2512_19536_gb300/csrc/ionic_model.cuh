// Barreto-Cressman ionic model (Sec. 2; Cressman et al. 2009, Barreto and
// Cressman 2011), pointwise, in outward-current convention.  V in mV, t in ms,
// concentrations in mM; state y = (n, h, K_o, Na_i, Ca_i).
//   f(V, y)  = I_Na + I_K + I_Cl
//   I_Na     = (g_Na m_inf(V)^3 h + g_NaL)(V - E_Na)
//   I_K      = (g_K n^4 + g_AHP Ca_i/(1 + Ca_i) + g_KL)(V - E_K)
//   I_Cl     = g_ClL (V - E_Cl)
//   n' = phi(a_n (1 - n) - b_n n),  h' = phi(a_h (1 - h) - b_h h)
//   K_o'     = (gamma beta I_K - 2 beta I_pump - I_glia - I_diff) / tau
//   Na_i'    = (-gamma I_Na - 3 I_pump) / tau
//   Ca_i'    = -0.002 g_Ca (V - E_Ca) / (1 + exp(-(V + 25)/2.5)) - Ca_i / 80
// with K_i = 140 + (18 - Na_i), Na_o = 144 - beta (Na_i - 18) and Nernst
// potentials E = 26.64 ln(c_out / c_in).  The model's m(u, y) is -y'.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define BC_HD __host__ __device__ __forceinline__
#else
#define BC_HD inline
#endif

namespace polydg {
namespace bc {

constexpr double gNa = 100.0, gK = 40.0, gAHP = 0.01, gKL = 0.05, gNaL = 0.0175, gClL = 0.05;
constexpr double phi = 3.0, rho = 1.25, Gglia = 66.0, eps = 1.2, kbath = 4.0;
constexpr double gamma = 0.0445, beta = 7.0, tau = 1000.0;
constexpr double Cli = 6.0, Clo = 130.0, gCa = 0.1, ECa = 120.0, RTF = 26.64;
constexpr int kStates = 5;

// x / (1 - exp(-x/s)); the removable point x = 0 takes its first-order limit.
BC_HD double lin_exp(double x, double s) {
    if (fabs(x / s) < 1e-6) return s * (1.0 + 0.5 * x / s);
    return x / (1.0 - exp(-x / s));
}

struct Rates { double an, bn, ah, bh; };

BC_HD Rates gate_rates(double V) {
    Rates r;
    r.an = 0.01 * lin_exp(V + 34.0, 10.0);
    r.bn = 0.125 * exp(-(V + 44.0) / 80.0);
    r.ah = 0.07 * exp(-(V + 44.0) / 20.0);
    r.bh = 1.0 / (1.0 + exp(-(V + 14.0) / 10.0));
    return r;
}

struct Currents { double INa, IK, ICl; };

BC_HD Currents currents(double V, double n, double h, double Ko, double Nai, double Cai) {
    const double am = 0.1 * lin_exp(V + 30.0, 10.0);
    const double bm = 4.0 * exp(-(V + 55.0) / 18.0);
    const double minf = am / (am + bm);
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    const double ENa = RTF * log(Nao / Nai);
    const double EK = RTF * log(Ko / Ki);
    const double ECl = RTF * log(Cli / Clo);
    Currents c;
    c.INa = (gNa * minf * minf * minf * h + gNaL) * (V - ENa);
    c.IK = (gK * (n * n) * (n * n) + gAHP * Cai / (1.0 + Cai) + gKL) * (V - EK);
    c.ICl = gClL * (V - ECl);
    return c;
}

// One explicit Euler step y <- y + dt y'(V, y).
BC_HD void euler(double V, double dt, double& n, double& h, double& Ko, double& Nai, double& Cai) {
    const Rates r = gate_rates(V);
    const Currents c = currents(V, n, h, Ko, Nai, Cai);
    const double pump = rho / (1.0 + exp((25.0 - Nai) / 3.0)) / (1.0 + exp(5.5 - Ko));
    const double glia = Gglia / (1.0 + exp((18.0 - Ko) / 2.5));
    const double diff = eps * (Ko - kbath);
    const double dn = phi * (r.an * (1.0 - n) - r.bn * n);
    const double dh = phi * (r.ah * (1.0 - h) - r.bh * h);
    const double dKo = (gamma * beta * c.IK - 2.0 * beta * pump - glia - diff) / tau;
    const double dNa = (-gamma * c.INa - 3.0 * pump) / tau;
    const double dCa = -0.002 * gCa * (V - ECa) / (1.0 + exp(-(V + 25.0) / 2.5)) - Cai / 80.0;
    n += dt * dn;
    h += dt * dh;
    Ko += dt * dKo;
    Nai += dt * dNa;
    Cai += dt * dCa;
}

// Rest state at potential V0: gates at steady state, K_o = 4, Na_i = 18, Ca_i = 0.
BC_HD void rest_state(double V0, double* y) {
    const Rates r = gate_rates(V0);
    y[0] = r.an / (r.an + r.bn);
    y[1] = r.ah / (r.ah + r.bh);
    y[2] = 4.0;
    y[3] = 18.0;
    y[4] = 0.0;
}

}  // namespace bc
}  // namespace polydg
