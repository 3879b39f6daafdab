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
// The device forms below evaluate the same expressions with the exponentials of V
// and of K_o regrouped (exp(a + b) = exp(a) exp(b)) and divisions by constants taken
// as products with reciprocals; results differ from the plain forms by rounding only.
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

// Constants of the per-node update that do not depend on the state (host-computed):
// the membrane-potential exponentials of the rates are all exp(-(V + c)/s) with
// s in {10, 20, 80, 2.5} -- integer divisors of 80 -- except beta_m (s = 18), so with
// E = exp(-V/80) they are exp(-c/s) E^(80/s); likewise the pump's exp(5.5 - K_o) and
// the glial exp((18 - K_o)/2.5) are e^5.5 X^5 and e^7.2 X^2 with X = exp(-K_o/5).
struct NodeConsts {
    double an, bn, ah, bh, am, ca;   // exp(-3.4), 0.125 exp(-0.55), 0.07 exp(-2.2), exp(-1.4), exp(-3), exp(-10)
    double pump, glia;               // exp(5.5), exp(7.2)
    double ECl;                      // RTF ln(Cl_i / Cl_o)
};

inline NodeConsts node_consts() {
    NodeConsts k;
    k.an = std::exp(-3.4); k.bn = 0.125 * std::exp(-0.55); k.ah = 0.07 * std::exp(-2.2);
    k.bh = std::exp(-1.4); k.am = std::exp(-3.0); k.ca = std::exp(-10.0);
    k.pump = std::exp(5.5); k.glia = std::exp(7.2);
    k.ECl = RTF * std::log(Cli / Clo);
    return k;
}

// x / (1 - ex) for ex = exp(-x/s) given; the removable point x = 0 takes its limit.
BC_HD double lin_exp_given(double x, double s, double ex) {
    if (fabs(x) < 1e-6 * s) return s + 0.5 * x;
    return x / (1.0 - ex);
}

// Divisions by constants are multiplications by their reciprocals, and the pump's two
// denominators share one division: the fp64 pipe, not memory, bounds the node update.
constexpr double kInv80 = 1.0 / 80.0, kInv18 = 1.0 / 18.0, kInv3 = 1.0 / 3.0, kInv5 = 1.0 / 5.0;
constexpr double kInvTau = 1.0 / tau, kInv10 = 1.0 / 10.0;

// I_Na + I_K + I_Cl at potential V for state (n, h, K_o, Na_i, Ca_i).
BC_HD double total_current(const NodeConsts& k, double V, double n, double h, double Ko, double Nai,
                           double Cai) {
    const double am = 0.1 * lin_exp_given(V + 30.0, 10.0, exp(-(V + 30.0) * kInv10));
    const double bm = 4.0 * exp(-(V + 55.0) * kInv18);
    const double minf = am / (am + bm);
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    const double INa = (gNa * minf * minf * minf * h + gNaL) * (V - RTF * log(Nao / Nai));
    const double IK = (gK * (n * n) * (n * n) + gAHP * Cai / (1.0 + Cai) + gKL) * (V - RTF * log(Ko / Ki));
    return INa + IK + gClL * (V - k.ECl);
}

// y'(V, y) of the Sec. 2 model (= -m(u, y)) at one point: d[0..4] for n, h, K_o, Na_i, Ca_i.
BC_HD void rates(const NodeConsts& k, double V, double n, double h, double Ko, double Nai, double Cai,
                 double* d) {
    const double E = exp(-V * kInv80);
    const double E2 = E * E, E4 = E2 * E2, E8 = E4 * E4, E16 = E8 * E8, E32 = E16 * E16;
    const double an = 0.01 * lin_exp_given(V + 34.0, 10.0, k.an * E8);
    const double bn = k.bn * E;
    const double ah = k.ah * E4;
    const double bh = 1.0 / (1.0 + k.bh * E8);
    const double am = 0.1 * lin_exp_given(V + 30.0, 10.0, k.am * E8);
    const double bm = 4.0 * exp(-(V + 55.0) * kInv18);
    const double minf = am / (am + bm);
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    const double INa = (gNa * minf * minf * minf * h + gNaL) * (V - RTF * log(Nao / Nai));
    const double IK = (gK * (n * n) * (n * n) + gAHP * Cai / (1.0 + Cai) + gKL) * (V - RTF * log(Ko / Ki));
    const double X = exp(-Ko * kInv5), X2 = X * X, X5 = X2 * X2 * X;
    const double pump = rho / ((1.0 + exp((25.0 - Nai) * kInv3)) * (1.0 + k.pump * X5));
    const double glia = Gglia / (1.0 + k.glia * X2);
    const double diff = eps * (Ko - kbath);
    const double dn = phi * (an * (1.0 - n) - bn * n);
    const double dh = phi * (ah * (1.0 - h) - bh * h);
    const double dKo = (gamma * beta * IK - 2.0 * beta * pump - glia - diff) * kInvTau;
    const double dNa = (-gamma * INa - 3.0 * pump) * kInvTau;
    const double dCa = -0.002 * gCa * (V - ECa) / (1.0 + k.ca * E32) - Cai * kInv80;
    d[0] = dn;
    d[1] = dh;
    d[2] = dKo;
    d[3] = dNa;
    d[4] = dCa;
}

// One explicit Euler step y <- y + dt y'(V, y) (Sec. 2 model, per quadrature node).
BC_HD void euler(const NodeConsts& k, double V, double dt, double& n, double& h, double& Ko,
                 double& Nai, double& Cai) {
    double d[5];
    rates(k, V, n, h, Ko, Nai, Cai, d);
    n += dt * d[0];
    h += dt * d[1];
    Ko += dt * d[2];
    Nai += dt * d[3];
    Cai += dt * d[4];
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
