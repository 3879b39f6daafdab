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
// and of K_o regrouped (exp(a + b) = exp(a) exp(b), one exponential per potential),
// the reciprocals of a node batched into one division, and the Nernst potentials after
// an Euler step updated from the old ones; the per-node update also carries E_Na, E_K
// and the two concentration exponentials from one step to the next (NodeCache) and
// takes exp(-u~/720) from exp(-u/720).  Results differ from the plain forms by rounding
// only.
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

// |x| < t for t > 0, as an integer comparison of the bit patterns (non-negative doubles
// order like their patterns; NaN and infinities compare false as with fabs): on GB300 a
// double comparison takes a slot of the narrow fp64 pipe that bounds the node update.
BC_HD bool abs_below(double x, double t) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)(__double_as_longlong(x) & 0x7fffffffffffffffLL) <
           (unsigned long long)__double_as_longlong(t);
#else
    return std::fabs(x) < t;
#endif
}

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

// Constants of the per-node update that do not depend on the state (host-computed).
// Every membrane-potential exponential of the rates is exp(-(V + c)/s) with s in
// {10, 18, 20, 80, 2.5}, all of which divide 720 into integers (72, 40, 36, 9, 288), so
// with B = exp(-V/720) they are exp(-c/s) B^(720/s): one exponential per potential, the
// powers by repeated squaring (relative error <= ~300 ulp, far below the model's use).
// Likewise the pump's exp(5.5 - K_o) and the glial exp((18 - K_o)/2.5) are e^5.5 X^5 and
// e^7.2 X^2 with X = exp(-K_o/5).
struct NodeConsts {
    double an, bn, ah, bh, am, bm, ca;   // exp(-3.4), 0.125 exp(-0.55), 0.07 exp(-2.2), exp(-1.4),
                                         // exp(-3), 4 exp(-55/18), exp(-10)
    double pump, glia;                   // exp(5.5), exp(7.2)
    double ECl;                          // RTF ln(Cl_i / Cl_o)
};

inline NodeConsts node_consts() {
    NodeConsts k;
    k.an = std::exp(-3.4); k.bn = 0.125 * std::exp(-0.55); k.ah = 0.07 * std::exp(-2.2);
    k.bh = std::exp(-1.4); k.am = std::exp(-3.0); k.bm = 4.0 * std::exp(-55.0 / 18.0);
    k.ca = std::exp(-10.0);
    k.pump = std::exp(5.5); k.glia = std::exp(7.2);
    k.ECl = RTF * std::log(Cli / Clo);
    return k;
}

// exp(-V/s) for s = 10, 18, 20, 80, 2.5 from B = exp(-V/720) (kept in B).
struct VPowers { double e10, e18, e20, e80, e25, B; };

BC_HD VPowers vpowers_from(double B) {
    const double B2 = B * B, B4 = B2 * B2, B8 = B4 * B4, B16 = B8 * B8, B32 = B16 * B16;
    const double B64 = B32 * B32, B256 = (B64 * B64) * (B64 * B64);
    VPowers p;
    p.e80 = B8 * B;
    p.e20 = B32 * B4;
    p.e18 = B32 * B8;
    p.e10 = B64 * B8;
    p.e25 = B256 * B32;
    p.B = B;
    return p;
}

BC_HD VPowers vpowers(double V) { return vpowers_from(exp(-V * (1.0 / 720.0))); }

// exp(-V/10) and exp(-V/18) only (the sodium gate of the current), from B = exp(-V/720).
BC_HD void vpowers_m_from(double B, double& e10, double& e18) {
    const double B2 = B * B, B4 = B2 * B2, B8 = B4 * B4, B16 = B8 * B8, B32 = B16 * B16;
    e18 = B32 * B8;
    e10 = (B32 * B32) * B8;
}

BC_HD void vpowers_m(double V, double& e10, double& e18) {
    vpowers_m_from(exp(-V * (1.0 / 720.0)), e10, e18);
}

// exp(a): for |a| < 2^-18 the Taylor polynomial of degree 3 (remainder < a^4 / 4! < 1e-23
// relative), for |a| < 2^-6 that of degree 7 (< a^8 / 8! < 1e-19), else the library
// function.  For the ratio of an exponential at two nearby arguments (the concentrations
// move by ~1e-6 relative per step, the potential by up to a few mV).
BC_HD double exp_small(double a) {
    if (abs_below(a, 0x1p-18)) return 1.0 + a * (1.0 + a * (0.5 + a * (1.0 / 6.0)));
    if (abs_below(a, 0x1p-6))
        return 1.0 + a * (1.0 + a * (0.5 + a * (1.0 / 6.0 + a * (1.0 / 24.0 + a * (1.0 / 120.0 +
                     a * (1.0 / 720.0 + a * (1.0 / 5040.0)))))));
    return exp(a);
}

// Reciprocals of M nonzero values with one division: prefix products, the reciprocal
// of the last one, then backwards (Montgomery's batch inversion); each result is within
// a few ulps of 1/x_i.  The fp64 pipe, not memory, bounds the node update, and a
// division costs several times a product there.
template <int M>
BC_HD void batch_reciprocal(const double (&x)[M], double (&inv)[M]) {
    double pre[M];
    pre[0] = x[0];
#pragma unroll
    for (int i = 1; i < M; ++i) pre[i] = pre[i - 1] * x[i];
    double r = 1.0 / pre[M - 1];
#pragma unroll
    for (int i = M - 1; i > 0; --i) {
        inv[i] = r * pre[i - 1];
        r *= x[i];
    }
    inv[0] = r;
}

// ln(1 + a): the Taylor series, three terms for |a| < 2^-18 (relative error < a^3 / 4 <
// 2e-17) and six for |a| < 2^-10 (< a^6 / 7 < 2e-19), else the library function.
BC_HD double log1p_small(double a) {
    if (abs_below(a, 0x1p-18)) return a - a * a * (0.5 - a * (1.0 / 3.0));
    if (abs_below(a, 0x1p-10)) {
        const double a2 = a * a;
        return a - a2 * (0.5 - a * (1.0 / 3.0 - a * (0.25 - a * (0.2 - a * (1.0 / 6.0)))));
    }
    return log1p(a);
}

// x / (1 - ex) for ex = exp(-x/s) given; the removable point x = 0 takes its limit.
BC_HD double lin_exp_given(double x, double s, double ex) {
    if (abs_below(x, 1e-6 * s)) return s + 0.5 * x;
    return x / (1.0 - ex);
}

constexpr double kInv80 = 1.0 / 80.0, kInv3 = 1.0 / 3.0, kInv5 = 1.0 / 5.0;
constexpr double kInvTau = 1.0 / tau;

// Nernst potentials and the reciprocals of the concentrations they came from (for the
// update of the potentials after an Euler step, see current_after_step).
struct Nernst { double ENa, EK, iNao, iNai, iKo, iKi; };

// Functions of a node's state that the update needs, carried from one step to the next:
// E_Na, E_K, X = exp(-K_o/5), exp((25 - Na_i)/3), the potential u at the node and
// B = exp(-u/720).  Each step changes the concentrations by small increments, so their
// functions follow from the old ones by logarithms and exponentials of numbers near 1 and
// 0 (short series); u^k's B follows from u^{k-1}'s the same way.
struct NodeCache { double ENa, EK, X, ep, up, B; };

BC_HD NodeCache node_cache(double Ko, double Nai, double u) {
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    return NodeCache{RTF * log(Nao / Nai), RTF * log(Ko / Ki), exp(-Ko * kInv5), exp((25.0 - Nai) * kInv3),
                     u, exp(-u * (1.0 / 720.0))};
}

// y'(V, y) of the Sec. 2 model (= -m(u, y)) at one point: d[0..4] for n, h, K_o, Na_i,
// Ca_i; also the Nernst potentials of the state in *ne (may be null).  CACHED: E_Na, E_K,
// the two concentration exponentials and B = exp(-V/720) are read from *c instead of
// evaluated.
template <bool CACHED = false>
BC_HD void rates(const NodeConsts& k, double V, double n, double h, double Ko, double Nai, double Cai,
                 double* d, Nernst* ne = nullptr, const NodeCache* c = nullptr) {
    const VPowers p = CACHED ? vpowers_from(c->B) : vpowers(V);
    const double xn = V + 34.0, xm = V + 30.0;
    const bool sn = abs_below(xn, 1e-5), sm = abs_below(xm, 1e-5);   // |x| < 1e-6 s, s = 10
    const double exn = k.an * p.e10, exm = k.am * p.e10;
    const double bm = k.bm * p.e18;
    // m_inf = am / (am + bm), am = 0.1 xm / (1 - exm): 0.1 xm / (0.1 xm + bm (1 - exm))
    const double am_num = sm ? 0.1 * (10.0 + 0.5 * xm) : 0.1 * xm;
    const double am_den = sm ? 1.0 : 1.0 - exm;
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    const double X = CACHED ? c->X : exp(-Ko * kInv5), X2 = X * X, X5 = X2 * X2 * X;
    const double ep = CACHED ? c->ep : exp((25.0 - Nai) * kInv3);
    double den[11] = {sn ? 1.0 : 1.0 - exn,                  // alpha_n
                      1.0 + k.bh * p.e10,                    // beta_h
                      am_num + bm * am_den,                  // m_inf
                      1.0 + Cai,                             // g_AHP term
                      (1.0 + ep) * (1.0 + k.pump * X5),      // pump
                      1.0 + k.glia * X2,                     // glia
                      1.0 + k.ca * p.e25,                    // calcium
                      Nai, Ki, Nao, Ko};
    double inv[11];
    batch_reciprocal(den, inv);
    const double an = sn ? 0.01 * (10.0 + 0.5 * xn) : 0.01 * xn * inv[0];
    const double bn = k.bn * p.e80;
    const double ah = k.ah * p.e20;
    const double bh = inv[1];
    const double minf = am_num * inv[2];
    const double ENa = CACHED ? c->ENa : RTF * log(Nao * inv[7]);
    const double EK = CACHED ? c->EK : RTF * log(Ko * inv[8]);
    const double INa = (gNa * minf * minf * minf * h + gNaL) * (V - ENa);
    const double IK = (gK * (n * n) * (n * n) + gAHP * Cai * inv[3] + gKL) * (V - EK);
    const double pump = rho * inv[4];
    const double glia = Gglia * inv[5];
    const double diff = eps * (Ko - kbath);
    d[0] = phi * (an * (1.0 - n) - bn * n);
    d[1] = phi * (ah * (1.0 - h) - bh * h);
    d[2] = (gamma * beta * IK - 2.0 * beta * pump - glia - diff) * kInvTau;
    d[3] = (-gamma * INa - 3.0 * pump) * kInvTau;
    d[4] = -0.002 * gCa * (V - ECa) * inv[6] - Cai * kInv80;
    if (ne) {
        ne->ENa = ENa; ne->EK = EK;
        ne->iNai = inv[7]; ne->iKi = inv[8]; ne->iNao = inv[9]; ne->iKo = inv[10];
    }
}

// Sodium gate m_inf(V) = num / den (the division is left to the caller's batch); B is
// exp(-V/720).
BC_HD void minf_parts_b(const NodeConsts& k, double V, double B, double& num, double& den) {
    double e10, e18;
    vpowers_m_from(B, e10, e18);
    const double xm = V + 30.0;
    const bool sm = abs_below(xm, 1e-5);
    const double exm = k.am * e10, bm = k.bm * e18;
    num = sm ? 0.1 * (10.0 + 0.5 * xm) : 0.1 * xm;
    den = num + bm * (sm ? 1.0 : 1.0 - exm);
}

BC_HD void minf_parts(const NodeConsts& k, double V, double& num, double& den) {
    minf_parts_b(k, V, exp(-V * (1.0 / 720.0)), num, den);
}

// I_Na + I_K + I_Cl at potential V for state (n, h, K_o, Na_i, Ca_i).
BC_HD double total_current(const NodeConsts& k, double V, double n, double h, double Ko, double Nai,
                           double Cai) {
    double num, den;
    minf_parts(k, V, num, den);
    const double Ki = 140.0 + (18.0 - Nai);
    const double Nao = 144.0 - beta * (Nai - 18.0);
    double dd[4] = {den, 1.0 + Cai, Nai, Ki}, inv[4];
    batch_reciprocal(dd, inv);
    const double minf = num * inv[0];
    const double INa = (gNa * minf * minf * minf * h + gNaL) * (V - RTF * log(Nao * inv[2]));
    const double IK = (gK * (n * n) * (n * n) + gAHP * Cai * inv[1] + gKL) * (V - RTF * log(Ko * inv[3]));
    return INa + IK + gClL * (V - k.ECl);
}

// The current at (V, y + dy) for a state y whose Nernst potentials ne rates() gave:
// with dNa = dy[3] (Na_o falls by beta dNa, K_i by dNa) and dK = dy[2],
//   E_Na' = E_Na + RTF (ln(1 - beta dNa / Na_o) - ln(1 + dNa / Na_i)),
//   E_K'  = E_K  + RTF (ln(1 + dK / K_o) - ln(1 - dNa / K_i)),
// logarithms of numbers within ~1e-3 of 1 (a short series) instead of two full ones.
// B = exp(-V/720); the new potentials go to *ENa1, *EK1 when given.
BC_HD double current_after_step_b(const NodeConsts& k, double V, double B, double n, double h, double Ko,
                                  double Nai, double Cai, const Nernst& ne, double dK, double dNa,
                                  double* ENa1 = nullptr, double* EK1 = nullptr) {
    double num, den;
    minf_parts_b(k, V, B, num, den);
    double dd[2] = {den, 1.0 + Cai}, inv[2];
    batch_reciprocal(dd, inv);
    const double minf = num * inv[0];
    const double ENa = ne.ENa + RTF * (log1p_small(-beta * dNa * ne.iNao) - log1p_small(dNa * ne.iNai));
    const double EK = ne.EK + RTF * (log1p_small(dK * ne.iKo) - log1p_small(-dNa * ne.iKi));
    if (ENa1) *ENa1 = ENa;
    if (EK1) *EK1 = EK;
    const double INa = (gNa * minf * minf * minf * h + gNaL) * (V - ENa);
    const double IK = (gK * (n * n) * (n * n) + gAHP * Cai * inv[1] + gKL) * (V - EK);
    return INa + IK + gClL * (V - k.ECl);
}

BC_HD double current_after_step(const NodeConsts& k, double V, double n, double h, double Ko,
                                double Nai, double Cai, const Nernst& ne, double dK, double dNa) {
    return current_after_step_b(k, V, exp(-V * (1.0 / 720.0)), n, h, Ko, Nai, Cai, ne, dK, dNa);
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

// The Euler step at potential V followed by the current at potential Vx and the new
// state (the per-node work of one time step), the new state's Nernst potentials taken
// from the old ones.  Returns f(Vx, y^{k+1}).
BC_HD double euler_and_current(const NodeConsts& k, double V, double Vx, double dt, double& n,
                               double& h, double& Ko, double& Nai, double& Cai) {
    double d[5];
    Nernst ne;
    rates(k, V, n, h, Ko, Nai, Cai, d, &ne);
    const double dK = dt * d[2], dNa = dt * d[3];
    n += dt * d[0];
    h += dt * d[1];
    Ko += dK;
    Nai += dNa;
    Cai += dt * d[4];
    return current_after_step(k, Vx, n, h, Ko, Nai, Cai, ne, dK, dNa);
}

// The same step with the node's carried functions c: on entry the old state's (with c.B
// already exp(-V/720) for this step's V), on return the new state's -- E_Na and E_K as
// above, X and the sodium exponential times exp(-dK/5) and exp(-dNa/3), c.up = V -- and
// the current at Vx with exp(-Vx/720) = exp(-V/720) exp((V - Vx)/720).
BC_HD double euler_and_current_c(const NodeConsts& k, double V, double Vx, double dt, double& n,
                                 double& h, double& Ko, double& Nai, double& Cai, NodeCache& c) {
    double d[5];
    Nernst ne;
    rates<true>(k, V, n, h, Ko, Nai, Cai, d, &ne, &c);
    const double B = c.B;
    const double dK = dt * d[2], dNa = dt * d[3];
    n += dt * d[0];
    h += dt * d[1];
    Ko += dK;
    Nai += dNa;
    Cai += dt * d[4];
    const double Bx = B * exp_small((V - Vx) * (1.0 / 720.0));
    const double f = current_after_step_b(k, Vx, Bx, n, h, Ko, Nai, Cai, ne, dK, dNa, &c.ENa, &c.EK);
    c.X *= exp_small(-dK * kInv5);
    c.ep *= exp_small(-dNa * kInv3);
    c.up = V;
    return f;
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
