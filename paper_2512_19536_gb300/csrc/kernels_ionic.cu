// Per-quadrature-node ionic update and ion-current load of one Crank-Nicolson
// step (Eq. fully-discrete-1), plus the per-step bookkeeping kernels.
#include <algorithm>

#include <cuda_runtime.h>

#include "device.cuh"
#include "ionic_model.cuh"
#include "kernels.h"

namespace polydg {

// LPC lanes per cell (32 / LPC consecutive cells per warp; nodes of cell e are
// node_ptr[e]..node_ptr[e+1]-1, lane l of its group takes nodes l, l + LPC, ...).  The
// host picks LPC from the cells' node counts (ionic_lanes_per_cell): a warp instruction
// costs the fp64 pipe the same with idle lanes, so the pick is the one with the fewest
// passes, e.g. 8 for 168-node cells (21 full passes per 4 cells, where a warp per cell
// would run 6 passes with 8 of 32 lanes busy in the last).  Per node:
//   u^k(x_q), y^{k+1} = y^k + dt y'(u^k, y^k),  u~ = 3/2 U^k - 1/2 U^{k-1} (U^0 at k = 0),
//   I_e[i] = sum_q w_q f(u~(x_q), y^{k+1}_q) phi_i(x_q).
// yc carries E_Na, E_K, exp(-K_o/5), exp((25 - Na_i)/3), u^{k-1}(x_q) and exp(-u^{k-1}/720)
// of each node from one step to the next (bc::NodeCache): the update reads them instead of
// two logarithms, three exponentials and the projection of U^{k-1}
// (u~ = 3/2 u^k - 1/2 u^{k-1} at the node), and leaves the new state's.  ionic_cache_kernel
// evaluates them afresh before the update when the state or the potentials were set from
// outside (ss->yc_ok = 0) and every 256 steps.
// The cell's coefficient vectors sit in shared memory (broadcast reads), so a thread
// keeps only its node's basis values and the NP partial sums in registers: two
// 256-thread blocks fit on an SM, which the fp64-latency-bound node update needs.
constexpr int kIonicThreads = 256;

template <int NP, int LPC>
__global__ void __launch_bounds__(kIonicThreads, 2)
ionic_kernel(const double* __restrict__ U, const double* __restrict__ Uprev,
             const int64_t* __restrict__ node_ptr, const double* __restrict__ node_w,
             const double* __restrict__ node_phi, double* __restrict__ y, double* __restrict__ yc,
             int64_t nn, int64_t nc, double dt, double* __restrict__ I, const SimScalars* ss,
             const bc::NodeConsts kc) {
    constexpr int CPW = 32 / LPC;                 // cells per warp
    __shared__ double su[kIonicThreads / 32][CPW][NP];
    if (ss->failed) return;
    const int64_t e0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * CPW;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (e0 >= nc) return;                         // the whole warp: the sums below need all lanes
    const int cw = lane / LPC, sl = lane % LPC;
    const int64_t e = e0 + cw;
    const bool first = (ss->k == 0);
    for (int t = lane; t < CPW * NP; t += 32)
        su[wl][t / NP][t % NP] = e0 + t / NP < nc ? U[e0 * NP + t] : 0.0;
    __syncwarp();
    double acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = 0.0;
    const int64_t q1 = e < nc ? node_ptr[e + 1] : 0;
    for (int64_t q = e < nc ? node_ptr[e] + sl : 0; q < q1; q += LPC) {
        const double* ph = node_phi + q * NP;
        double uk = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) uk = fma(__ldg(ph + j), su[wl][cw][j], uk);
        double n = y[q], h = y[nn + q], Ko = y[2 * nn + q], Nai = y[3 * nn + q], Cai = y[4 * nn + q];
        bc::NodeCache c{yc[q], yc[nn + q], yc[2 * nn + q], yc[3 * nn + q], yc[4 * nn + q], yc[5 * nn + q]};
        // u~ = 3/2 u^k - 1/2 u^{k-1} (u^0 at k = 0); exp(-u^k/720) from exp(-u^{k-1}/720)
        const double ux = first ? uk : 1.5 * uk - 0.5 * c.up;
        c.B *= bc::exp_small((c.up - uk) * (1.0 / 720.0));
        // explicit Euler with u^k, then f(u~, y^{k+1})
        const double f = bc::euler_and_current_c(kc, uk, ux, dt, n, h, Ko, Nai, Cai, c);
        y[q] = n; y[nn + q] = h; y[2 * nn + q] = Ko; y[3 * nn + q] = Nai; y[4 * nn + q] = Cai;
        yc[q] = c.ENa; yc[nn + q] = c.EK; yc[2 * nn + q] = c.X; yc[3 * nn + q] = c.ep;
        yc[4 * nn + q] = c.up; yc[5 * nn + q] = c.B;
        const double wf = node_w[q] * f;
        // the basis values again (L1 hits): keeping them in registers across the node
        // update would spill
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = fma(wf, __ldg(ph + j), acc[j]);
    }
    // sums over each cell's LPC lanes (xor offsets below LPC stay inside the group)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double s = acc[j];
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sl == 0 && e < nc) I[e * NP + j] = s;
    }
}

int ionic_lanes_per_cell(const int64_t* node_ptr, int64_t nc) {
    int best = 32;
    long double best_cost = 0.0L;
    for (int lpc : {32, 16, 8}) {
        const int cpw = 32 / lpc;
        long double passes = 0.0L;
        for (int64_t g = 0; g < nc; g += cpw) {
            int64_t m = 0;
            for (int64_t e = g; e < std::min<int64_t>(nc, g + cpw); ++e)
                m = std::max<int64_t>(m, (node_ptr[e + 1] - node_ptr[e] + lpc - 1) / lpc);
            passes += (long double)m;
        }
        if (lpc == 32 || passes <= best_cost) { best = lpc; best_cost = passes; }
    }
    return best;
}

// The carried functions of every node, evaluated from the state and from U^{k-1} (U^0 at
// k = 0), warp per cell: all of them every 256th step and when the state was set from
// outside (bit 0 of ss->yc_ok clear), those of u^{k-1} alone when only the potentials were
// (bit 1 clear); nothing otherwise.
template <int NP>
__global__ void __launch_bounds__(kIonicThreads)
ionic_cache_kernel(const double* __restrict__ U, const double* __restrict__ Uprev,
                   const int64_t* __restrict__ node_ptr, const double* __restrict__ node_phi,
                   const double* __restrict__ y, double* __restrict__ yc, int64_t nn, int64_t nc,
                   const SimScalars* ss) {
    __shared__ double su[kIonicThreads / 32][NP];
    if (ss->failed) return;
    const bool all = (ss->k & 255) == 0 || !(ss->yc_ok & 1);
    if (!all && (ss->yc_ok & 2)) return;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (e >= nc) return;
    if (lane < NP) su[wl][lane] = (ss->k == 0 ? U : Uprev)[e * NP + lane];
    __syncwarp();
    for (int64_t q = node_ptr[e] + lane; q < node_ptr[e + 1]; q += 32) {
        double up = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) up = fma(node_phi[q * NP + j], su[wl][j], up);
        if (all) {
            const bc::NodeCache c = bc::node_cache(y[2 * nn + q], y[3 * nn + q], up);
            yc[q] = c.ENa;
            yc[nn + q] = c.EK;
            yc[2 * nn + q] = c.X;
            yc[3 * nn + q] = c.ep;
        }
        yc[4 * nn + q] = up;
        yc[5 * nn + q] = exp(-up * (1.0 / 720.0));
    }
}

cudaError_t launch_ionic(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                         const double* node_w, const double* node_phi, double* y, double* yc, int64_t nn,
                         int64_t nc, double dt, double* I, const SimScalars* ss, int lpc, cudaStream_t s) {
    const unsigned g = (unsigned)((nc * 32 + kIonicThreads - 1) / kIonicThreads);
    static const bc::NodeConsts kc = bc::node_consts();
    if (lpc != 32 && lpc != 16 && lpc != 8) return cudaErrorInvalidValue;
    const int64_t warps = (nc + 32 / lpc - 1) / (32 / lpc);
    const unsigned gi = (unsigned)((warps * 32 + kIonicThreads - 1) / kIonicThreads);
    switch (np) {
        case 3: ionic_cache_kernel<3><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_phi, y, yc, nn, nc, ss); break;
        case 6: ionic_cache_kernel<6><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_phi, y, yc, nn, nc, ss); break;
        case 10: ionic_cache_kernel<10><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_phi, y, yc, nn, nc, ss); break;
        case 15: ionic_cache_kernel<15><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_phi, y, yc, nn, nc, ss); break;
        default: return cudaErrorInvalidValue;
    }
    auto run = [&](auto kern) {
        kern<<<gi, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, y, yc, nn, nc, dt, I, ss, kc);
    };
#define POLYDG_IONIC_CASE(NP_)                                                  \
    case NP_:                                                                   \
        if (lpc == 32) run(ionic_kernel<NP_, 32>);                              \
        else if (lpc == 16) run(ionic_kernel<NP_, 16>);                         \
        else run(ionic_kernel<NP_, 8>);                                         \
        break;
    switch (np) {
        POLYDG_IONIC_CASE(3)
        POLYDG_IONIC_CASE(6)
        POLYDG_IONIC_CASE(10)
        POLYDG_IONIC_CASE(15)
        default: return cudaErrorInvalidValue;
    }
#undef POLYDG_IONIC_CASE
    return cudaGetLastError();
}

// The ionic state in the DG basis (Eq. fully-discrete-1, second line: M_h Y^{k+1} =
// M_h Y^k - dt G^k, M_h block diagonal).  Warp per cell, Y_l the cell's n_p coefficients
// of state l (Ym[l][c n_p + j]):
//   pass 1, per node:  d_l(x_q) = dt y'_l(u^k(x_q), y_h^k(x_q))  (into the node buffer y),
//   pass 2, per state: G_l = sum_q w_q d_l(x_q) phi(x_q),  Y_l += M_K^{-1} G_l,
//   pass 3, per node:  y_h^{k+1}(x_q) into y, and I_e = sum_q w_q f(u~(x_q), y_h^{k+1}(x_q)) phi(x_q).
// The node buffer then holds the modal state's values at the nodes.
template <int NP>
__global__ void __launch_bounds__(kIonicThreads, 2)
ionic_modal_kernel(const double* __restrict__ U, const double* __restrict__ Uprev,
                   const int64_t* __restrict__ node_ptr, const double* __restrict__ node_w,
                   const double* __restrict__ node_phi, const double* __restrict__ Minv,
                   double* __restrict__ Ym, double* __restrict__ y, int64_t nn, int64_t nc, double dt,
                   double* __restrict__ I, const SimScalars* ss, const bc::NodeConsts kc) {
    constexpr int W = kIonicThreads / 32;
    __shared__ double su[W][2][NP];
    __shared__ double sy[W][5][NP];
    __shared__ double sg[W][5][NP];
    if (ss->failed) return;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (e >= nc) return;
    const bool first = (ss->k == 0);
    const int64_t n = nc * NP;
    if (lane < NP) {
        const double ue = U[e * NP + lane];
        su[wl][0][lane] = ue;
        su[wl][1][lane] = first ? ue : 1.5 * ue - 0.5 * Uprev[e * NP + lane];
#pragma unroll
        for (int l = 0; l < 5; ++l) sy[wl][l][lane] = Ym[l * n + e * NP + lane];
    }
    __syncwarp();
    const int64_t q0 = node_ptr[e], q1 = node_ptr[e + 1];
    for (int64_t q = q0 + lane; q < q1; q += 32) {          // pass 1
        const double* ph = node_phi + q * NP;
        double uk = 0.0, yv[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const double pv = __ldg(ph + j);
            uk = fma(pv, su[wl][0][j], uk);
#pragma unroll
            for (int l = 0; l < 5; ++l) yv[l] = fma(pv, sy[wl][l][j], yv[l]);
        }
        double d[5];
        bc::rates(kc, uk, yv[0], yv[1], yv[2], yv[3], yv[4], d);
#pragma unroll
        for (int l = 0; l < 5; ++l) y[l * nn + q] = dt * d[l];
    }
    __syncwarp();
    for (int l = 0; l < 5; ++l) {                           // pass 2
        double acc[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = 0.0;
        for (int64_t q = q0 + lane; q < q1; q += 32) {
            const double* ph = node_phi + q * NP;
            const double wd = node_w[q] * y[l * nn + q];
#pragma unroll
            for (int j = 0; j < NP; ++j) acc[j] = fma(wd, __ldg(ph + j), acc[j]);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const double sum = warp_sum(acc[j]);
            if (lane == j) sg[wl][l][j] = sum;
        }
    }
    __syncwarp();
    if (lane < NP) {
        const double* Mr = Minv + (e * NP + lane) * NP;     // row `lane` of M_K^{-1}
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            double v = sy[wl][l][lane];
#pragma unroll
            for (int c = 0; c < NP; ++c) v = fma(__ldg(Mr + c), sg[wl][l][c], v);
            Ym[l * n + e * NP + lane] = v;
            sy[wl][l][lane] = v;                            // read back after the warp sync
        }
    }
    __syncwarp();
    double acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = 0.0;
    for (int64_t q = q0 + lane; q < q1; q += 32) {          // pass 3
        const double* ph = node_phi + q * NP;
        double phv[NP];
        double ux = 0.0, yv[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            phv[j] = __ldg(ph + j);
            ux = fma(phv[j], su[wl][1][j], ux);
#pragma unroll
            for (int l = 0; l < 5; ++l) yv[l] = fma(phv[j], sy[wl][l][j], yv[l]);
        }
#pragma unroll
        for (int l = 0; l < 5; ++l) y[l * nn + q] = yv[l];
        const double wf = node_w[q] * bc::total_current(kc, ux, yv[0], yv[1], yv[2], yv[3], yv[4]);
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = fma(wf, phv[j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const double sum = warp_sum(acc[j]);
        if (lane == 0) I[e * NP + j] = sum;
    }
}

cudaError_t launch_ionic_modal(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                               const double* node_w, const double* node_phi, const double* Minv,
                               double* Ym, double* y, int64_t nn, int64_t nc, double dt, double* I,
                               const SimScalars* ss, cudaStream_t s) {
    const unsigned g = (unsigned)((nc * 32 + kIonicThreads - 1) / kIonicThreads);
    static const bc::NodeConsts kc = bc::node_consts();
    switch (np) {
        case 3: ionic_modal_kernel<3><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, Minv, Ym, y, nn, nc, dt, I, ss, kc); break;
        case 6: ionic_modal_kernel<6><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, Minv, Ym, y, nn, nc, dt, I, ss, kc); break;
        case 10: ionic_modal_kernel<10><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, Minv, Ym, y, nn, nc, dt, I, ss, kc); break;
        case 15: ionic_modal_kernel<15><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, Minv, Ym, y, nn, nc, dt, I, ss, kc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Modal initial state: Y_l = y0_l times the constant mode (phi_0 = 1), other modes 0.
__global__ void init_modal_kernel(double* Ym, int64_t nc, int np, const double* y0) {
    const int64_t n = nc * np;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 5 * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = t / n, r = t - l * n;
        Ym[t] = (r % np == 0) ? y0[l] : 0.0;
    }
}

cudaError_t launch_init_modal(double* Ym, int64_t nc, int np, const double* y0, cudaStream_t s) {
    const int64_t total = 5 * nc * np;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    init_modal_kernel<<<g, 256, 0, s>>>(Ym, nc, np, y0);
    return cudaGetLastError();
}

// y_caller[pos[q]][s] = y_int[q][s] for the 5 state rows.
__global__ void node_gather_kernel(const double* __restrict__ yi, double* __restrict__ yc,
                                   const int64_t* __restrict__ pos, int64_t nn, int ns) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nn) return;
    const int64_t d = pos[q];
    for (int s = 0; s < ns; ++s) yc[s * nn + d] = yi[s * nn + q];
}

cudaError_t launch_node_gather(const double* y_int, double* y_caller,
                               const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s, int ns) {
    node_gather_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(y_int, y_caller,
                                                                   node_to_caller_pos, nn, ns);
    return cudaGetLastError();
}

// The reverse of node_gather_kernel: caller node order -> internal node order.
__global__ void node_scatter_kernel(const double* __restrict__ yc, double* __restrict__ yi,
                                    const int64_t* __restrict__ pos, int64_t nn, int ns) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nn) return;
    const int64_t d = pos[q];
    for (int s = 0; s < ns; ++s) yi[s * nn + q] = yc[s * nn + d];
}

cudaError_t launch_node_scatter(const double* y_caller, double* y_int,
                                const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s, int ns) {
    node_scatter_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(y_caller, y_int,
                                                                    node_to_caller_pos, nn, ns);
    return cudaGetLastError();
}

__global__ void ionic_aux_flag_kernel(SimScalars* ss, int ok) { ss->yc_ok = ok < 0 ? (ss->yc_ok & 1) : ok; }

cudaError_t launch_ionic_aux_valid(SimScalars* ss, cudaStream_t s, int ok) {
    ionic_aux_flag_kernel<<<1, 1, 0, s>>>(ss, ok);
    return cudaGetLastError();
}

__global__ void set_step_kernel(SimScalars* ss, int64_t k) {
    ss->k = k;
    ss->failed = 0;
    ss->yc_ok = 0;             // the state was set from outside
}

cudaError_t launch_set_step(SimScalars* ss, int64_t k, cudaStream_t s) {
    set_step_kernel<<<1, 1, 0, s>>>(ss, k);
    return cudaGetLastError();
}

__global__ void init_y_kernel(double* y, int64_t nn, const double* y0) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nn) return;
#pragma unroll
    for (int s = 0; s < 5; ++s) y[s * nn + q] = y0[s];
}

cudaError_t launch_init_y(double* y, int64_t nn, const double* y0, cudaStream_t s) {
    init_y_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(y, nn, y0);
    return cudaGetLastError();
}

// Reset the PCG scalars at the start of a step (no-op after a failed step).
__global__ void step_begin_kernel(PcgScalars* sc, SimScalars* ss) {
    if (threadIdx.x != 0) return;
    sc->done = ss->failed ? 1 : 0;
    sc->it = 0;
    sc->status = 0;
    ss->use_guess = 0;
}

cudaError_t launch_step_begin(PcgScalars* sc, SimScalars* ss, cudaStream_t s) {
    step_begin_kernel<<<1, 32, 0, s>>>(sc, ss);
    return cudaGetLastError();
}

// U^{k-2} <- U^{k-1} (if kept), U^{k-1} <- U^k, U^k <- x (also into the solution ring,
// slot k+1), k <- k + 1 and the step statistics.
__global__ void step_finish_kernel(double* __restrict__ U, double* __restrict__ Uprev,
                                   double* __restrict__ Uprev2, const double* __restrict__ x0,
                                   const double* __restrict__ x1, int64_t n, const PcgScalars* sc,
                                   SimScalars* ss, double* __restrict__ ring) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = !ss->failed;
    const double* x = (sc->pass & 1) ? x1 : x0;   // the iterate lives in buffer (pass & 1)
    if (ok && t < n) {
        if (Uprev2) Uprev2[t] = Uprev[t];
        Uprev[t] = U[t];
        U[t] = x[t];
        if (ring) ring[((ss->k + 1) % kHistRing) * n + t] = x[t];
    }
}

__global__ void step_stats_kernel(const PcgScalars* sc, SimScalars* ss) {
    if (threadIdx.x != 0 || ss->failed) return;
    if (ss->hist_len < kHistRing) ss->hist_len += 1;
    ss->yc_ok = 3;             // the step's ionic update left the new state's carried functions
    ss->k += 1;
    ss->steps_done += 1;
    ss->total_its += sc->it;
    if (sc->it > ss->max_its) ss->max_its = sc->it;
    ss->last_relres = sc->relres;
    if (sc->status != 0) {
        ss->status = sc->status;
        ss->failed = 1;
    }
}

cudaError_t launch_step_finish(double* U, double* Uprev, double* Uprev2, const double* x0,
                               const double* x1, int64_t n, const PcgScalars* sc, SimScalars* ss,
                               double* ring,
                               cudaStream_t s) {
    step_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U, Uprev, Uprev2, x0, x1, n, sc, ss, ring);
    step_stats_kernel<<<1, 32, 0, s>>>(sc, ss);
    return cudaGetLastError();
}

}  // namespace polydg
