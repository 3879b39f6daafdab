// Per-quadrature-node ionic update and ion-current load of one Crank-Nicolson
// step (Eq. fully-discrete-1), plus the per-step bookkeeping kernels.
#include <cuda_runtime.h>

#include "device.cuh"
#include "ionic_model.cuh"
#include "kernels.h"

namespace polydg {

// Warp per cell: nodes of cell e are node_ptr[e]..node_ptr[e+1]-1.  Per node:
//   u^k(x_q), y^{k+1} = y^k + dt y'(u^k, y^k),  u~ = 3/2 U^k - 1/2 U^{k-1} (U^0 at k = 0),
//   I_e[i] = sum_q w_q f(u~(x_q), y^{k+1}_q) phi_i(x_q).
// The cell's coefficient vectors sit in shared memory (broadcast reads), so a thread
// keeps only its node's basis values and the NP partial sums in registers: two
// 256-thread blocks fit on an SM, which the fp64-latency-bound node update needs.
constexpr int kIonicThreads = 256;

template <int NP>
__global__ void __launch_bounds__(kIonicThreads, 2)
ionic_kernel(const double* __restrict__ U, const double* __restrict__ Uprev,
             const int64_t* __restrict__ node_ptr, const double* __restrict__ node_w,
             const double* __restrict__ node_phi, double* __restrict__ y, int64_t nn, int64_t nc,
             double dt, double* __restrict__ I, const SimScalars* ss, const bc::NodeConsts kc) {
    __shared__ double su[kIonicThreads / 32][2][NP];
    if (ss->failed) return;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (e >= nc) return;
    const bool first = (ss->k == 0);
    if (lane < NP) {
        const double ue = U[e * NP + lane];
        su[wl][0][lane] = ue;
        su[wl][1][lane] = first ? ue : 1.5 * ue - 0.5 * Uprev[e * NP + lane];
    }
    __syncwarp();
    double acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = 0.0;
    const int64_t q1 = node_ptr[e + 1];
    for (int64_t q = node_ptr[e] + lane; q < q1; q += 32) {
        const double* ph = node_phi + q * NP;
        double phv[NP];
        double uk = 0.0, ux = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            phv[j] = __ldg(ph + j);
            uk = fma(phv[j], su[wl][0][j], uk);
            ux = fma(phv[j], su[wl][1][j], ux);
        }
        double n = y[q], h = y[nn + q], Ko = y[2 * nn + q], Nai = y[3 * nn + q], Cai = y[4 * nn + q];
        bc::euler(kc, uk, dt, n, h, Ko, Nai, Cai);    // explicit Euler with u^k
        y[q] = n; y[nn + q] = h; y[2 * nn + q] = Ko; y[3 * nn + q] = Nai; y[4 * nn + q] = Cai;
        const double wf = node_w[q] * bc::total_current(kc, ux, n, h, Ko, Nai, Cai);
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = fma(wf, phv[j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const double s = warp_sum(acc[j]);
        if (lane == 0) I[e * NP + j] = s;
    }
}

cudaError_t launch_ionic(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                         const double* node_w, const double* node_phi, double* y, int64_t nn,
                         int64_t nc, double dt, double* I, const SimScalars* ss, cudaStream_t s) {
    const unsigned g = (unsigned)((nc * 32 + kIonicThreads - 1) / kIonicThreads);
    static const bc::NodeConsts kc = bc::node_consts();
    switch (np) {
        case 3: ionic_kernel<3><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, y, nn, nc, dt, I, ss, kc); break;
        case 6: ionic_kernel<6><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, y, nn, nc, dt, I, ss, kc); break;
        case 10: ionic_kernel<10><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, y, nn, nc, dt, I, ss, kc); break;
        case 15: ionic_kernel<15><<<g, kIonicThreads, 0, s>>>(U, Uprev, node_ptr, node_w, node_phi, y, nn, nc, dt, I, ss, kc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// y_caller[pos[q]][s] = y_int[q][s] for the 5 state rows.
__global__ void node_gather_kernel(const double* __restrict__ yi, double* __restrict__ yc,
                                   const int64_t* __restrict__ pos, int64_t nn) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nn) return;
    const int64_t d = pos[q];
#pragma unroll
    for (int s = 0; s < 5; ++s) yc[s * nn + d] = yi[s * nn + q];
}

cudaError_t launch_node_gather(const double* y_int, double* y_caller,
                               const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s) {
    node_gather_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(y_int, y_caller,
                                                                   node_to_caller_pos, nn);
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
