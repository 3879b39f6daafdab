// Input features of the learned initial guess's per-element network (shared by its
// inference and training kernels).
#pragma once

#include <cstdint>

#include "kernels.h"

namespace polydg {

__host__ __device__ constexpr int guess_inputs(int np) { return 9 * np + 3; }

// Features of element e into x[0 .. 9 NP + 3) (fp32), by one warp: lane l handles
// component l of the own vector [a | d1 | d2] and its mean and max over the face
// neighbours (the blocks of row e of K_h after the diagonal one).  off(c) is the
// position of cell c's first coefficient in the U arrays.  The scales enter as
// reciprocals: a division costs GB300's narrow fp64 pipe about ten times a product, and
// the features are rounded to fp16 afterwards.
template <int NP, typename Off>
__device__ __forceinline__ void element_features(const GuessFeat& f, const double* __restrict__ Uk,
                                                 const double* __restrict__ Uk1,
                                                 const double* __restrict__ Uk2, int64_t e, float* x,
                                                 Off&& off) {
    const int lane = threadIdx.x & 31;
    auto own = [&](int64_t cell, int l) {
        const int grp = l / NP, j = l - grp * NP;
        const int64_t o = off(cell) + j;
        if (grp == 0) return (Uk[o] - (j == 0 ? f.u_rest : 0.0)) * f.inv_s_u;
        if (grp == 1) return (Uk[o] - Uk1[o]) * f.inv_s_d;
        return (Uk1[o] - Uk2[o]) * f.inv_s_d;
    };
    const int32_t b0 = f.row_ptr[e], b1 = f.row_ptr[e + 1];
    const int cnt = b1 - b0 - 1;
    for (int l = lane; l < 3 * NP; l += 32) {
        x[l] = (float)own(e, l);
        double sum = 0.0, mx = 0.0;
        for (int32_t b = b0 + 1; b < b1; ++b) {
            const double v = own(f.col[b], l);
            sum += v;
            mx = (b == b0 + 1) ? v : fmax(mx, v);
        }
        x[3 * NP + l] = cnt > 0 ? (float)(sum / cnt) : 0.f;
        x[6 * NP + l] = cnt > 0 ? (float)mx : 0.f;
    }
    if (lane == 0) {
        x[9 * NP] = (float)(f.diam[e] / f.h_ref);
        x[9 * NP + 1] = (float)(f.dt / f.dt_ref);
        x[9 * NP + 2] = (float)cnt / 10.f;
    }
}

__device__ __forceinline__ void zero_row(float* x, int F) {
    for (int l = threadIdx.x & 31; l < F; l += 32) x[l] = 0.f;
}

}  // namespace polydg
