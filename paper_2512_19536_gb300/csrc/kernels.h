// Launch wrappers of libpolydg's CUDA kernels (host-callable, no torch types).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"

namespace polydg {

enum MatvecMode { MODE_PLAIN = 0, MODE_PCG = 1, MODE_RESID = 2, MODE_RHS = 3 };

// Per-simulation scalars resident in device memory.
struct SimScalars {
    int64_t k;             // current step index (U holds U^k)
    int32_t failed;        // set once a step's solve failed: later steps do nothing
    int32_t max_its;
    int64_t steps_done;
    int64_t total_its;
    int32_t status;
    int32_t pad;
    double last_relres;
};

// Block-sparse K_h on the device (internal cell order).
struct DeviceMatrix {
    int64_t nc = 0, nblk = 0;
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;        // K_h
    double* val_minus = nullptr;  // chi_cm M - dt/2 A
};

cudaError_t launch_matvec(int mode, int np, const DeviceMatrix& K, const double* val,
                          const double* x, double* y, const double* v1, const double* v2,
                          double c1, double c2, PcgScalars* sc, double* partials,
                          const SimScalars* ss, double dt, double stim_duration, cudaStream_t s);
cudaError_t launch_update(double* x, double* r, const double* p, const double* q, int64_t n,
                          PcgScalars* sc, double* partials, cudaGraphConditionalHandle cond,
                          int use_cond, cudaStream_t s);
cudaError_t launch_direction(double* p, const double* z, int64_t n, const PcgScalars* sc,
                             cudaStream_t s);
cudaError_t launch_identity_dots(const double* r, const double* q, int64_t n, PcgScalars* sc,
                                 double* partials, cudaStream_t s);
cudaError_t launch_restrict(int np, int nq, const double* r, const double* T,
                            const int64_t* agg_ptr, const int32_t* agg_cells, int n_agg,
                            double* r0, const int* done, cudaStream_t s);
cudaError_t launch_prolong(int np, int nq, double* z, const double* T, const int32_t* agg,
                           const double* y0, int64_t nc, const double* r, const double* q,
                           PcgScalars* sc, double* partials, cudaStream_t s);
cudaError_t launch_gemv(const GemvBlock* blocks, const GemvTile* tiles, int ntiles, int rows,
                        int max_ld, const double* st64, const float* st32,
                        const __nv_bfloat16* st16, const double* r, const double* r0,
                        double* z, double* y0, const int* done, cudaStream_t s);
cudaError_t set_gemv_smem(int max_ld);
cudaError_t launch_permute(const double* src, double* dst, const int64_t* to_caller, int64_t nc,
                           int np, int to_internal, const PcgScalars* zero_if_b0, cudaStream_t s);
cudaError_t launch_copy(const double* src, double* dst, int64_t n, const SimScalars* ss,
                        cudaStream_t s);
cudaError_t launch_extract_local(const DeviceMatrix& K, const int64_t* sub_ptr, int n_sub,
                                 const int64_t* mat_off, const int32_t* ld, double* dense,
                                 int np, cudaStream_t s);
cudaError_t launch_chol_inverse(double* store, const int64_t* mat_off, const int32_t* nrow,
                                const int32_t* ld, double* work, const int64_t* work_off,
                                const int32_t* wld, int* status, int nmat, int max_n,
                                cudaStream_t s);
cudaError_t launch_cast_store(const double* src, float* d32, __nv_bfloat16* d16, int64_t n,
                              cudaStream_t s);

// Ionic update + ion-current load (Eq. fully-discrete-1).
cudaError_t launch_ionic(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                         const double* node_w, const double* node_phi, double* y, int64_t nn,
                         int64_t nc, double dt, double* I, const SimScalars* ss, cudaStream_t s);
cudaError_t launch_node_gather(const double* y_int, double* y_caller,
                               const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s);
cudaError_t launch_step_finish(double* U, double* Uprev, const double* x, int64_t n,
                               const PcgScalars* sc, SimScalars* ss, cudaStream_t s);
cudaError_t launch_step_begin(PcgScalars* sc, const SimScalars* ss, cudaStream_t s);
cudaError_t launch_init_y(double* y, int64_t nn, const double* y0, cudaStream_t s);

}  // namespace polydg
