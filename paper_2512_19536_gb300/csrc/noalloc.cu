// polydg_spd_inverse_static: in-place inversion of a batch of symmetric positive
// definite float64 matrices, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is owned by
// another allocator (a framework's caching allocator, or a fixed arena reserved up
// front by an embedded or real-time runtime, where a stray cudaMalloc would take
// memory the arena counted on), or code that must not fail on allocation in the
// middle of a time step.  This entry point needs nothing from them but the
// matrices: the kernel's workspace lives in one file-scope static device array
// of fixed size, set aside when the library is loaded.
//
// It runs the same kernel as asm_setup's local and coarse inversions (Cholesky
// factorisation, triangular inverse, product of the inverse factors).
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "polydg.h"

namespace polydg {

constexpr int kStaticMaxBatch = 256;                  // matrices per call
constexpr int64_t kStaticWorkDoubles = int64_t(1) << 20;  // 8 MiB: sum of roundup(n, 32)^2
constexpr int kStaticMaxN = 1024;                     // order of each matrix
constexpr int kMaxDevices = 64;

// Layout of the scratch array: [workspace doubles][descriptors][status].
struct StaticDesc {
    int64_t mat_off[kStaticMaxBatch];
    int64_t work_off[kStaticMaxBatch];
    int32_t nrow[kStaticMaxBatch];
    int32_t ld[kStaticMaxBatch];
    int32_t wld[kStaticMaxBatch];
    int32_t status[kStaticMaxBatch];
};
constexpr size_t kStaticBytes = (size_t)kStaticWorkDoubles * sizeof(double) + sizeof(StaticDesc);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch per device (a host-side symbol is only a
// stand-in for it, not a device address).
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mutex;

static int static_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("polydg_spd_inverse_static: device index out of range");
        return POLYDG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("polydg_spd_inverse_static: cudaGetSymbolAddress: ") +
                      cudaGetErrorString(e));
            return POLYDG_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return POLYDG_OK;
}

}  // namespace polydg

using namespace polydg;

extern "C" int polydg_spd_inverse_static(double* mats_dev, int n, int ld, int batch,
                                         void* stream) {
    if (!mats_dev || n < 1 || ld < n || batch < 1) {
        set_error("polydg_spd_inverse_static: need a matrix pointer, n >= 1, ld >= n, batch >= 1");
        return POLYDG_EINVAL;
    }
    const int64_t wld = (n + 31) / 32 * 32;
    if (n > kStaticMaxN || batch > kStaticMaxBatch || wld * wld * batch > kStaticWorkDoubles) {
        set_error("polydg_spd_inverse_static: batch too large for the static workspace (n <= 1024, "
                  "batch <= 256, batch * roundup(n, 32)^2 <= 1048576 doubles)");
        return POLYDG_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_error("polydg_spd_inverse_static: no CUDA device");
        return POLYDG_ECUDA;
    }
    // the matrices must live on the current device: the kernel runs there, and a pointer
    // to another GPU's (or host) memory would be read through the wrong address space
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, mats_dev) != cudaSuccess ||
        (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) || attr.device != dev) {
        cudaGetLastError();
        set_error("polydg_spd_inverse_static: mats_dev is not device memory of the current device");
        return POLYDG_EINVAL;
    }
    unsigned char* base = nullptr;
    if (int st = static_scratch(dev, &base)) return st;
    double* work = reinterpret_cast<double*>(base);
    StaticDesc* desc = reinterpret_cast<StaticDesc*>(base + (size_t)kStaticWorkDoubles * sizeof(double));
    cudaStream_t s = (cudaStream_t)stream;

    StaticDesc h;
    std::memset(&h, 0, sizeof(h));
    for (int m = 0; m < batch; ++m) {
        h.mat_off[m] = (int64_t)m * n * ld;
        h.work_off[m] = (int64_t)m * wld * wld;
        h.nrow[m] = n;
        h.ld[m] = ld;
        h.wld[m] = (int32_t)wld;
    }
    // the array keeps the previous call's contents: the triangular workspace must
    // start at zero, the descriptors and status are rewritten
    cudaError_t e = cudaMemsetAsync(work, 0, (size_t)wld * wld * batch * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(desc, &h, sizeof(StaticDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_chol_inverse(mats_dev, desc->mat_off, desc->nrow, desc->ld, work, desc->work_off,
                                desc->wld, desc->status, batch, n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.status, desc->status, batch * sizeof(int32_t),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("polydg_spd_inverse_static: ") + cudaGetErrorString(e));
        return POLYDG_ECUDA;
    }
    for (int m = 0; m < batch; ++m)
        if (h.status[m] != 0) {
            set_error("polydg_spd_inverse_static: a matrix is not positive definite");
            return POLYDG_ENOTSPD;
        }
    return POLYDG_OK;
}
