// Material-form constitutive update entry: P [9][n], A [81][n] per point.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstdint>

#include "update_kernel.cuh"

namespace commet {

__global__ void status_init_kernel(int32_t *status) {
    status[0] = 0;
    status[1] = INT32_MAX;
}

int launch_status_init(int32_t *status, cudaStream_t s) {
    status_init_kernel<<<1, 1, 0, s>>>(status);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_sm_count[kMaxDevices];  // 0 = not looked up yet
}  // namespace

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int n = dev < kMaxDevices ? g_sm_count[dev].load(std::memory_order_relaxed) : 0;
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        // a racing first lookup on the same device stores the same value
        if (dev < kMaxDevices) g_sm_count[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

int launch_const_update(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, cudaStream_t s, void *dN_out) {
    if (status != nullptr) {
        int rc = launch_status_init(status, s);
        if (rc != COMMET_OK) return rc;
    }
    if (n_qp == 0) return COMMET_OK;
    if (m->precision == COMMET_F64) return dispatch<double, false>(m, n_qp, F, psi, P, A, status, s, dN_out);
    if (m->precision == COMMET_F32) return dispatch<float, false>(m, n_qp, F, psi, P, A, status, s, dN_out);
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
