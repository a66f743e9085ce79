// commet_const_backward_noalloc: the backward of the constitutive update for callers
// that cannot allocate device memory.
//
// Who needs it: a host application that owns every byte of device memory (a solver
// that reserves a fixed budget at start-up and treats any later allocation as a fault,
// or a plugin host whose ABI gives the library no way to receive a workspace pointer)
// cannot call cudaMalloc itself and has no buffer to hand over for the backward's
// per-CTA partial sums. This entry point keeps that scratch in a fixed array compiled
// into the library instead, and calls no allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// its COMMET_NOALLOC_SCRATCH_BYTES until the process exits. Host code cannot use the
// array's name as a device address (in host code it names a host-side stand-in), so the
// first call on each device, with that device current, looks the address up with
// cudaGetSymbolAddress and caches it; make that first call before any stream capture.
// The cache is keyed by device ordinal only: a device reset, which can load the module
// at a new address, voids it, and the entry point must not be used after one until the
// library is loaded anew.
// All calls share the one array and it keeps the last call's contents; the kernel
// writes every scratch word before reading it, so nothing has to start at zero. Calls
// whose kernels overlap on the GPU (other streams, other host threads) race on the
// array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_backward_scratch[COMMET_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_backward_scratch on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return COMMET_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return COMMET_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_backward_scratch) != cudaSuccess || p == nullptr) return COMMET_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return COMMET_OK;
}

bool aligned16(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int commet_const_backward_noalloc(const commet_model *m, int64_t n_qp, const void *F, const void *dL_dP,
                                             void *dL_dF, void *dL_dtheta, void *stream) {
    if (m == nullptr || n_qp < 0 || dL_dtheta == nullptr) return COMMET_ERR_INVALID_ARG;
    if (m->inner != COMMET_INNER_MICNN) return COMMET_ERR_UNSUPPORTED;
    if (n_qp > 0 && (F == nullptr || dL_dP == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(F) || !aligned16(dL_dP) || !aligned16(dL_dF) || !aligned16(dL_dtheta)) return COMMET_ERR_INVALID_ARG;
    if (m->kp.stress_free) return COMMET_ERR_UNSUPPORTED;
    const size_t need = commet::backward_workspace_bytes(m, n_qp);
    if (need > (size_t)COMMET_NOALLOC_SCRATCH_BYTES) return COMMET_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != COMMET_OK) return rc;
    return commet::launch_const_backward(m, n_qp, F, dL_dP, dL_dF, dL_dtheta, scratch, need,
                                         reinterpret_cast<cudaStream_t>(stream));
}
