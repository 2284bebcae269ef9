// noalloc.cu -- edp_solve without a caller workspace.
//
// For callers that cannot allocate device memory at all: code whose device
// memory is entirely reserved up front by another allocator (a host
// framework's fixed pool, an embedded or real-time loop with a fixed budget),
// or code that must not call cudaMalloc because cudaMalloc may synchronise
// the device.  Such a caller still passes its own inputs and outputs; the
// scratch space of the solve is a fixed-size array in the library's own
// device memory instead.
#include <mutex>

#include <cuda_runtime.h>

#include "edp.h"

namespace {

// The scratch of edp_solve_noalloc.  Every GPU that loads the library holds
// these EDP_NOALLOC_SCRATCH_BYTES until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[EDP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.  The
// cached address belongs to the device's primary context: after a
// cudaDeviceReset of that device it is stale (see edp.h).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EDP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return EDP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EDP_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EDP_OK;
}

}  // namespace

extern "C" int edp_solve_noalloc(const int32_t *C, int W, int H, const edp_label_space *space,
                                 const edp_params *params, int32_t *labels, edp_stream_t stream) {
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc) return rc;
    // edp_solve with the array as its workspace: the same argument checks in
    // the same order, so the same codes (EDP_ERR_WORKSPACE when the problem
    // needs more than the array holds).  It clears the status word, the
    // counters and the hand-off records it uses at the start of every call;
    // the message arrays need no clearing.
    return edp_solve(C, W, H, space, params, labels, ws, EDP_NOALLOC_SCRATCH_BYTES, stream);
}

extern "C" int edp_noalloc_get_device_status(int *status, edp_stream_t stream) {
    if (!status) return EDP_ERR_INVALID_ARG;
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc) return rc;
    return edp_get_device_status(ws, EDP_NOALLOC_SCRATCH_BYTES, status, stream);
}
