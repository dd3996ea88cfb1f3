// k_sk_static.cu -- the stateless structure factor rho(k_d) = sum_j q_j
// e^{i k_d . r_j} with its scratch in a fixed device array of this module
// instead of a caller workspace, so that the call allocates nothing.
//
// Who needs it: a host program that embeds the electrostatics in its own MD
// loop and has handed all device memory to its own pool, or that keeps work
// running on other streams, cannot let a library call reach cudaMalloc or
// cudaFree: the first can fail or fragment a fixed budget in the middle of a
// run, the second waits for the whole device.  Such a caller passes only its
// inputs and outputs and this entry point uses the module's scratch.
//
// Limits: the scratch holds kSkStaticBytes; a call that needs more (see
// sk_stateless_workspace) is refused before anything is launched.  There is
// one scratch per device, so calls on one device must not overlap in time (two
// streams running this entry point at once race on the same bytes).  Nothing
// in the scratch has to start at zero: every byte a call reads it has written
// earlier in the same call.  The first call on a device does a one-time
// set-up (it looks up the scratch's device address with that device
// current); make that first call before any stream capture begins.
#include <mutex>

#include "internal.h"

namespace rbsog {

namespace {

constexpr int kMaxDevices = 64;
__device__ __align__(256) unsigned char g_sk_scratch[kSkStaticBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

// Device address of this device's scratch (set up on first use, with the
// device current).  Returns the CUDA error of the set-up, if any.
cudaError_t sk_static_scratch(void **ptr)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sk_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace rbsog
