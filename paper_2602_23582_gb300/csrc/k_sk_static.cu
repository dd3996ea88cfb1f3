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
// sk_stateless_workspace) is refused before anything is launched.  The array
// is a module global, so there is one scratch per CUDA context (the primary
// context of a device, or each context a driver-API caller creates); calls in
// one context must not overlap in time (two streams running this entry point
// at once race on the same bytes).  Nothing in the scratch has to start at
// zero: every byte a call reads it has written earlier in the same call.
// The first call in a context does a one-time set-up (it looks up the
// scratch's device address in that context, which also loads the module
// there); make that first call before any stream capture begins.  The address
// is cached per device together with the unique id of the context it was
// looked up in, and looked up again when a call comes from another context
// (after cudaDeviceReset, or from a context of the caller's own), so a call
// never hands a kernel an address of another or a destroyed context.
#include <mutex>

#include <cuda.h>

#include "internal.h"

namespace rbsog {

namespace {

constexpr int kMaxDevices = 64;
__device__ __align__(256) unsigned char g_sk_scratch[kSkStaticBytes];

std::mutex g_setup_mu;
struct ScratchAddr {
    void *ptr = nullptr;
    unsigned long long ctx_id = 0;   // unique id of the context ptr belongs to
};
ScratchAddr g_scratch[kMaxDevices];

// Driver calls that name the current context, resolved once through the
// runtime (the library does not link the driver library itself).
using PfnCtxGetCurrent = CUresult (*)(CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);
PfnCtxGetCurrent g_get_current = nullptr;
PfnCtxGetId g_get_id = nullptr;
bool g_resolved = false;

// Unique id of the calling thread's current context; false when there is
// none yet or the driver cannot say (then the address is looked up again).
bool current_ctx_id(unsigned long long *id)
{
    if (!g_resolved) {
        g_resolved = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_get_id = reinterpret_cast<PfnCtxGetId>(f);
    }
    if (!g_get_current || !g_get_id) return false;
    CUcontext c = nullptr;
    if (g_get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
    return g_get_id(c, id) == CUDA_SUCCESS;
}

}  // namespace

// Device address of the scratch in the calling thread's current context (the
// lookup happens on the first call in a context; it also initialises the
// device's primary context when nothing is current yet).  Returns the CUDA
// error of the lookup, if any.
cudaError_t sk_static_scratch(void **ptr)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    unsigned long long id = 0;
    if (current_ctx_id(&id) && g_scratch[dev].ptr && g_scratch[dev].ctx_id == id) {
        *ptr = g_scratch[dev].ptr;
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sk_scratch);
    if (e != cudaSuccess) return e;
    // after the lookup a context is current: remember which one
    if (current_ctx_id(&id)) {
        g_scratch[dev].ptr = p;
        g_scratch[dev].ctx_id = id;
    } else {
        g_scratch[dev].ptr = nullptr;   // no id to key on: look up on every call
    }
    *ptr = p;
    return cudaSuccess;
}

}  // namespace rbsog
