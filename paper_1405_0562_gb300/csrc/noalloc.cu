// sfa_match_noalloc: the D-SFA match for callers that must not allocate
// device memory while matching (see include/sfa.h).  The kernel's scratch is
// one fixed array in device memory, compiled into the library; host code
// only ever passes its device address, looked up on every call.
#include <cuda_runtime.h>

#include "launch.h"
#include "sfa.h"

namespace {

// Scratch of sfa_match_noalloc.  In host code this name is only a stand-in
// for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SFA_NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device.  Looked up on every
// call (the lookup allocates nothing) rather than cached, so that an address
// never outlives the context it was taken in (cudaDeviceReset, a new primary
// context).  The first lookup on a device loads the library's device code
// there if it is not loaded yet.
int scratch_address(uint8_t **out, int *dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? SFA_ERR_NO_DEVICE : SFA_ERR_CUDA;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return SFA_ERR_CUDA;
    *out = static_cast<uint8_t *>(p);
    *dev_out = dev;
    return SFA_OK;
}

}  // namespace

extern "C" int sfa_match_noalloc(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out,
                                 sfa_stream_t stream) {
    // every refusal first (arguments, mode, the handle's device, a text whose
    // scratch would not fit): nothing is enqueued and the array's address is
    // not looked up unless the call can go ahead
    int rc = sfa_impl::check_into_scratch(h, d_text, n, d_out, SFA_NOALLOC_SCRATCH_BYTES);
    if (rc) return rc;
    uint8_t *scratch = nullptr;
    int dev = -1;
    rc = scratch_address(&scratch, &dev);
    if (rc) return rc;
    return sfa_impl::match_into_scratch(h, d_text, n, d_out, (cudaStream_t)stream, scratch,
                                        SFA_NOALLOC_SCRATCH_BYTES, dev);
}
