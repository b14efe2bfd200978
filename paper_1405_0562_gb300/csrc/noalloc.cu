// sfa_match_noalloc: the D-SFA match for callers that must not allocate
// device memory while matching (see include/sfa.h).  The kernel's scratch is
// one fixed array in device memory, compiled into the library; host code
// only ever passes its device address, looked up once per device.
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "sfa.h"

namespace {

// Scratch of sfa_match_noalloc.  In host code this name is only a stand-in
// for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SFA_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of the array on the current device; looked up on the first
// call for that device.
int scratch_address(uint8_t **out, int *dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? SFA_ERR_NO_DEVICE : SFA_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return SFA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return SFA_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = static_cast<uint8_t *>(g_addr[dev]);
    *dev_out = dev;
    return SFA_OK;
}

}  // namespace

extern "C" int sfa_match_noalloc(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out,
                                 sfa_stream_t stream) {
    // every check that needs no device first: a text that does not fit is
    // rejected before anything touches the GPU
    int rc = sfa_impl::check_into_scratch(h, d_text, n, d_out, SFA_NOALLOC_SCRATCH_BYTES);
    if (rc) return rc;
    uint8_t *scratch = nullptr;
    int dev = -1;
    rc = scratch_address(&scratch, &dev);
    if (rc) return rc;
    return sfa_impl::match_into_scratch(h, d_text, n, d_out, (cudaStream_t)stream, scratch,
                                        SFA_NOALLOC_SCRATCH_BYTES, dev);
}
