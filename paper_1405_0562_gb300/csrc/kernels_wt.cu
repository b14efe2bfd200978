// Warp-tile instances of the persistent matching kernel (single texts): each
// warp takes its own tiles of 32 chunks, in D-SFA and in simulation mode.
#include "launch.h"
#include "sfa_device.cuh"

namespace sfa_impl {

using sfa_dev::sfa_match_kernel;

#define WT_K(T, NQ) reinterpret_cast<const void *>(&sfa_match_kernel<T, 1, NQ, false, true>)

const void *kernel_for_wt(int threads, int simnq) {
    if (simnq == 0) {
        if (threads == 256) return WT_K(256, 0);
        if (threads == 512) return WT_K(512, 0);
        if (threads == 1024) return WT_K(1024, 0);
        return nullptr;
    }
    if (threads == 128 && simnq == 16) return WT_K(128, 16);
    if (threads == 128 && simnq == 32) return WT_K(128, 32);
    if (threads == 128 && simnq == 64) return WT_K(128, 64);
    if (threads == 256 && simnq == 16) return WT_K(256, 16);
    if (threads == 256 && simnq == 32) return WT_K(256, 32);
    if (threads == 256 && simnq == 64) return WT_K(256, 64);
    return nullptr;
}

}  // namespace sfa_impl
