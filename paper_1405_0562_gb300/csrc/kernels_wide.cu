// 16-bit-id instances of the persistent matching kernel (automata with more
// than 256 kept states): single texts, CTA tiles, D-SFA mode.
#include "launch.h"
#include "sfa_device.cuh"

namespace sfa_impl {

using sfa_dev::sfa_match_kernel;

#define WIDE_K(T, C) reinterpret_cast<const void *>(&sfa_match_kernel<T, C, 0, false, false, true>)

const void *kernel_for_wide(int threads, int chains) {
    if (threads == 128 && chains == 1) return WIDE_K(128, 1);
    if (threads == 256 && chains == 1) return WIDE_K(256, 1);
    if (threads == 256 && chains == 2) return WIDE_K(256, 2);
    if (threads == 512 && chains == 1) return WIDE_K(512, 1);
    if (threads == 1024 && chains == 1) return WIDE_K(1024, 1);
    return nullptr;
}

size_t smem_bytes_wide(int threads, int chains, uint32_t nr_max, uint32_t ncls) {
    using namespace sfa_dev;
    switch (threads * 8 + chains) {
        case 128 * 8 + 1: return SmemLayout<128, 1, 0, true>::bytes(nr_max, ncls);
        case 256 * 8 + 1: return SmemLayout<256, 1, 0, true>::bytes(nr_max, ncls);
        case 256 * 8 + 2: return SmemLayout<256, 2, 0, true>::bytes(nr_max, ncls);
        case 512 * 8 + 1: return SmemLayout<512, 1, 0, true>::bytes(nr_max, ncls);
        case 1024 * 8 + 1: return SmemLayout<1024, 1, 0, true>::bytes(nr_max, ncls);
        default: return 0;
    }
}

}  // namespace sfa_impl
