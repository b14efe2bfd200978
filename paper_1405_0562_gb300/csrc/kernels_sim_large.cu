// Simulation-mode (Alg. 3) instances for 65..256 kept states: vectors of 128
// and 256 entries, kept in shared memory (one byte per state and chunk).
#include "launch.h"
#include "sfa_device.cuh"

namespace sfa_impl {

using sfa_dev::sfa_match_kernel;

#define SIML_K(T, C, NQ) reinterpret_cast<const void *>(&sfa_match_kernel<T, C, NQ, false>)

#define SIMLB_K(T, NQ) reinterpret_cast<const void *>(&sfa_match_kernel<T, 1, NQ, true>)

const void *kernel_for_sim_batch_large(int threads, int simnq) {
    if (threads == 256 && simnq == 128) return SIMLB_K(256, 128);
    if (threads == 256 && simnq == 256) return SIMLB_K(256, 256);
    return nullptr;
}

const void *kernel_for_sim_large(int threads, int chains, int simnq) {
    if (threads == 128 && chains == 1 && simnq == 128) return SIML_K(128, 1, 128);
    if (threads == 128 && chains == 1 && simnq == 256) return SIML_K(128, 1, 256);
    if (threads == 256 && chains == 1 && simnq == 128) return SIML_K(256, 1, 128);
    if (threads == 256 && chains == 1 && simnq == 256) return SIML_K(256, 1, 256);
    return nullptr;
}

}  // namespace sfa_impl
