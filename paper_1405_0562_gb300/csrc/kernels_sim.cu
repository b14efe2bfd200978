// Simulation-mode (Alg. 3) instances of the persistent matching kernel.
#include "launch.h"
#include "sfa_device.cuh"

namespace sfa_impl {

using sfa_dev::sfa_match_kernel;

#define SIM_K(T, C, NQ) reinterpret_cast<const void *>(&sfa_match_kernel<T, C, NQ, false>)
#define SIMB_K(T, NQ) reinterpret_cast<const void *>(&sfa_match_kernel<T, 1, NQ, true>)

// batches of simulation-mode texts: one persistent launch per vector size
const void *kernel_for_sim_batch(int threads, int simnq) {
    if (threads == 128 && simnq == 16) return SIMB_K(128, 16);
    if (threads == 128 && simnq == 32) return SIMB_K(128, 32);
    if (threads == 128 && simnq == 64) return SIMB_K(128, 64);
    return kernel_for_sim_batch_large(threads, simnq);
}

const void *kernel_for_sim(int threads, int chains, int simnq) {
    if (threads == 128 && chains == 1 && simnq == 16) return SIM_K(128, 1, 16);
    if (threads == 128 && chains == 1 && simnq == 32) return SIM_K(128, 1, 32);
    if (threads == 128 && chains == 1 && simnq == 64) return SIM_K(128, 1, 64);
    if (threads == 256 && chains == 1 && simnq == 16) return SIM_K(256, 1, 16);
    if (threads == 256 && chains == 1 && simnq == 32) return SIM_K(256, 1, 32);
    if (threads == 256 && chains == 1 && simnq == 64) return SIM_K(256, 1, 64);
    if (threads == 128 && chains == 2 && simnq == 16) return SIM_K(128, 2, 16);
    if (threads == 128 && chains == 2 && simnq == 32) return SIM_K(128, 2, 32);
    return kernel_for_sim_large(threads, chains, simnq);
}

}  // namespace sfa_impl
