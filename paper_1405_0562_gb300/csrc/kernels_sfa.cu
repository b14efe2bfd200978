// D-SFA-mode instances of the persistent matching kernel (single text and
// batch forms) for every supported launch shape.
#include "launch.h"
#include "sfa_device.cuh"

namespace sfa_impl {

using sfa_dev::sfa_match_kernel;

#define SFA_K(T, C, B) reinterpret_cast<const void *>(&sfa_match_kernel<T, C, 0, B>)
#define SFA_SHAPES(B)                                              \
    if (threads == 128 && chains == 1) return SFA_K(128, 1, B);    \
    if (threads == 128 && chains == 2) return SFA_K(128, 2, B);    \
    if (threads == 128 && chains == 4) return SFA_K(128, 4, B);    \
    if (threads == 256 && chains == 1) return SFA_K(256, 1, B);    \
    if (threads == 256 && chains == 2) return SFA_K(256, 2, B);    \
    if (threads == 256 && chains == 4) return SFA_K(256, 4, B);    \
    if (threads == 512 && chains == 1) return SFA_K(512, 1, B);    \
    if (threads == 512 && chains == 2) return SFA_K(512, 2, B);    \
    if (threads == 1024 && chains == 1) return SFA_K(1024, 1, B);

const void *kernel_for_sfa(int threads, int chains, bool batch) {
    if (batch) {
        SFA_SHAPES(true)
        return nullptr;
    }
    SFA_SHAPES(false)
    return nullptr;
}

size_t smem_bytes(int threads, int chains, uint32_t nr_max, int simnq) {
    using namespace sfa_dev;
    // simulation vectors of more than 64 entries live in shared memory after
    // the common layout (SmemLayout::vec_off)
    const size_t vec = simnq > 64 ? (size_t)threads * chains * simnq : 0;
    return smem_bytes_common(threads, chains, nr_max) + vec;
}

size_t smem_bytes_common(int threads, int chains, uint32_t nr_max) {
    using namespace sfa_dev;
    switch (threads * 8 + chains) {
        case 128 * 8 + 1: return SmemLayout<128, 1>::bytes(nr_max);
        case 128 * 8 + 2: return SmemLayout<128, 2>::bytes(nr_max);
        case 128 * 8 + 4: return SmemLayout<128, 4>::bytes(nr_max);
        case 256 * 8 + 1: return SmemLayout<256, 1>::bytes(nr_max);
        case 256 * 8 + 2: return SmemLayout<256, 2>::bytes(nr_max);
        case 256 * 8 + 4: return SmemLayout<256, 4>::bytes(nr_max);
        case 512 * 8 + 1: return SmemLayout<512, 1>::bytes(nr_max);
        case 512 * 8 + 2: return SmemLayout<512, 2>::bytes(nr_max);
        case 1024 * 8 + 1: return SmemLayout<1024, 1>::bytes(nr_max);
        default: return 0;
    }
}

const void *kernel_for(int threads, int chains, int simnq, bool batch, bool wt) {
    if (wt) return batch || chains != 1 ? nullptr : kernel_for_wt(threads, simnq);
    if (simnq == 0) return kernel_for_sfa(threads, chains, batch);
    if (batch) return chains == 1 ? kernel_for_sim_batch(threads, simnq) : nullptr;
    return kernel_for_sim(threads, chains, simnq);
}

}  // namespace sfa_impl
