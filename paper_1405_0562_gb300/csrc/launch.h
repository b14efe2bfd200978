// Kernel registry shared by the instantiation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "sfa_types.h"

namespace sfa_impl {

// The kernel instance for a launch shape, or nullptr if it is not built.
//   simnq 0 = D-SFA mode, 16/32/64 = simulation with vectors of that size
const void *kernel_for(int threads, int chains, int simnq, bool batch);
const void *kernel_for_sfa(int threads, int chains, bool batch);
const void *kernel_for_sim(int threads, int chains, int simnq);

// Dynamic shared memory of a launch shape.
size_t smem_bytes(int threads, int chains, uint32_t nr_max);

}  // namespace sfa_impl
