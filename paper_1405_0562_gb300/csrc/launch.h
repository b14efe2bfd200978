// Kernel registry shared by the instantiation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "sfa.h"
#include "sfa_types.h"

namespace sfa_impl {

// The kernel instance for a launch shape, or nullptr if it is not built.
//   simnq 0 = D-SFA mode, 16/32/64 = simulation with vectors of that size
//   wt = warp tiles (single texts, one chunk per thread)
const void *kernel_for(int threads, int chains, int simnq, bool batch, bool wt = false);
const void *kernel_for_sfa(int threads, int chains, bool batch);
const void *kernel_for_sim(int threads, int chains, int simnq);
const void *kernel_for_wt(int threads, int simnq);

// Dynamic shared memory of a launch shape.
size_t smem_bytes(int threads, int chains, uint32_t nr_max);

// The D-SFA match of sfa_match with automatic shape, on a caller-provided
// scratch buffer of `cap` bytes that lives on device `scratch_device`.
// Allocates nothing; SFA_ERR_SCRATCH_LIMIT if the launch needs more.
int match_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
                       uint8_t *scratch, size_t cap, int scratch_device);
// The checks of match_into_scratch that need no device: arguments, mode and
// the scratch the text would need (SFA_ERR_SCRATCH_LIMIT).
int check_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, const sfa_result *d_out, size_t cap);

}  // namespace sfa_impl
