// Kernel registry shared by the instantiation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "sfa.h"
#include "sfa_types.h"

namespace sfa_impl {

// The kernel instance for a launch shape, or nullptr if it is not built.
//   simnq 0 = D-SFA mode, 16/32/64/128/256 = simulation with vectors of that size
//   wt = warp tiles (single texts, one chunk per thread)
const void *kernel_for(int threads, int chains, int simnq, bool batch, bool wt = false);
const void *kernel_for_sfa(int threads, int chains, bool batch);
const void *kernel_for_sim(int threads, int chains, int simnq);
const void *kernel_for_sim_large(int threads, int chains, int simnq);
const void *kernel_for_sim_batch(int threads, int simnq);
const void *kernel_for_sim_batch_large(int threads, int simnq);
const void *kernel_for_wt(int threads, int simnq);
// 16-bit state ids (more than 256 kept states): single texts, CTA tiles
const void *kernel_for_wide(int threads, int chains);
size_t smem_bytes_wide(int threads, int chains, uint32_t nr_max, uint32_t ncls);

// Dynamic shared memory of a launch shape (simnq: the simulation vector size,
// 0 in D-SFA mode).
size_t smem_bytes(int threads, int chains, uint32_t nr_max, int simnq = 0);
size_t smem_bytes_common(int threads, int chains, uint32_t nr_max);

// The D-SFA match of sfa_match with automatic shape, on a caller-provided
// scratch buffer of `cap` bytes that lives on device `scratch_device`.
// Allocates nothing; SFA_ERR_SCRATCH_LIMIT if the launch needs more.
int match_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
                       uint8_t *scratch, size_t cap, int scratch_device);
// The refusals of match_into_scratch, all taken before any work is enqueued:
// arguments, mode, a handle without device tables or on another device, and
// the scratch the text would need (SFA_ERR_SCRATCH_LIMIT).
int check_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, const sfa_result *d_out, size_t cap);

// The slice mapping of sfa_match_map: enqueue one small kernel that composes
// the `tiles` tile aggregates (agg, tile t at agg + t*nr, in tile order) and
// writes d_map[q] for every caller state q (-1 for states not kept).
int launch_compose_tiles(const uint8_t *agg, uint32_t tiles, uint32_t nr, const int32_t *orig_of, uint32_t nq_in,
                         int32_t *d_map, cudaStream_t s);

}  // namespace sfa_impl
