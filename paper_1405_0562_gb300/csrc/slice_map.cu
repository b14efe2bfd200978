// The mapping of a text slice (sfa_match_map): the reverse composition, in
// tile order, of the tile aggregates that a map-mode launch of the matching
// kernel leaves in scratch (Lemma 1: the mapping of w = w_1 w_2 ... w_k is
// f_{w_1} . f_{w_2} . ... . f_{w_k}).
#include <cuda_runtime.h>

#include "api_internal.h"

namespace sfa_impl {

namespace {

constexpr int COMPOSE_THREADS = 256;   // one thread per kept state (nr <= 256)
constexpr uint32_t COMPOSE_TILES = 32; // tile vectors staged in shared memory per round

// Thread q follows state q through every tile vector in order; the vectors
// are staged COMPOSE_TILES at a time with coalesced loads.
__global__ void __launch_bounds__(COMPOSE_THREADS) compose_tiles_kernel(const uint8_t *agg, uint32_t tiles,
                                                                         uint32_t nr, const int32_t *orig_of,
                                                                         uint32_t nq_in, int32_t *d_map) {
    __shared__ uint8_t blk[COMPOSE_TILES * 256];
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < nq_in; i += COMPOSE_THREADS) d_map[i] = -1;
    uint32_t v = tid;
    for (uint32_t t0 = 0; t0 < tiles; t0 += COMPOSE_TILES) {
        const uint32_t nt = min(COMPOSE_TILES, tiles - t0);
        __syncthreads();
        for (uint32_t i = tid; i < nt * nr; i += COMPOSE_THREADS) {
            const uint32_t t = i / nr, q = i - t * nr;
            blk[t * 256 + q] = agg[(size_t)(t0 + t) * nr + q];
        }
        __syncthreads();
        if (tid < nr)
            for (uint32_t t = 0; t < nt; ++t) v = blk[t * 256 + v];
    }
    // the -1 fill above is ordered before the images of the kept states
    __syncthreads();
    if (tid < nr) d_map[orig_of[tid]] = orig_of[v];
}

}  // namespace

int launch_compose_tiles(const uint8_t *agg, uint32_t tiles, uint32_t nr, const int32_t *orig_of, uint32_t nq_in,
                         int32_t *d_map, cudaStream_t s) {
    if (nr == 0 || nr > 256) return SFA_ERR_UNSUPPORTED;
    compose_tiles_kernel<<<1, COMPOSE_THREADS, 0, s>>>(agg, tiles, nr, orig_of, nq_in, d_map);
    CK(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

}  // namespace sfa_impl
