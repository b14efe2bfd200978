// Copy-in of a batch's texts from host memory the device can read (pinned,
// mapped) into device buffers with one kernel launch, instead of one
// cudaMemcpyAsync per text (each of which costs microseconds of host time:
// at the serving workload's 64 KiB median that bound the copy-in to about
// 20 GB/s).  The texts are cut into GATHER_UNIT-byte units; CTAs take units
// in a grid-stride loop and find a unit's text by binary search over the
// units' prefix sums.
#include <cuda.h>
#include <cuda_runtime.h>

#include "api_internal.h"

namespace sfa_impl {

namespace {

constexpr int GATHER_THREADS = 256;
constexpr uint32_t GATHER_LOADS = 4;   // 16-byte loads in flight per thread

__global__ void __launch_bounds__(GATHER_THREADS) gather_kernel(const GatherDesc *g, const uint32_t *unit0,
                                                                 uint32_t k) {
    __shared__ uint32_t s_cnt;
    const uint32_t total = unit0[k];
    for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
        // the text of unit u: the last r with unit0[r] <= u, i.e. the number
        // of such r less one (unit0 strictly increases from unit0[0] = 0: a
        // text of the copy has at least one unit), counted by the whole block
        // with independent loads, not a chain of dependent ones
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        uint32_t c = 0;
        for (uint32_t r = threadIdx.x; r < k; r += GATHER_THREADS) c += unit0[r] <= u ? 1u : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31u) == 0 && c) atomicAdd(&s_cnt, c);
        __syncthreads();
        const uint32_t lo = s_cnt - 1u;
        __syncthreads();   // s_cnt is read before the next unit resets it
        const GatherDesc d = g[lo];
        const uint64_t b = (uint64_t)(u - unit0[lo]) * GATHER_UNIT;
        const uint64_t e = min(d.len, b + GATHER_UNIT);
        const uint8_t *src = d.src;
        uint8_t *dst = d.dst;
        if (((reinterpret_cast<uintptr_t>(src) ^ reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
            // same alignment on both sides: bytes up to the first 16-byte
            // boundary, 16-byte vectors, then the last bytes
            const uint64_t a = min(e, b + ((16u - ((reinterpret_cast<uintptr_t>(src) + b) & 15u)) & 15u));
            const uint64_t z = a + ((e - a) & ~(uint64_t)15);
            for (uint64_t p = b + threadIdx.x; p < a; p += GATHER_THREADS) dst[p] = src[p];
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src + a);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst + a);
            const uint64_t n4 = (z - a) >> 4;
            for (uint64_t i = threadIdx.x; i < n4; i += GATHER_THREADS * GATHER_LOADS) {
                uint4 v[GATHER_LOADS];
#pragma unroll
                for (uint32_t j = 0; j < GATHER_LOADS; ++j)
                    if (i + j * GATHER_THREADS < n4) v[j] = s4[i + j * GATHER_THREADS];
#pragma unroll
                for (uint32_t j = 0; j < GATHER_LOADS; ++j)
                    if (i + j * GATHER_THREADS < n4) d4[i + j * GATHER_THREADS] = v[j];
            }
            for (uint64_t p = z + threadIdx.x; p < e; p += GATHER_THREADS) dst[p] = src[p];
        } else {
            for (uint64_t p = b + threadIdx.x; p < e; p += GATHER_THREADS) dst[p] = src[p];
        }
    }
}

}  // namespace

int launch_gather(const GatherDesc *d_descs, const uint32_t *d_unit0, uint32_t k, uint32_t units, cudaStream_t s) {
    if (k == 0 || units == 0) return SFA_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // a few CTAs per SM keep enough 16-byte loads in flight to cover the
    // host link's latency; more would only wait
    const uint32_t grid = std::min<uint32_t>(units, 2u * (uint32_t)std::max(1, device_props(dev).sms));
    gather_kernel<<<grid, GATHER_THREADS, 0, s>>>(d_descs, d_unit0, k);
    CK(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

const uint8_t *device_readable(const uint8_t *h, ReadableRange *cache) {
    const uintptr_t p = reinterpret_cast<uintptr_t>(h);
    if (cache && cache->hi && p >= cache->lo && p < cache->hi)
        return reinterpret_cast<const uint8_t *>(p + cache->delta);
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();   // clear the error of an unknown pointer
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    if (cache) {
        // the allocation's range, from the driver, so that the next texts of
        // the same allocation need no query
        using GetAttr = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
        static GetAttr get = [] {
            void *f = nullptr;
            cudaDriverEntryPointQueryResult q{};
            if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess) {
                cudaGetLastError();
                return (GetAttr) nullptr;
            }
            return reinterpret_cast<GetAttr>(f);
        }();
        CUdeviceptr lo = 0;
        size_t size = 0;
        if (get && get(&lo, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)p) == CUDA_SUCCESS &&
            get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)p) == CUDA_SUCCESS && size &&
            p >= (uintptr_t)lo && p < (uintptr_t)lo + size) {
            cache->lo = (uintptr_t)lo;
            cache->hi = (uintptr_t)lo + size;
            cache->delta = reinterpret_cast<uintptr_t>(a.devicePointer) - p;
        }
    }
    return static_cast<const uint8_t *>(a.devicePointer);
}

}  // namespace sfa_impl
