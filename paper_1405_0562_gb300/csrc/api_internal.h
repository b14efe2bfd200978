// Internals shared by the C ABI units (sfa_api.cpp, batch_api.cpp,
// noalloc.cu): the handle, launch shapes, scratch plans, launch helpers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "host_compile.h"
#include "launch.h"
#include "sfa.h"

namespace sfa_impl {

constexpr uint32_t DEFAULT_TIMEOUT_US = 2000000;   // 2 s per device-side wait
constexpr uint64_t WARP_TILE_ROUNDS = 1;           // automatic chunks: warp tiles per resident warp
// Two CTAs per SM: the share of the text (parts per million) given to the
// level of the CTA that starts first on each SM, which runs faster
#ifndef SFA_OLDER_SHARE_PPM
#define SFA_OLDER_SHARE_PPM 525000
#endif
constexpr uint64_t OLDER_SHARE_PPM = SFA_OLDER_SHARE_PPM;
constexpr uint64_t MAX_TEXT = 1ull << 40;
constexpr uint64_t MAX_CHUNK = 1ull << 31;         // per-chunk counters are 32-bit
constexpr uint32_t MAX_FORCED = 1u << 20;
constexpr uint64_t HOST_PIECE = 64ull << 20;       // sfa_match_host copy granularity

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return SFA_OK;
    if (e == cudaErrorMemoryAllocation) return SFA_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SFA_ERR_NO_DEVICE;
    return SFA_ERR_CUDA;
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return sfa_impl::cuda_err(e_); \
    } while (0)

extern std::atomic<uint64_t> g_launches;   // kernels enqueued since load

struct DeviceProps {
    int sms = 0;
    size_t smem_optin = 0;
};
DeviceProps device_props(int dev);

// resident CTAs per SM for a kernel instance and shared-memory size (cached;
// also raises the kernel's dynamic shared-memory limit)
int blocks_per_sm(const void *k, int threads, size_t smem);

struct Shape {
    int threads = 256;
    int chains = 2;
    int simnq = 0;
    uint64_t chunk = 1024;
    uint32_t forced = 0;
    int max_ctas = 0;
    uint32_t timeout_us = DEFAULT_TIMEOUT_US;
    uint32_t debug = 0;
    bool wt = false;   // warp tiles (32 chunks per tile) instead of CTA tiles
    bool auto_chunk = false;   // chunk length chosen by choose_shape
    int bps = 0;               // resident CTAs per SM (automatic chunks)
    int sms = 0;
    uint64_t tile_chunks() const { return wt ? 32u : (uint64_t)threads * chains; }
    // CTAs that have work for `tiles` tiles
    uint64_t ctas_for(uint64_t tiles) const { return wt ? (tiles + threads / 32 - 1) / (threads / 32) : tiles; }
};

inline int simnq_for(uint32_t nr) {
    return nr <= 16 ? 16 : nr <= 32 ? 32 : nr <= 64 ? 64 : nr <= 128 ? 128 : 256;
}

// scratch layout of a launch over `ntext` texts and `tiles` tiles
struct ScratchPlan {
    size_t off_texts, off_status, off_agg, off_vec, total, zero;
};
ScratchPlan plan_scratch(uint32_t ntext, uint64_t tiles, uint32_t nr_max, uint64_t vec_bytes);
sfa_dev::Scratch make_scratch(uint8_t *base, const ScratchPlan &p, uint32_t nr_max, uint32_t tiles,
                              const Shape &sh);

}  // namespace sfa_impl

struct sfa_handle {
    sfa_impl::HostTables host;
    bool on_device = false;
    int device = -1;
    uint8_t *d_tables = nullptr;
    size_t table_bytes = 0;
    sfa_dev::Tables dev{};
    uint8_t *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // sfa_match_host
    uint8_t *d_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    sfa_result *d_res = nullptr;
    sfa_result *h_res = nullptr;       // in-place matches: a mapped pinned result record
    sfa_result *h_res_dev = nullptr;   // its device address
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
};

namespace sfa_impl {

// launch shape for one text (automatic fields filled in)
int choose_shape(const sfa_handle *h, uint64_t n, const sfa_launch_opts *o, Shape &sh);
// grow the handle's scratch to at least `bytes` (may synchronise and cudaMalloc)
int ensure_scratch(sfa_handle *h, size_t bytes);
// If the text can be staged by 2-D tensor copies (16-byte-aligned text,
// chunks of a multiple of 16 bytes, not a forced chunk count), encode the
// tensor map of its full chunks and set d.rows2d; else leave d.rows2d = 0.
void fill_text_map(sfa_dev::TextDesc &d, CUtensorMap &map);
// enqueue one persistent kernel on `s` (tmap: the text's tensor map, or NULL)
int launch_kernel(const void *k, int threads, size_t smem, uint32_t ctas, int max_ctas, cudaStream_t s,
                  const sfa_dev::Tables &tab, const sfa_dev::TextDesc &desc, const CUtensorMap *tmap,
                  const CUtensorMap *tmap_b, const sfa_dev::Tables *tabs,
                  const sfa_dev::TextDesc *descs, const uint32_t *tile_text, const sfa_dev::Scratch &S,
                  sfa_result *out);
// Copy-in of host texts by one kernel (gather.cu): text i of a batch is
// copied from src (a device address of host memory) to dst, len bytes.
constexpr uint64_t GATHER_UNIT = 64 << 10;   // bytes per unit of work of the copy kernel
struct GatherDesc {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t len;
};
// d_unit0[i] = first unit of text i, d_unit0[k] = all units (device arrays)
int launch_gather(const GatherDesc *d_descs, const uint32_t *d_unit0, uint32_t k, uint32_t units, cudaStream_t s);
// The device address of host memory the device can read (pinned and mapped
// into the device's address space), or NULL.
// cache: the last allocation found readable, for a run of texts whose host
// memory the caller keeps allocated meanwhile (one call's texts): a range
// kept longer could have been freed and reused since
struct ReadableRange {
    uintptr_t lo = 0, hi = 0;
    uintptr_t delta = 0;   // device address - host address (mod 2^64)
};
const uint8_t *device_readable(const uint8_t *h, ReadableRange *cache = nullptr);

// kernels_small.cu: the short-text kernel (one CTA or a cluster of up to 16,
// no scratch, no look-back); texts of up to 1 MiB
bool small_fits(uint64_t n);
// n_nc: the handle's stored non-constant rows (staged in shared memory when
// they fit)
int launch_small(const sfa_dev::Tables &T, uint64_t n_nc, const uint8_t *text, uint64_t n, bool carry,
                 sfa_result *out, cudaStream_t s);

// regex.cpp
int regex_to_dfa(const char *pattern, size_t len, uint32_t flags, int32_t cap, std::vector<int32_t> &delta,
                 std::vector<uint8_t> &accept, sfa_regex_info *info, size_t *err_pos);
int regex_nsfa_states(const char *pattern, size_t len, uint32_t flags, uint64_t cap, uint64_t *n_states);

// one text (sfa_match_ex / sfa_match_continue)
int match_impl(sfa_handle *h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
               const sfa_launch_opts *o, bool carry, int32_t *d_map = nullptr);

}  // namespace sfa_impl
