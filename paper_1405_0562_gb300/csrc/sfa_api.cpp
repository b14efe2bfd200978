// C ABI of the matcher (declared in include/sfa.h): handles, device tables,
// scratch, launch shapes, the streaming host path, batch plans and graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "host_compile.h"
#include "launch.h"
#include "sfa.h"

using sfa_dev::Scratch;
using sfa_dev::Tables;
using sfa_dev::TextDesc;

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr uint32_t DEFAULT_TIMEOUT_US = 2000000;   // 2 s per device-side wait
constexpr uint64_t MAX_TEXT = 1ull << 40;
constexpr uint64_t MAX_CHUNK = 1ull << 31;         // per-chunk counters are 32-bit
constexpr uint32_t MAX_FORCED = 1u << 20;
constexpr uint64_t HOST_PIECE = 64ull << 20;       // sfa_match_host copy granularity

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return SFA_OK;
    if (e == cudaErrorMemoryAllocation) return SFA_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SFA_ERR_NO_DEVICE;
    return SFA_ERR_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_err(e_); \
    } while (0)

struct DeviceProps {
    int sms = 0;
    size_t smem_optin = 0;
};

DeviceProps device_props(int dev) {
    static std::mutex mu;
    static std::map<int, DeviceProps> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceProps p;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) p.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) p.smem_optin = v;
    cache[dev] = p;
    return p;
}

// resident CTAs per SM for a kernel instance and shared-memory size
int blocks_per_sm(const void *k, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(k, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)device_props(dev).smem_optin);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, threads, smem) != cudaSuccess) b = 0;
    cache[key] = b;
    return b;
}

struct Shape {
    int threads = 256;
    int chains = 2;
    int simnq = 0;
    uint64_t chunk = 1024;
    uint32_t forced = 0;
    int max_ctas = 0;
    uint32_t timeout_us = DEFAULT_TIMEOUT_US;
    uint32_t debug = 0;
};

int simnq_for(uint32_t nr) { return nr <= 16 ? 16 : (nr <= 32 ? 32 : 64); }

}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct sfa_handle {
    sfa_impl::HostTables host;
    bool on_device = false;
    int device = -1;
    uint8_t *d_tables = nullptr;
    size_t table_bytes = 0;
    Tables dev{};
    uint8_t *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // sfa_match_host
    uint8_t *d_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    sfa_result *d_res = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
};

namespace {

int upload_tables(sfa_handle *h) {
    const auto &H = h->host;
    const size_t nr = (size_t)H.nr;
    size_t off_dfa = 0;
    size_t off_cls = align_up(off_dfa + nr * 256, 256);
    size_t off_nc = align_up(off_cls + 256, 256);
    size_t off_maps = align_up(off_nc + H.nc.size() * 4, 256);
    size_t off_orig = align_up(off_maps + H.maps.size(), 256);
    size_t off_kept = align_up(off_orig + nr * 4, 256);
    size_t total = align_up(off_kept + (size_t)H.nq_in * 4, 256);
    std::vector<uint8_t> img(total, 0);
    std::memcpy(img.data() + off_dfa, H.dfa.data(), H.dfa.size());
    std::memcpy(img.data() + off_cls, H.cls, 256);
    if (!H.nc.empty()) std::memcpy(img.data() + off_nc, H.nc.data(), H.nc.size() * 4);
    if (!H.maps.empty()) std::memcpy(img.data() + off_maps, H.maps.data(), H.maps.size());
    std::memcpy(img.data() + off_orig, H.orig_of.data(), nr * 4);
    std::memcpy(img.data() + off_kept, H.kept_of.data(), (size_t)H.nq_in * 4);
    CK(cudaMalloc(&h->d_tables, total));
    cudaError_t e = cudaMemcpy(h->d_tables, img.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(h->d_tables);
        h->d_tables = nullptr;
        return cuda_err(e);
    }
    h->table_bytes = total;
    Tables &T = h->dev;
    T.dfa = h->d_tables + off_dfa;
    T.cls = h->d_tables + off_cls;
    T.nc = reinterpret_cast<const uint32_t *>(h->d_tables + off_nc);
    T.maps = h->d_tables + off_maps;
    T.orig_of = reinterpret_cast<const int32_t *>(h->d_tables + off_orig);
    T.kept_of = reinterpret_cast<const int32_t *>(h->d_tables + off_kept);
    T.nr = H.nr;
    T.ncls = H.ncls;
    T.first_accept = H.first_accept;
    T.q0 = H.q0;
    T.ident = H.ident;
    T.nq_in = H.nq_in;
    T.mode = H.mode;
    return SFA_OK;
}

// scratch layout of a launch over `ntext` texts and `tiles` tiles
struct ScratchPlan {
    size_t off_texts, off_status, off_agg, off_vec, total, zero;
};

ScratchPlan plan_scratch(uint32_t ntext, uint64_t tiles, uint32_t nr_max, uint64_t vec_bytes) {
    ScratchPlan p;
    p.off_texts = sizeof(sfa_dev::LaunchHeader);
    p.off_status = p.off_texts + (size_t)ntext * sizeof(sfa_dev::TextState);
    p.zero = p.off_status + tiles * 8;
    p.off_agg = align_up(p.zero, 256);
    p.off_vec = align_up(p.off_agg + tiles * nr_max, 256);
    p.total = align_up(p.off_vec + vec_bytes, 256);
    return p;
}

Scratch make_scratch(uint8_t *base, const ScratchPlan &p, uint32_t nr_max, uint32_t tiles, const Shape &sh) {
    Scratch S;
    S.hdr = reinterpret_cast<sfa_dev::LaunchHeader *>(base);
    S.texts = reinterpret_cast<sfa_dev::TextState *>(base + p.off_texts);
    S.status = reinterpret_cast<uint64_t *>(base + p.off_status);
    S.agg = base + p.off_agg;
    S.chainvec = base + p.off_vec;
    S.nr_max = nr_max;
    S.timeout_us = sh.timeout_us;
    S.debug = sh.debug;
    S.total_tiles = tiles;
    return S;
}

// launch shape for one text
int choose_shape(const sfa_handle *h, uint64_t n, const sfa_launch_opts *o, Shape &sh) {
    const bool sim = h->host.mode == SFA_MODE_SIM;
    sh = Shape();
    sh.simnq = sim ? simnq_for(h->host.nr) : 0;
    sh.threads = sim ? 128 : 256;
    sh.chains = sim ? 1 : 2;
    if (o) {
        if (o->block_threads) sh.threads = (int)o->block_threads;
        if (o->chains) sh.chains = (int)o->chains;
        if (o->timeout_us) sh.timeout_us = o->timeout_us;
        sh.debug = o->debug_flags;
        sh.max_ctas = (int)o->max_ctas;
    }
    if (!sfa_impl::kernel_for(sh.threads, sh.chains, sh.simnq, false)) return SFA_ERR_UNSUPPORTED;
    const uint64_t cpt = (uint64_t)sh.threads * sh.chains;
    if (o && o->forced_chunks) {
        if (o->forced_chunks > MAX_FORCED) return SFA_ERR_INVALID;
        sh.forced = o->forced_chunks;
        if (n / sh.forced + 1 > MAX_CHUNK) return SFA_ERR_INVALID;
        return SFA_OK;
    }
    if (o && o->chunk_bytes) {
        sh.chunk = o->chunk_bytes;
        if (sh.chunk > MAX_CHUNK) return SFA_ERR_INVALID;
        return SFA_OK;
    }
    // automatic: about six tiles per resident CTA, chunks of 256 B .. 4 KiB
    // (simulation: 4 KiB .. 64 KiB, the vector phase needs long chunks)
    const size_t smem = sfa_impl::smem_bytes(sh.threads, sh.chains, h->host.nr);
    const int bps = blocks_per_sm(sfa_impl::kernel_for(sh.threads, sh.chains, sh.simnq, false), sh.threads, smem);
    const uint64_t ctas = (uint64_t)std::max(1, bps) * std::max(1, device_props(h->device).sms);
    uint64_t want = n / (ctas * 6 * cpt);
    const uint64_t lo = sim ? 4096 : 256, hi = sim ? 65536 : 4096;
    want = std::min(hi, std::max(lo, align_up(want, 16)));
    sh.chunk = want;
    return SFA_OK;
}

int ensure_scratch(sfa_handle *h, size_t bytes) {
    if (bytes <= h->scratch_bytes) return SFA_OK;
    if (h->d_scratch) {
        // the previous scratch may still be in use by enqueued work
        CK(cudaDeviceSynchronize());
        cudaFree(h->d_scratch);
        h->d_scratch = nullptr;
        h->scratch_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    CK(cudaMalloc(&h->d_scratch, want));
    h->scratch_bytes = want;
    return SFA_OK;
}

int launch_kernel(const void *k, int threads, size_t smem, uint32_t tiles, int max_ctas, cudaStream_t s,
                  const Tables &tab, const TextDesc &desc, const Tables *tabs, const TextDesc *descs,
                  const uint32_t *tile_text, const Scratch &S, sfa_result *out) {
    const int bps = blocks_per_sm(k, threads, smem);
    if (bps < 1) return SFA_ERR_UNSUPPORTED;
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t grid = (uint64_t)bps * device_props(dev).sms;
    if (max_ctas > 0) grid = std::min<uint64_t>(grid, (uint64_t)max_ctas);
    grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, tiles));
    Tables a0 = tab;
    TextDesc a1 = desc;
    const Tables *a2 = tabs;
    const TextDesc *a3 = descs;
    const uint32_t *a4 = tile_text;
    Scratch a5 = S;
    sfa_result *a6 = out;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
    CK(cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, smem, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

int match_impl(sfa_handle *h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
               const sfa_launch_opts *o, bool carry) {
    if (!h || !d_out) return SFA_ERR_INVALID;
    if (!h->on_device) return SFA_ERR_HOST_ONLY;
    if (n > MAX_TEXT || (n > 0 && !d_text)) return SFA_ERR_INVALID;
    Shape sh;
    int rc = choose_shape(h, n, o, sh);
    if (rc) return rc;
    TextDesc d{};
    d.text = d_text;
    d.n = n;
    d.chunk = sh.chunk;
    d.forced = sh.forced;
    d.tile_base = 0;
    d.table = 0;
    d.out_index = 0;
    d.carry = carry ? 1u : 0u;
    const uint64_t cpt = (uint64_t)sh.threads * sh.chains;
    // chunk indices (and, in simulation mode, the ids nr + chunk) stay below 2^31
    if (sfa_dev::num_chunks(d) >= (1ull << 31) - 256) return SFA_ERR_INVALID;
    const uint64_t tiles = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
    d.ntiles = (uint32_t)tiles;
    const uint32_t nr = h->host.nr;
    const uint64_t vec = sh.simnq ? tiles * cpt * nr : 0;
    ScratchPlan p = plan_scratch(1, tiles, nr, vec);
    rc = ensure_scratch(h, p.total);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->d_scratch, 0, p.zero, s));
    Scratch S = make_scratch(h->d_scratch, p, nr, (uint32_t)tiles, sh);
    const void *k = sfa_impl::kernel_for(sh.threads, sh.chains, sh.simnq, false);
    const size_t smem = sfa_impl::smem_bytes(sh.threads, sh.chains, nr);
    return launch_kernel(k, sh.threads, smem, (uint32_t)tiles, sh.max_ctas, s, h->dev, d, nullptr, nullptr,
                         nullptr, S, d_out);
}

void free_handle_device(sfa_handle *h) {
    if (h->d_tables) cudaFree(h->d_tables);
    if (h->d_scratch) cudaFree(h->d_scratch);
    for (int i = 0; i < 2; ++i) {
        if (h->d_stage[i]) cudaFree(h->d_stage[i]);
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    }
    if (h->d_res) cudaFree(h->d_res);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
}

}  // namespace

extern "C" {

int sfa_compile(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                const sfa_compile_opts *opts, sfa_handle_t *out) {
    if (!out) return SFA_ERR_INVALID;
    *out = nullptr;
    sfa_compile_opts o{};
    if (opts) o = *opts;
    sfa_handle *h = new (std::nothrow) sfa_handle();
    if (!h) return SFA_ERR_OOM;
    int rc;
    try {
        rc = sfa_impl::build_tables(delta, nq, q0, accept, o.cap_states, o.force_mode, h->host);
    } catch (const std::bad_alloc &) {
        rc = SFA_ERR_OOM;
    }
    if (rc) {
        delete h;
        return rc;
    }
    if (!(o.flags & SFA_COMPILE_HOST_ONLY)) {
        int count = 0;
        cudaError_t e = cudaGetDeviceCount(&count);
        if (e != cudaSuccess || count == 0) {
            delete h;
            return SFA_ERR_NO_DEVICE;
        }
        cudaGetDevice(&h->device);
        rc = upload_tables(h);
        if (rc) {
            free_handle_device(h);
            delete h;
            return rc;
        }
        h->on_device = true;
    }
    *out = h;
    return SFA_OK;
}

void sfa_destroy(sfa_handle_t h) {
    if (!h) return;
    if (h->on_device) free_handle_device(h);
    delete h;
}

int sfa_info(sfa_handle_t h, sfa_info_t *out) {
    if (!h || !out) return SFA_ERR_INVALID;
    const auto &H = h->host;
    std::memset(out, 0, sizeof *out);
    out->mode = (uint32_t)H.mode;
    out->nq = (uint32_t)H.nq_in;
    out->n_reachable = (uint32_t)H.nr;
    out->n_accepting = (uint32_t)(H.nr - H.first_accept);
    out->ncls = (uint32_t)H.ncls;
    out->on_device = h->on_device ? 1u : 0u;
    out->n_nonconst = H.mode == SFA_MODE_SFA ? (H.nr > 1 ? H.n_nc : 0) : 0;
    out->n_sfa_states = H.mode == SFA_MODE_SFA ? out->n_nonconst + H.n_const : 0;
    out->table_bytes = h->table_bytes;
    out->compile_seconds = H.seconds;
    return SFA_OK;
}

int sfa_export(sfa_handle_t h, int32_t which, void *dst, size_t bytes, size_t *size_out) {
    if (!h) return SFA_ERR_INVALID;
    const auto &H = h->host;
    const void *src = nullptr;
    size_t sz = 0;
    switch (which) {
        case SFA_TABLE_CLASS: src = H.cls; sz = 256; break;
        case SFA_TABLE_DFA: src = H.dfa.data(); sz = H.dfa.size(); break;
        case SFA_TABLE_NC: src = H.nc.data(); sz = H.nc.size() * 4; break;
        case SFA_TABLE_MAPS: src = H.maps.data(); sz = H.maps.size(); break;
        case SFA_TABLE_ORIG: src = H.orig_of.data(); sz = H.orig_of.size() * 4; break;
        default: return SFA_ERR_INVALID;
    }
    if (size_out) *size_out = sz;
    if (dst && sz) std::memcpy(dst, src, std::min(bytes, sz));
    return SFA_OK;
}

const char *sfa_strerror(int code) {
    switch (code) {
        case SFA_OK: return "success";
        case SFA_ERR_INVALID: return "invalid argument";
        case SFA_ERR_UNSUPPORTED: return "outside the limits of this build";
        case SFA_ERR_OOM: return "out of memory";
        case SFA_ERR_CUDA: return "CUDA runtime error";
        case SFA_ERR_TIMEOUT: return "a device-side bounded wait gave up";
        case SFA_ERR_NO_DEVICE: return "no usable CUDA device";
        case SFA_ERR_HOST_ONLY: return "handle has no device tables (compiled host-only)";
        case SFA_ERR_SCRATCH_LIMIT: return "text needs more scratch than the fixed no-allocation buffer holds";
        default: return "unknown error code";
    }
}

int sfa_match(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, sfa_stream_t stream) {
    return match_impl(h, d_text, n, d_out, (cudaStream_t)stream, nullptr, false);
}

int sfa_match_ex(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, sfa_stream_t stream,
                 const sfa_launch_opts *opts) {
    return match_impl(h, d_text, n, d_out, (cudaStream_t)stream, opts, false);
}

int sfa_match_continue(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_inout,
                       sfa_stream_t stream, const sfa_launch_opts *opts) {
    return match_impl(h, d_text, n, d_inout, (cudaStream_t)stream, opts, true);
}

int sfa_match_host(sfa_handle_t h, const uint8_t *h_text, uint64_t n, sfa_result *h_out, sfa_stream_t stream,
                   const sfa_launch_opts *opts) {
    if (!h || !h_out || (n > 0 && !h_text)) return SFA_ERR_INVALID;
    if (!h->on_device) return SFA_ERR_HOST_ONLY;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t piece = std::min<uint64_t>(HOST_PIECE, std::max<uint64_t>(n, 16));
    if (!h->copy_stream) {
        CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming));
        }
        CK(cudaMalloc(&h->d_res, sizeof(sfa_result)));
    }
    if (h->stage_bytes < piece) {
        CK(cudaDeviceSynchronize());
        for (int i = 0; i < 2; ++i) {
            if (h->d_stage[i]) cudaFree(h->d_stage[i]);
            h->d_stage[i] = nullptr;
        }
        h->stage_bytes = 0;
        for (int i = 0; i < 2; ++i) CK(cudaMalloc(&h->d_stage[i], piece));
        h->stage_bytes = piece;
    }
    int rc = SFA_OK;
    if (n == 0) {
        rc = match_impl(h, nullptr, 0, h->d_res, s, opts, false);
        if (rc) return rc;
    }
    // the copy stream may reuse a staging buffer only after the match that
    // read it; the match of piece i waits for its copy
    CK(cudaEventRecord(h->ev_done[0], s));
    CK(cudaEventRecord(h->ev_done[1], s));
    uint64_t i = 0;
    for (uint64_t off = 0; off < n; off += piece, ++i) {
        const uint64_t len = std::min(piece, n - off);
        const int b = (int)(i & 1);
        CK(cudaStreamWaitEvent(h->copy_stream, h->ev_done[b], 0));
        CK(cudaMemcpyAsync(h->d_stage[b], h_text + off, len, cudaMemcpyHostToDevice, h->copy_stream));
        CK(cudaEventRecord(h->ev_copied[b], h->copy_stream));
        CK(cudaStreamWaitEvent(s, h->ev_copied[b], 0));
        rc = match_impl(h, h->d_stage[b], len, h->d_res, s, opts, off > 0);
        if (rc) return rc;
        CK(cudaEventRecord(h->ev_done[b], s));
    }
    CK(cudaMemcpyAsync(h_out, h->d_res, sizeof(sfa_result), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SFA_OK;
}

uint64_t sfa_kernel_launch_count(void) { return g_launches.load(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct sfa_batch {
    int device = -1;
    int32_t k = 0;
    Shape shape;
    uint8_t *d_mem = nullptr;           // tables array, descriptors, tile map
    uint8_t *d_scratch = nullptr;
    ScratchPlan plan{};
    Scratch S{};
    const Tables *d_tabs = nullptr;
    const TextDesc *d_descs = nullptr;
    const uint32_t *d_tile_text = nullptr;
    uint32_t total_tiles = 0;
    uint32_t nr_max = 0;
    size_t smem = 0;
    const void *kernel = nullptr;
    // texts whose handle is in simulation mode: matched one by one
    std::vector<int32_t> sim_index;
    std::vector<sfa_handle_t> sim_handle;
    std::vector<const uint8_t *> sim_text;
    std::vector<uint64_t> sim_len;
    // CUDA graph of the launch, keyed by the output pointer
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    sfa_result *exec_out = nullptr;
};

namespace {

int batch_enqueue(sfa_batch *b, sfa_result *d_out, cudaStream_t s) {
    if (b->total_tiles > 0) {
        CK(cudaMemsetAsync(b->d_scratch, 0, b->plan.zero, s));
        int rc = launch_kernel(b->kernel, b->shape.threads, b->smem, b->total_tiles, b->shape.max_ctas, s, Tables{},
                               TextDesc{}, b->d_tabs, b->d_descs, b->d_tile_text, b->S, d_out);
        if (rc) return rc;
    }
    for (size_t i = 0; i < b->sim_index.size(); ++i) {
        int rc = match_impl(b->sim_handle[i], b->sim_text[i], b->sim_len[i], d_out + b->sim_index[i], s, nullptr,
                            false);
        if (rc) return rc;
    }
    return SFA_OK;
}

void batch_free(sfa_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->d_scratch) cudaFree(b->d_scratch);
}

}  // namespace

extern "C" {

int sfa_batch_create(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens, int32_t k,
                     const sfa_launch_opts *opts, sfa_batch_t *out) {
    if (!out || k < 0 || (k > 0 && (!hs || !d_texts || !lens))) return SFA_ERR_INVALID;
    *out = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    sfa_batch *b = new (std::nothrow) sfa_batch();
    if (!b) return SFA_ERR_OOM;
    b->device = dev;
    b->k = k;
    Shape &sh = b->shape;
    sh.threads = 256;
    sh.chains = 2;
    if (opts) {
        if (opts->block_threads) sh.threads = (int)opts->block_threads;
        if (opts->chains) sh.chains = (int)opts->chains;
        if (opts->timeout_us) sh.timeout_us = opts->timeout_us;
        sh.debug = opts->debug_flags;
        sh.max_ctas = (int)opts->max_ctas;
    }
    b->kernel = sfa_impl::kernel_for(sh.threads, sh.chains, 0, true);
    if (!b->kernel) {
        delete b;
        return SFA_ERR_UNSUPPORTED;
    }
    const uint64_t cpt = (uint64_t)sh.threads * sh.chains;
    // texts in SFA mode, grouped by automaton (stable in text order)
    std::vector<int32_t> order;
    std::vector<sfa_handle_t> distinct;
    std::map<sfa_handle_t, uint32_t> tab_of;
    uint64_t total_bytes = 0;
    for (int32_t i = 0; i < k; ++i) {
        sfa_handle_t h = hs[i];
        if (!h || !h->on_device || h->device != dev || lens[i] > MAX_TEXT || (lens[i] && !d_texts[i])) {
            delete b;
            return h && !h->on_device ? SFA_ERR_HOST_ONLY : SFA_ERR_INVALID;
        }
        if (h->host.mode == SFA_MODE_SIM) {
            b->sim_index.push_back(i);
            b->sim_handle.push_back(h);
            b->sim_text.push_back(d_texts[i]);
            b->sim_len.push_back(lens[i]);
            continue;
        }
        if (!tab_of.count(h)) {
            tab_of[h] = (uint32_t)distinct.size();
            distinct.push_back(h);
            b->nr_max = std::max<uint32_t>(b->nr_max, (uint32_t)h->host.nr);
        }
        order.push_back(i);
        total_bytes += lens[i];
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return tab_of[hs[x]] < tab_of[hs[y]]; });
    b->smem = sfa_impl::smem_bytes(sh.threads, sh.chains, std::max<uint32_t>(b->nr_max, 1));
    // chunk length: as for one text of the batch's total size, shortened
    // for texts that would not fill a tile
    uint64_t chunk = opts && opts->chunk_bytes ? opts->chunk_bytes : 0;
    const int bps = blocks_per_sm(b->kernel, sh.threads, b->smem);   // also caches it before any capture
    if (!chunk) {
        const uint64_t ctas = (uint64_t)std::max(1, bps) * std::max(1, device_props(dev).sms);
        chunk = std::min<uint64_t>(4096, std::max<uint64_t>(256, align_up(total_bytes / (ctas * 6 * cpt), 16)));
    }
    if (chunk > MAX_CHUNK) {
        delete b;
        return SFA_ERR_INVALID;
    }
    std::vector<TextDesc> descs;
    std::vector<uint32_t> tile_text;
    for (int32_t i : order) {
        TextDesc d{};
        d.text = d_texts[i];
        d.n = lens[i];
        uint64_t want = align_up((d.n + cpt - 1) / cpt, 16);
        d.chunk = std::min<uint64_t>(chunk, std::max<uint64_t>(64, want));
        d.forced = 0;
        const uint64_t t = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
        d.ntiles = (uint32_t)t;
        d.tile_base = (uint32_t)tile_text.size();
        d.table = tab_of[hs[i]];
        d.out_index = (uint32_t)i;
        d.carry = 0;
        if (sfa_dev::num_chunks(d) >= (1ull << 31) || tile_text.size() + t >= (1ull << 30)) {
            delete b;
            return SFA_ERR_INVALID;
        }
        for (uint64_t j = 0; j < t; ++j) tile_text.push_back((uint32_t)descs.size());
        descs.push_back(d);
    }
    b->total_tiles = (uint32_t)tile_text.size();
    std::vector<Tables> tabs;
    for (auto h : distinct) tabs.push_back(h->dev);
    const size_t off_tabs = 0;
    const size_t off_descs = align_up(off_tabs + tabs.size() * sizeof(Tables), 256);
    const size_t off_tt = align_up(off_descs + descs.size() * sizeof(TextDesc), 256);
    const size_t mem = align_up(off_tt + tile_text.size() * 4, 256) + 256;
    std::vector<uint8_t> img(mem, 0);
    if (!tabs.empty()) std::memcpy(img.data() + off_tabs, tabs.data(), tabs.size() * sizeof(Tables));
    if (!descs.empty()) std::memcpy(img.data() + off_descs, descs.data(), descs.size() * sizeof(TextDesc));
    if (!tile_text.empty()) std::memcpy(img.data() + off_tt, tile_text.data(), tile_text.size() * 4);
    cudaError_t e = cudaMalloc(&b->d_mem, mem);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_mem, img.data(), mem, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        b->plan = plan_scratch((uint32_t)std::max<size_t>(descs.size(), 1), b->total_tiles, std::max<uint32_t>(b->nr_max, 1), 0);
        e = cudaMalloc(&b->d_scratch, b->plan.total);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return cuda_err(e);
    }
    b->d_tabs = reinterpret_cast<const Tables *>(b->d_mem + off_tabs);
    b->d_descs = reinterpret_cast<const TextDesc *>(b->d_mem + off_descs);
    b->d_tile_text = reinterpret_cast<const uint32_t *>(b->d_mem + off_tt);
    b->S = make_scratch(b->d_scratch, b->plan, std::max<uint32_t>(b->nr_max, 1), b->total_tiles, sh);
    // simulation-mode texts: size their handles' scratch now, so that
    // launches (and graph captures) of the plan never allocate
    for (size_t i = 0; i < b->sim_index.size(); ++i) {
        Shape ss;
        int rc = choose_shape(b->sim_handle[i], b->sim_len[i], nullptr, ss);
        if (!rc) {
            TextDesc d{};
            d.n = b->sim_len[i];
            d.chunk = ss.chunk;
            const uint64_t c2 = (uint64_t)ss.threads * ss.chains;
            const uint64_t t = (sfa_dev::num_chunks(d) + c2 - 1) / c2;
            rc = ensure_scratch(b->sim_handle[i], plan_scratch(1, t, b->sim_handle[i]->host.nr,
                                                               t * c2 * b->sim_handle[i]->host.nr).total);
        }
        if (rc) {
            batch_free(b);
            delete b;
            return rc;
        }
    }
    *out = b;
    return SFA_OK;
}

int sfa_batch_launch(sfa_batch_t b, sfa_result *d_out, sfa_stream_t stream) {
    if (!b || (b->k > 0 && !d_out)) return SFA_ERR_INVALID;
    return batch_enqueue(b, d_out, (cudaStream_t)stream);
}

int sfa_batch_graph_launch(sfa_batch_t b, sfa_result *d_out, sfa_stream_t stream) {
    if (!b || (b->k > 0 && !d_out)) return SFA_ERR_INVALID;
    if (!b->exec || b->exec_out != d_out) {
        if (b->exec) {
            CK(cudaStreamSynchronize((cudaStream_t)stream));
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = g_launches.load();
        int rc = batch_enqueue(b, d_out, b->cap_stream);
        g_launches.store(before);   // captured, not launched
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_err(e);
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e);
        b->exec_out = d_out;
    }
    CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    g_launches.fetch_add((b->total_tiles > 0 ? 1 : 0) + b->sim_index.size(), std::memory_order_relaxed);
    return SFA_OK;
}

void sfa_batch_destroy(sfa_batch_t b) {
    if (!b) return;
    batch_free(b);
    delete b;
}

int sfa_match_batch(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens, int32_t k,
                    sfa_result *d_out, sfa_stream_t stream) {
    sfa_batch_t b = nullptr;
    int rc = sfa_batch_create(hs, d_texts, lens, k, nullptr, &b);
    if (rc) return rc;
    rc = sfa_batch_launch(b, d_out, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    sfa_batch_destroy(b);
    if (rc) return rc;
    return cuda_err(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// matching on a fixed, caller-provided scratch buffer (sfa_match_noalloc)
// ---------------------------------------------------------------------------
namespace sfa_impl {

int match_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
                       uint8_t *scratch, size_t cap, int scratch_device) {
    if (!h || !d_out || !scratch) return SFA_ERR_INVALID;
    if (n > MAX_TEXT || (n > 0 && !d_text)) return SFA_ERR_INVALID;
    if (!h->on_device) return SFA_ERR_HOST_ONLY;
    if (h->host.mode != SFA_MODE_SFA) return SFA_ERR_UNSUPPORTED;
    if (h->device != scratch_device) return SFA_ERR_INVALID;
    Shape sh;
    int rc = choose_shape(h, n, nullptr, sh);
    if (rc) return rc;
    TextDesc d{};
    d.text = d_text;
    d.n = n;
    d.chunk = sh.chunk;
    d.forced = 0;
    const uint64_t cpt = (uint64_t)sh.threads * sh.chains;
    if (sfa_dev::num_chunks(d) >= (1ull << 31) - 256) return SFA_ERR_SCRATCH_LIMIT;
    const uint64_t tiles = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
    d.ntiles = (uint32_t)tiles;
    const uint32_t nr = h->host.nr;
    const ScratchPlan p = plan_scratch(1, tiles, nr, 0);
    if (p.total > cap) return SFA_ERR_SCRATCH_LIMIT;
    // the buffer keeps the previous call's contents: clear the header, the
    // text record and the look-back descriptors
    CK(cudaMemsetAsync(scratch, 0, p.zero, s));
    const Scratch S = make_scratch(scratch, p, nr, (uint32_t)tiles, sh);
    const void *k = kernel_for(sh.threads, sh.chains, 0, false);
    const size_t smem = smem_bytes(sh.threads, sh.chains, nr);
    return launch_kernel(k, sh.threads, smem, (uint32_t)tiles, 0, s, h->dev, d, nullptr, nullptr, nullptr, S,
                         d_out);
}

}  // namespace sfa_impl
