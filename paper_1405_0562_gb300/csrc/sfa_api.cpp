// C ABI of the matcher for single texts (declared in include/sfa.h):
// handles, device tables, scratch, launch shapes, the streaming host path.
// Batches are in batch_api.cpp, the no-allocation entry point in noalloc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "api_internal.h"

using sfa_dev::Scratch;
using sfa_dev::Tables;
using sfa_dev::TextDesc;

namespace sfa_impl {

std::atomic<uint64_t> g_launches{0};

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


// The device's point-mapping encoding of the non-constant rows (see
// sfa_types.h): with an absorbing non-final state z (the sink), every entry
// whose target maps all states but one, s, to z carries s and the image p
// of s instead of the target's id, and pid[s*nr + p] gives the id back; an
// entry whose target maps a set S of two or more states to one p and the
// rest to z carries NC_SET, the id of S and p (set-point mapping), with
// spid[sid*nr + p] the id and setbits the sets (at most 255 of them; past
// that the targets keep their ids).  Returns the sink, or NO_SINK (no such
// state, simulation mode, or 256 kept states, where a byte-wide "no point"
// marker would be a state).
uint32_t point_encoding(const HostTables &H, std::vector<uint32_t> &nc, std::vector<uint32_t> &pid,
                        std::vector<uint32_t> &setbits, std::vector<uint32_t> &spid) {
    nc = H.nc;
    pid.clear();
    setbits.clear();
    spid.clear();
    const int nr = H.nr;
    if (H.mode != SFA_MODE_SFA || nr < 2 || nr > 255 || H.n_nc == 0) return sfa_dev::NO_SINK;
    int z = -1;
    for (int q = 0; q < H.first_accept && z < 0; ++q) {
        bool absorbing = true;
        for (int b = 0; b < 256 && absorbing; ++b) absorbing = H.dfa[(size_t)q * 256 + b] == q;
        if (absorbing) z = q;
    }
    if (z < 0) return sfa_dev::NO_SINK;
    const uint32_t words = ((uint32_t)nr + 31) / 32;
    std::vector<int32_t> src(H.n_nc, -1), img(H.n_nc, 0), set_of(H.n_nc, -1);
    std::map<std::vector<uint32_t>, int32_t> set_id;
    bool any = false;
    for (uint64_t i = 0; i < H.n_nc; ++i) {
        const uint8_t *f = H.maps.data() + i * nr;
        int live = 0, s = -1, p = -1;
        bool one_image = true;
        std::vector<uint32_t> bits(words, 0);
        for (int q = 0; q < nr; ++q)
            if (f[q] != z) {
                ++live;
                s = q;
                one_image &= p < 0 || f[q] == p;
                p = f[q];
                bits[q >> 5] |= 1u << (q & 31);
            }
        if (live == 1) {
            src[i] = s;
            img[i] = f[s];
            any = true;
        } else if (live >= 2 && one_image) {
            auto it = set_id.find(bits);
            if (it == set_id.end()) {
                if (set_id.size() >= 255) continue;
                it = set_id.emplace(bits, (int32_t)set_id.size()).first;
            }
            set_of[i] = it->second;
            img[i] = p;
            any = true;
        }
    }
    if (!any) return sfa_dev::NO_SINK;
    pid.assign((size_t)nr * nr, 0);
    spid.assign(set_id.size() * (size_t)nr, 0);
    setbits.assign(set_id.size() * words, 0);
    for (const auto &kv : set_id) std::copy(kv.first.begin(), kv.first.end(), setbits.begin() + (size_t)kv.second * words);
    for (uint64_t i = 0; i < H.n_nc; ++i) {
        if (src[i] >= 0) pid[(size_t)src[i] * nr + img[i]] = (uint32_t)(nr + i);
        if (set_of[i] >= 0) spid[(size_t)set_of[i] * nr + img[i]] = (uint32_t)(nr + i);
    }
    for (uint32_t &e : nc) {
        const uint32_t id = e & sfa_dev::NC_ID_MASK;
        if (id < (uint32_t)nr) continue;
        const uint64_t k = id - nr;
        if (src[k] >= 0)
            e = (e & ~sfa_dev::NC_ID_MASK) | sfa_dev::NC_POINT | (uint32_t)src[k] << 8 | (uint32_t)img[k];
        else if (set_of[k] >= 0)
            e = (e & ~sfa_dev::NC_ID_MASK) | sfa_dev::NC_POINT | sfa_dev::NC_SET | (uint32_t)set_of[k] << 8 |
                (uint32_t)img[k];
    }
    return (uint32_t)z;
}

// Device tables of a handle with more than 256 kept states: the class table,
// the class-indexed 16-bit DFA, the non-constant rows (point entries already
// encoded by the construction), the stored mappings and the id maps.
int upload_tables_wide(sfa_handle *h) {
    const auto &H = h->host;
    const size_t nr = (size_t)H.nr;
    size_t off_cdfa = 0;
    size_t off_cls = align_up(off_cdfa + H.cdfa.size() * 2, 256);
    size_t off_nc = align_up(off_cls + 256, 256);
    size_t off_maps = align_up(off_nc + H.nc.size() * 4, 256);
    size_t off_orig = align_up(off_maps + H.maps16.size() * 2, 256);
    size_t off_kept = align_up(off_orig + nr * 4, 256);
    size_t off_sets = align_up(off_kept + (size_t)H.nq_in * 4, 256);
    size_t total = align_up(off_sets + H.setbits.size() * 4, 256);
    std::vector<uint8_t> img(total, 0);
    std::memcpy(img.data() + off_cdfa, H.cdfa.data(), H.cdfa.size() * 2);
    std::memcpy(img.data() + off_cls, H.cls, 256);
    if (!H.nc.empty()) std::memcpy(img.data() + off_nc, H.nc.data(), H.nc.size() * 4);
    if (!H.maps16.empty()) std::memcpy(img.data() + off_maps, H.maps16.data(), H.maps16.size() * 2);
    std::memcpy(img.data() + off_orig, H.orig_of.data(), nr * 4);
    std::memcpy(img.data() + off_kept, H.kept_of.data(), (size_t)H.nq_in * 4);
    if (!H.setbits.empty()) std::memcpy(img.data() + off_sets, H.setbits.data(), H.setbits.size() * 4);
    CK(cudaMalloc(&h->d_tables, total));
    cudaError_t e = cudaMemcpy(h->d_tables, img.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(h->d_tables);
        h->d_tables = nullptr;
        return cuda_err(e);
    }
    h->table_bytes = total;
    Tables &T = h->dev;
    T = Tables{};
    T.setbits = H.setbits.empty() ? nullptr : reinterpret_cast<const uint32_t *>(h->d_tables + off_sets);
    T.set_words = H.set_words;
    T.cdfa = reinterpret_cast<const uint16_t *>(h->d_tables + off_cdfa);
    T.cls = h->d_tables + off_cls;
    T.nc = reinterpret_cast<const uint32_t *>(h->d_tables + off_nc);
    T.maps16 = reinterpret_cast<const uint16_t *>(h->d_tables + off_maps);
    T.orig_of = reinterpret_cast<const int32_t *>(h->d_tables + off_orig);
    T.kept_of = reinterpret_cast<const int32_t *>(h->d_tables + off_kept);
    T.sink = H.sink >= 0 ? (uint32_t)H.sink : sfa_dev::NO_SINK;
    T.nr = H.nr;
    T.ncls = H.ncls;
    T.first_accept = H.first_accept;
    T.q0 = H.q0;
    T.ident = H.ident;
    T.nq_in = H.nq_in;
    T.mode = H.mode;
    return SFA_OK;
}

int upload_tables(sfa_handle *h) {
    const auto &H = h->host;
    if (H.wide) return upload_tables_wide(h);
    const size_t nr = (size_t)H.nr;
    std::vector<uint32_t> nc, pid, setbits, spid;
    const uint32_t sink = point_encoding(H, nc, pid, setbits, spid);
    size_t off_dfa = 0;
    size_t off_cls = align_up(off_dfa + nr * 256, 256);
    size_t off_nc = align_up(off_cls + 256, 256);
    size_t off_maps = align_up(off_nc + nc.size() * 4, 256);
    size_t off_orig = align_up(off_maps + H.maps.size(), 256);
    size_t off_kept = align_up(off_orig + nr * 4, 256);
    size_t off_pid = align_up(off_kept + (size_t)H.nq_in * 4, 256);
    size_t off_sets = align_up(off_pid + pid.size() * 4, 256);
    size_t off_spid = align_up(off_sets + setbits.size() * 4, 256);
    size_t total = align_up(off_spid + spid.size() * 4, 256);
    std::vector<uint8_t> img(total, 0);
    std::memcpy(img.data() + off_dfa, H.dfa.data(), H.dfa.size());
    std::memcpy(img.data() + off_cls, H.cls, 256);
    if (!nc.empty()) std::memcpy(img.data() + off_nc, nc.data(), nc.size() * 4);
    if (!pid.empty()) std::memcpy(img.data() + off_pid, pid.data(), pid.size() * 4);
    if (!setbits.empty()) std::memcpy(img.data() + off_sets, setbits.data(), setbits.size() * 4);
    if (!spid.empty()) std::memcpy(img.data() + off_spid, spid.data(), spid.size() * 4);
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
    T = Tables{};
    T.dfa = h->d_tables + off_dfa;
    T.cls = h->d_tables + off_cls;
    T.nc = reinterpret_cast<const uint32_t *>(h->d_tables + off_nc);
    T.maps = h->d_tables + off_maps;
    T.orig_of = reinterpret_cast<const int32_t *>(h->d_tables + off_orig);
    T.kept_of = reinterpret_cast<const int32_t *>(h->d_tables + off_kept);
    T.pid = pid.empty() ? nullptr : reinterpret_cast<const uint32_t *>(h->d_tables + off_pid);
    T.setbits = setbits.empty() ? nullptr : reinterpret_cast<const uint32_t *>(h->d_tables + off_sets);
    T.spid = spid.empty() ? nullptr : reinterpret_cast<const uint32_t *>(h->d_tables + off_spid);
    T.set_words = ((uint32_t)nr + 31) / 32;
    T.sink = sink;
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
    S.map_mode = 0;
    S.single = 0;
    return S;
}

// the kernel instance and shared memory of a single-text launch shape
const void *shape_kernel(const sfa_handle *h, const Shape &sh) {
    if (h->host.wide) return sh.wt || sh.simnq ? nullptr : kernel_for_wide(sh.threads, sh.chains);
    return kernel_for(sh.threads, sh.chains, sh.simnq, false, sh.wt);
}
size_t shape_smem(const sfa_handle *h, const Shape &sh) {
    if (h->host.wide) return smem_bytes_wide(sh.threads, sh.chains, (uint32_t)h->host.nr, (uint32_t)h->host.ncls);
    return smem_bytes(sh.threads, sh.chains, (uint32_t)h->host.nr, sh.simnq);
}

// launch shape for one text
int choose_shape(const sfa_handle *h, uint64_t n, const sfa_launch_opts *o, Shape &sh) {
    const bool sim = h->host.mode == SFA_MODE_SIM;
    sh = Shape();
    sh.simnq = sim ? simnq_for(h->host.nr) : 0;
    // simulation vectors of 128 and 256 entries live in shared memory, which
    // then allows one or two CTAs per SM: 256 threads keep 8 warps resident
    sh.threads = sim ? (sh.simnq > 64 ? 256 : 128) : 256;
    sh.chains = sim ? 1 : 2;
    if (!sim) {
        // one chunk per thread; 512-thread CTAs when two fit on an SM (one
        // CTA's scan and look-back then overlap the other's lookups), else
        // the largest CTA whose shared memory fits
        sh.chains = 1;
        Shape s512 = sh;
        s512.threads = 512;
        const int b512 = blocks_per_sm(shape_kernel(h, s512), 512, shape_smem(h, s512));
        if (b512 >= 2) {
            sh.threads = 512;
        } else {
            const size_t optin = device_props(h->device).smem_optin;
            sh.threads = 256;
            for (int t : {1024, 512}) {
                Shape st = sh;
                st.threads = t;
                if (optin == 0 || shape_smem(h, st) <= optin) {
                    sh.threads = t;
                    break;
                }
            }
        }
    }
    uint32_t tiling = SFA_TILING_AUTO;
    if (o) {
        if (o->block_threads) sh.threads = (int)o->block_threads;
        if (o->chains) sh.chains = (int)o->chains;
        if (o->timeout_us) sh.timeout_us = o->timeout_us;
        sh.debug = o->debug_flags;
        sh.max_ctas = (int)o->max_ctas;
        tiling = o->tiling;
    }
    if (tiling > SFA_TILING_WARP) return SFA_ERR_INVALID;
    // CTA tiles unless the caller asks for warp tiles (measured slower on the
    // single-text workloads: their look-back and recount do not overlap)
    sh.wt = tiling == SFA_TILING_WARP;
    if (!shape_kernel(h, sh)) return SFA_ERR_UNSUPPORTED;
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
    const size_t smem = shape_smem(h, sh);
    const int bps = blocks_per_sm(shape_kernel(h, sh), sh.threads, smem);
    const uint64_t ctas = (uint64_t)std::max(1, bps) * std::max(1, device_props(h->device).sms);
    sh.auto_chunk = true;
    sh.bps = bps;
    sh.sms = device_props(h->device).sms;
    uint64_t want;
    if (sim) {
        // one tile per resident CTA, chunks of at least 4 KiB: every chunk
        // starts with the vector phase (up to |Q| lookups per byte until its
        // entries converge), so chunks are made as long as the CTAs allow
        want = std::max<uint64_t>(4096, align_up((n + ctas * cpt - 1) / (ctas * cpt), (uint64_t)sfa_dev::SLICE));
        want = std::min<uint64_t>(want, MAX_CHUNK);
    } else {
        // CTA tiles: one tile per resident CTA, so that the scan, look-back
        // and recount after the lookups are paid once per CTA.  Warp tiles:
        // WARP_TILE_ROUNDS tiles per resident warp.  Whole 64-byte slices (a
        // short text takes one slice per chunk: its latency is then the
        // kernel's fixed cost plus one slice)
        const uint64_t slots = ctas * cpt * (sh.wt ? WARP_TILE_ROUNDS : 1);
        want = std::max<uint64_t>(sfa_dev::SLICE, align_up((n + slots - 1) / slots, (uint64_t)sfa_dev::SLICE));
        want = std::min<uint64_t>(want, MAX_CHUNK);
    }
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

void fill_text_map(TextDesc &d, CUtensorMap &map) {
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<EncodeFn>(fn);
    }();
    d.rows2d = 0;
    std::memset(&map, 0, sizeof map);
    const uint8_t *base = d.text + d.origin;   // chunk 0's body, then chunk k at base + k*chunk
    const uint64_t rows = d.chunk && d.n > d.origin ? (d.n - d.origin) / d.chunk : 0;
    if (!encode || d.forced || d.chunk % 16 || d.chunk > 0xffffffffull ||
        (reinterpret_cast<uintptr_t>(base) & 15) || rows == 0 || rows >= (1ull << 31))
        return;
    // the chunk bodies as a [rows][chunk] byte matrix; boxes of 32 chunks x
    // SLICE bytes, 64-byte swizzled in shared memory
    const cuuint64_t dims[2] = {d.chunk, rows};
    const cuuint64_t strides[1] = {d.chunk};
    const cuuint32_t box[2] = {(cuuint32_t)sfa_dev::SLICE, 32};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        d.rows2d = (uint32_t)rows;
}

int launch_kernel(const void *k, int threads, size_t smem, uint32_t ctas, int max_ctas, cudaStream_t s,
                  const Tables &tab, const TextDesc &desc, const CUtensorMap *tmap, const CUtensorMap *tmap_b,
                  const Tables *tabs,
                  const TextDesc *descs, const uint32_t *tile_text, const Scratch &S, sfa_result *out) {
    const int bps = blocks_per_sm(k, threads, smem);
    if (bps < 1) return SFA_ERR_UNSUPPORTED;
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t grid = (uint64_t)bps * device_props(dev).sms;
    if (max_ctas > 0) grid = std::min<uint64_t>(grid, (uint64_t)max_ctas);
    grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, ctas));
    Tables a0 = tab;
    TextDesc a1 = desc;
    alignas(64) CUtensorMap a2, a2b;
    if (tmap)
        a2 = *tmap;
    else
        std::memset(&a2, 0, sizeof a2);
    if (tmap_b)
        a2b = *tmap_b;
    else
        std::memset(&a2b, 0, sizeof a2b);
    const Tables *a3 = tabs;
    const TextDesc *a4 = descs;
    const uint32_t *a5 = tile_text;
    Scratch a6 = S;
    sfa_result *a7 = out;
    void *args[] = {&a0, &a1, &a2, &a2b, &a3, &a4, &a5, &a6, &a7};
    CK(cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, smem, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

// Two levels for a text matched by two CTAs per SM with automatic chunks:
// level A, OLDER_SHARE_PPM of the text, in one tile per SM for the CTA that
// starts first there; level B, the rest, in one tile per SM for the other.
// Sets the level fields of d and returns its tile count, or 0 (one level).
uint64_t plan_two_levels(const Shape &sh, uint64_t n, TextDesc &d) {
    if (sh.wt || sh.forced || !sh.auto_chunk || sh.bps != 2 || sh.simnq || sh.sms < 1) return 0;
    const uint64_t cpt = sh.tile_chunks(), per = (uint64_t)sh.sms * cpt;
    if (n < 4 * per * 256) return 0;
    const uint64_t la = align_up((n / 1000000 * OLDER_SHARE_PPM + n % 1000000 * OLDER_SHARE_PPM / 1000000 + per - 1) / per,
                                 (uint64_t)sfa_dev::SLICE);
    // level B starts on a 16-byte boundary: level A is the origin and per
    // chunks of la bytes
    const uint64_t split = d.origin + per * la;
    if (split >= n) return 0;
    const uint64_t rest = n - split;
    const uint64_t lb = std::max<uint64_t>(256, align_up((rest + per - 1) / per, (uint64_t)sfa_dev::SLICE));
    if (la > MAX_CHUNK || lb > MAX_CHUNK) return 0;
    d.chunk = la;
    d.split = split;
    d.chunk_b = lb;
    d.split_tile = (uint32_t)sh.sms;
    return sh.sms + ((rest + lb - 1) / lb + cpt - 1) / cpt;
}

// the tensor map of level B (d.rows2d_b), when d has two levels
void fill_level_b_map(TextDesc &d, CUtensorMap &map_b) {
    std::memset(&map_b, 0, sizeof map_b);
    d.rows2d_b = 0;
    if (!d.split_tile) return;
    TextDesc b{};
    b.text = d.text + d.split;
    b.n = d.n - d.split;
    b.chunk = d.chunk_b;
    fill_text_map(b, map_b);
    d.rows2d_b = b.rows2d;
}

int match_impl(sfa_handle *h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
               const sfa_launch_opts *o, bool carry, int32_t *d_map) {
    if (!h || !d_out) return SFA_ERR_INVALID;
    if (!h->on_device) return SFA_ERR_HOST_ONLY;
    if (n > MAX_TEXT || (n > 0 && !d_text)) return SFA_ERR_INVALID;
    // the slice mapping is composed from CTA-tile aggregates of byte ids
    if (d_map && o && o->tiling == SFA_TILING_WARP) return SFA_ERR_INVALID;
    if (d_map && h->host.wide) return SFA_ERR_UNSUPPORTED;
    // a text of up to 1 MiB with the automatic shape: one CTA or one cluster
    // of CTAs, no scratch (its latency is a kernel launch and the text's
    // dependent lookups); UNSUPPORTED when no such cluster can be resident
    const bool shape_given = o && (o->chunk_bytes || o->block_threads || o->chains || o->max_ctas ||
                                   o->forced_chunks || o->debug_flags || o->tiling);
    if (!d_map && !shape_given && h->host.mode == SFA_MODE_SFA && !h->host.wide && h->host.nr <= 255 &&
        small_fits(n)) {
        const int rc = launch_small(h->dev, h->host.n_nc, d_text, n, carry, d_out, s);
        if (rc != SFA_ERR_UNSUPPORTED) return rc;   // else: the persistent kernel below
    }
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
    d.origin = d.forced ? 0u : sfa_dev::text_origin(d_text);
    const uint64_t cpt = sh.tile_chunks();
    // chunk indices (and, in simulation mode, the ids nr + chunk) stay below 2^31
    if (sfa_dev::num_chunks(d) >= (1ull << 31) - 256) return SFA_ERR_INVALID;
    uint64_t tiles = plan_two_levels(sh, n, d);
    if (!tiles) tiles = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
    d.ntiles = (uint32_t)tiles;
    const uint32_t nr = h->host.nr;
    const uint64_t vec = sh.simnq ? tiles * cpt * nr : 0;
    // tile aggregates hold one state id per kept state: 2 bytes with 16-bit ids
    ScratchPlan p = plan_scratch(1, tiles, nr * (h->host.wide ? 2u : 1u), vec);
    rc = ensure_scratch(h, p.total);
    if (rc) return rc;
    // a text of one CTA tile: its CTA clears what it reads, no memset
    const bool single = tiles == 1 && !sh.wt;
    if (!single) CK(cudaMemsetAsync(h->d_scratch, 0, p.zero, s));
    Scratch S = make_scratch(h->d_scratch, p, nr, (uint32_t)tiles, sh);
    S.map_mode = d_map ? 1u : 0u;
    S.single = single ? 1u : 0u;
    const void *k = shape_kernel(h, sh);
    const size_t smem = shape_smem(h, sh);
    alignas(64) CUtensorMap map, map_b;
    fill_text_map(d, map);
    fill_level_b_map(d, map_b);
    rc = launch_kernel(k, sh.threads, smem, (uint32_t)sh.ctas_for(tiles), sh.max_ctas, s, h->dev, d, &map,
                       &map_b, nullptr, nullptr, nullptr, S, d_out);
    if (rc || !d_map) return rc;
    return launch_compose_tiles(S.agg, (uint32_t)tiles, nr, h->dev.orig_of, (uint32_t)h->host.nq_in, d_map, s);
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
    if (h->h_res) cudaFreeHost(h->h_res);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
}

}  // namespace sfa_impl

using namespace sfa_impl;

extern "C" {

int sfa_compile(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                const sfa_compile_opts *opts, sfa_handle_t *out) {
    return sfa_compile_sample(delta, nq, q0, accept, opts, nullptr, 0, out);
}

int sfa_compile_sample(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                       const sfa_compile_opts *opts, const uint8_t *sample, uint64_t sample_len,
                       sfa_handle_t *out) {
    if (!out) return SFA_ERR_INVALID;
    *out = nullptr;
    if (!sample && sample_len) return SFA_ERR_INVALID;
    sfa_compile_opts o{};
    if (opts) o = *opts;
    sfa_handle *h = new (std::nothrow) sfa_handle();
    if (!h) return SFA_ERR_OOM;
    int rc;
    try {
        rc = sfa_impl::build_tables(delta, nq, q0, accept, o.cap_states, o.force_mode, h->host,
                                    !(o.flags & SFA_COMPILE_NO_BANK_TUNE), sample, sample_len);
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
    out->n_nonconst = H.mode == SFA_MODE_SFA ? (H.nr > 1 ? H.n_nc + H.n_points : 0) : 0;
    out->n_sfa_states = H.mode == SFA_MODE_SFA ? out->n_nonconst + H.n_const : 0;
    out->table_bytes = h->table_bytes;
    out->compile_seconds = H.seconds;
    out->n_stored = H.mode == SFA_MODE_SFA ? (H.nr > 1 ? H.n_nc : 0) : 0;
    out->id_bits = H.wide ? 16u : 8u;
    if (H.mode == SFA_MODE_SIM)
        out->placement = SFA_PLACE_SMEM_DFA | (simnq_for((uint32_t)H.nr) > 64 ? SFA_PLACE_SMEM_VECTORS : 0u);
    else
        out->placement = (H.wide ? SFA_PLACE_SMEM_DFA_CLASSES : SFA_PLACE_SMEM_DFA) |
                         (out->n_stored ? SFA_PLACE_GLOBAL_NC : 0u);
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
        case SFA_TABLE_CDFA16: src = H.cdfa.data(); sz = H.cdfa.size() * 2; break;
        case SFA_TABLE_MAPS16: src = H.maps16.data(); sz = H.maps16.size() * 2; break;
        case SFA_TABLE_SETS: src = H.setbits.data(); sz = H.setbits.size() * 4; break;
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
        case SFA_ERR_UNSUPPORTED: return "outside the limits of the library";
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

int sfa_match_map(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, int32_t *d_map,
                  sfa_stream_t stream, const sfa_launch_opts *opts) {
    if (!d_map) return SFA_ERR_INVALID;
    return match_impl(h, d_text, n, d_out, (cudaStream_t)stream, opts, false, d_map);
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
    // a short text in host memory the device can read (pinned and mapped):
    // the short-text kernel reads it in place over the host link, so there
    // is no staging copy and no event (up to IN_PLACE_MAX bytes: past that
    // the staged copy, a copy-engine transfer, is faster than the kernel's
    // reads of host memory); any other case is copied in pieces (the
    // persistent kernel's bulk copies read device memory only)
    constexpr uint64_t IN_PLACE_MAX = 256 << 10;
    const bool shape_given = opts && (opts->chunk_bytes || opts->block_threads || opts->chains || opts->max_ctas ||
                                      opts->forced_chunks || opts->debug_flags || opts->tiling);
    if (n > 0 && n <= IN_PLACE_MAX && !shape_given && h->host.mode == SFA_MODE_SFA && !h->host.wide &&
        h->host.nr <= 255 && small_fits(n)) {
        if (const uint8_t *dp = device_readable(h_text)) {
            // the kernel writes its result straight to mapped pinned memory
            if (!h->h_res) {
                CK(cudaHostAlloc(reinterpret_cast<void **>(&h->h_res), sizeof(sfa_result), cudaHostAllocMapped));
                CK(cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->h_res_dev), h->h_res, 0));
            }
            rc = launch_small(h->dev, h->host.n_nc, dp, n, false, h->h_res_dev, s);
            if (rc == SFA_OK) {
                CK(cudaStreamSynchronize(s));
                std::memcpy(h_out, h->h_res, sizeof(sfa_result));
                return SFA_OK;
            }
            if (rc != SFA_ERR_UNSUPPORTED) return rc;
            rc = SFA_OK;
        }
    }
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
// matching on a fixed, caller-provided scratch buffer (sfa_match_noalloc)
// ---------------------------------------------------------------------------
namespace sfa_impl {

namespace {

// Host-side part of sfa_match_noalloc: argument checks, the handle's device,
// the launch shape and the scratch it needs, all decided before any work is
// enqueued and before the fixed array's address is looked up.  (The shape
// itself asks the runtime for occupancy figures: those calls enqueue nothing.)
int plan_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, const sfa_result *d_out, size_t cap,
                      Shape &sh, TextDesc &d, ScratchPlan &p) {
    if (!h || !d_out) return SFA_ERR_INVALID;
    if (n > MAX_TEXT || (n > 0 && !d_text)) return SFA_ERR_INVALID;
    if (h->host.mode != SFA_MODE_SFA) return SFA_ERR_UNSUPPORTED;
    if (!h->on_device) return SFA_ERR_HOST_ONLY;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return SFA_ERR_INVALID;
    // the automatic shape: with automatic chunks a text has at most one CTA
    // tile per resident CTA, whatever its length
    int rc = choose_shape(h, n, nullptr, sh);
    if (rc) return rc;
    d = TextDesc{};
    d.text = d_text;
    d.n = n;
    d.chunk = sh.chunk;
    d.forced = 0;
    d.origin = sfa_dev::text_origin(d_text);
    const uint64_t cpt = sh.tile_chunks();
    if (sfa_dev::num_chunks(d) >= (1ull << 31) - 256) return SFA_ERR_SCRATCH_LIMIT;
    uint64_t tiles = plan_two_levels(sh, n, d);
    if (!tiles) tiles = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
    d.ntiles = (uint32_t)tiles;
    p = plan_scratch(1, tiles, h->host.nr * (h->host.wide ? 2u : 1u), 0);
    return p.total <= cap ? SFA_OK : SFA_ERR_SCRATCH_LIMIT;
}

}  // namespace

int check_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, const sfa_result *d_out, size_t cap) {
    Shape sh;
    TextDesc d;
    ScratchPlan p;
    return plan_into_scratch(h, d_text, n, d_out, cap, sh, d, p);
}

int match_into_scratch(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, cudaStream_t s,
                       uint8_t *scratch, size_t cap, int scratch_device) {
    Shape sh;
    TextDesc d;
    ScratchPlan p;
    int rc = plan_into_scratch(h, d_text, n, d_out, cap, sh, d, p);
    if (rc) return rc;
    if (!scratch) return SFA_ERR_INVALID;
    if (h->device != scratch_device) return SFA_ERR_INVALID;
    const uint64_t tiles = d.ntiles;
    const uint32_t nr = h->host.nr;
    // the buffer keeps the previous call's contents: clear the header, the
    // text record and the look-back descriptors
    CK(cudaMemsetAsync(scratch, 0, p.zero, s));
    const Scratch S = make_scratch(scratch, p, nr, (uint32_t)tiles, sh);
    const void *k = shape_kernel(h, sh);
    const size_t smem = shape_smem(h, sh);
    alignas(64) CUtensorMap map, map_b;
    fill_text_map(d, map);
    fill_level_b_map(d, map_b);
    return launch_kernel(k, sh.threads, smem, (uint32_t)sh.ctas_for(tiles), 0, s, h->dev, d, &map, &map_b, nullptr,
                         nullptr, nullptr, S, d_out);
}

}  // namespace sfa_impl
