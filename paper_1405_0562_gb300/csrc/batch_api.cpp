// Batches (declared in include/sfa.h): one persistent launch over many
// (automaton, text) pairs, each text with its own look-back chain and record
// (Theorem 3 applied per text).  Plans are either exact (sfa_batch_create:
// one work list, uploaded once) or reserved (sfa_batch_reserve: capacity
// only; sfa_batch_update refills the work list asynchronously from pinned
// staging, for the serving loop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "api_internal.h"

using sfa_dev::Scratch;
using sfa_dev::Tables;
using sfa_dev::TextDesc;
using namespace sfa_impl;

struct sfa_batch {
    int device = -1;
    Shape shape;
    const void *kernel = nullptr;
    size_t smem = 0;
    bool reserved = false;
    uint64_t chunk = 0;                 // chunk length of texts that fill a tile
    // capacity and device layout: [tables][descriptors][tensor maps][tile map:
    // count, then grab position -> tile, then tile -> text]
    int32_t cap_texts = 0;
    uint64_t cap_tiles = 0;
    uint32_t nr_max = 0;
    size_t off_tabs = 0, off_descs = 0, off_maps = 0, off_tt = 0, mem_bytes = 0;
    size_t off_gd = 0, off_gu = 0;      // copy-in by one kernel: descriptors, unit prefix sums
    uint8_t *d_mem = nullptr;
    uint8_t *d_scratch = nullptr;
    ScratchPlan plan{};
    Scratch S{};
    // current work list
    int32_t k = 0;
    uint32_t total_tiles = 0;
    size_t used_tabs = 0, used_descs = 0, used_maps = 0, used_tt = 0;
    std::vector<int32_t> sim_index;     // texts whose handle is in simulation mode:
    std::vector<sfa_handle_t> sim_handle;   // matched one by one
    std::vector<const uint8_t *> sim_text;
    std::vector<uint64_t> sim_len;
    // pinned staging of the work list (reserved plans), double buffered
    uint8_t *h_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    int stage = 0;
    // CUDA graph of the launch
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    sfa_result *exec_out = nullptr;
    // The texts a plan takes: 0 = D-SFA texts of byte-id automata; > 0 =
    // simulation-mode texts whose vectors have this many entries.  An exact
    // plan holds one sub-plan per vector size among its texts (each a
    // persistent launch of that size's kernel); texts of 16-bit-id automata,
    // and simulation texts of reserved plans, take per-text launches.
    int want_simnq = 0;
    std::vector<sfa_batch *> subs;
};

namespace {

void set_layout(sfa_batch *b) {
    b->off_tabs = 0;
    b->off_descs = align_up((size_t)b->cap_texts * sizeof(Tables), 256);
    b->off_maps = align_up(b->off_descs + (size_t)b->cap_texts * sizeof(TextDesc), 256);
    b->off_tt = align_up(b->off_maps + (size_t)b->cap_texts * sizeof(CUtensorMap), 256);
    b->off_gd = align_up(b->off_tt + (size_t)(1 + 2 * b->cap_tiles) * 4, 256);
    b->off_gu = b->off_gd + (size_t)b->cap_texts * sizeof(GatherDesc);
    b->mem_bytes = align_up(b->off_gu + (size_t)(b->cap_texts + 1) * 4, 256);
}

// Chunk length of one text: `chunk`, shortened for texts that would not fill
// a tile, so that small texts still spread over many threads.
uint64_t text_chunk(uint64_t n, uint64_t chunk, uint64_t cpt) {
    return std::min<uint64_t>(chunk, std::max<uint64_t>(64, align_up((n + cpt - 1) / cpt, 16)));
}

// (an upper bound for any origin: an origin never adds a chunk)
uint64_t text_tiles(uint64_t n, uint64_t chunk, uint64_t cpt) {
    TextDesc d{};
    d.n = n;
    d.chunk = text_chunk(n, chunk, cpt);
    return (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
}

int check_inputs(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens, int32_t k,
                 int dev) {
    if (k < 0 || (k > 0 && (!hs || !d_texts || !lens))) return SFA_ERR_INVALID;
    for (int32_t i = 0; i < k; ++i) {
        sfa_handle_t h = hs[i];
        if (!h) return SFA_ERR_INVALID;
        if (!h->on_device) return SFA_ERR_HOST_ONLY;
        if (h->device != dev || lens[i] > MAX_TEXT || (lens[i] && !d_texts[i])) return SFA_ERR_INVALID;
    }
    return SFA_OK;
}

// Builds the work list of the texts into `img` (the device layout of b):
// texts sorted by automaton (stable), every text's tiles consecutive (tile
// ids: the look-back walks a text's tiles by id).  CTAs take the tiles in
// another order: texts by decreasing chunk-length class (a tile lasts about
// as long as its chunks), automata still grouped within a class, each text's
// tiles in id order (a tile's look-back only waits for tiles taken before
// it), so that the last tiles taken are the shortest.
int fill_worklist(sfa_batch *b, const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                  int32_t k, uint8_t *img) {
    const uint64_t cpt = (uint64_t)b->shape.threads * b->shape.chains;
    b->sim_index.clear();
    b->sim_handle.clear();
    b->sim_text.clear();
    b->sim_len.clear();
    std::vector<int32_t> order;
    std::vector<sfa_handle_t> distinct;
    std::map<sfa_handle_t, uint32_t> tab_of;
    for (int32_t i = 0; i < k; ++i) {
        sfa_handle_t h = hs[i];
        const bool sim = h->host.mode == SFA_MODE_SIM;
        if (b->want_simnq > 0) {
            if (!sim || simnq_for((uint32_t)h->host.nr) != b->want_simnq) continue;   // another plan's
        } else if (sim && !b->reserved) {
            continue;   // a sub-plan's
        } else if (sim || h->host.wide) {
            b->sim_index.push_back(i);
            b->sim_handle.push_back(h);
            b->sim_text.push_back(d_texts[i]);
            b->sim_len.push_back(lens[i]);
            continue;
        }
        if ((uint32_t)h->host.nr > b->nr_max) return SFA_ERR_INVALID;
        if (!tab_of.count(h)) {
            tab_of[h] = (uint32_t)distinct.size();
            distinct.push_back(h);
        }
        order.push_back(i);
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return tab_of[hs[x]] < tab_of[hs[y]]; });
    Tables *tabs = reinterpret_cast<Tables *>(img + b->off_tabs);
    TextDesc *descs = reinterpret_cast<TextDesc *>(img + b->off_descs);
    uint32_t *tt = reinterpret_cast<uint32_t *>(img + b->off_tt);
    for (size_t j = 0; j < distinct.size(); ++j) tabs[j] = distinct[j]->dev;
    uint64_t tiles = 0;
    std::vector<uint32_t> text_of;   // tile id -> text
    for (size_t j = 0; j < order.size(); ++j) {
        const int32_t i = order[j];
        TextDesc d{};
        d.text = d_texts[i];
        d.n = lens[i];
        d.chunk = text_chunk(d.n, b->chunk, cpt);
        d.forced = 0;
        d.origin = sfa_dev::text_origin(d.text);
        if (sfa_dev::num_chunks(d) >= (1ull << 31)) return SFA_ERR_INVALID;
        const uint64_t t = (sfa_dev::num_chunks(d) + cpt - 1) / cpt;
        if (tiles + t > b->cap_tiles) return SFA_ERR_INVALID;
        d.ntiles = (uint32_t)t;
        d.tile_base = (uint32_t)tiles;
        d.table = tab_of[hs[i]];
        d.out_index = (uint32_t)i;
        d.carry = 0;
        // the text's tensor map, in the plan's device memory
        alignas(64) CUtensorMap map;
        fill_text_map(d, map);
        std::memcpy(img + b->off_maps + j * sizeof(CUtensorMap), &map, sizeof map);
        d.map = d.rows2d ? b->d_mem + b->off_maps + j * sizeof(CUtensorMap) : nullptr;
        text_of.insert(text_of.end(), t, (uint32_t)j);
        tiles += t;
        descs[j] = d;
    }
    std::vector<uint32_t> by(order.size());
    for (size_t j = 0; j < by.size(); ++j) by[j] = (uint32_t)j;
    auto cls = [&](uint32_t j) { return 63 - __builtin_clzll(std::max<uint64_t>(descs[j].chunk, 1)); };
    std::stable_sort(by.begin(), by.end(), [&](uint32_t x, uint32_t y) { return cls(x) > cls(y); });
    tt[0] = (uint32_t)tiles;
    uint64_t pos = 0;
    for (uint32_t j : by)
        for (uint32_t u = 0; u < descs[j].ntiles; ++u) tt[1 + pos++] = descs[j].tile_base + u;
    std::memcpy(tt + 1 + tiles, text_of.data(), text_of.size() * sizeof(uint32_t));
    b->k = k;
    b->total_tiles = (uint32_t)tiles;
    b->used_tabs = distinct.size() * sizeof(Tables);
    b->used_descs = order.size() * sizeof(TextDesc);
    b->used_maps = order.size() * sizeof(CUtensorMap);
    b->used_tt = (size_t)(1 + 2 * tiles) * 4;
    return SFA_OK;
}

// simulation-mode texts and texts of 16-bit-id automata are matched with
// their handle's own scratch: size it now, so that launches of the plan (and
// graph captures) never allocate.  The tile count is bounded above (a text
// of two levels has up to one more tile per SM than one level would).
int size_sim_scratch(sfa_batch *b) {
    for (size_t i = 0; i < b->sim_index.size(); ++i) {
        sfa_handle_t h = b->sim_handle[i];
        Shape ss;
        int rc = choose_shape(h, b->sim_len[i], nullptr, ss);
        if (rc) return rc;
        TextDesc d{};
        d.n = b->sim_len[i];
        d.chunk = ss.chunk;
        const uint64_t c2 = ss.tile_chunks();
        const uint64_t t = (sfa_dev::num_chunks(d) + c2 - 1) / c2 + (uint64_t)std::max(ss.sms, 0) + 2;
        const uint64_t vec = ss.simnq ? t * c2 * h->host.nr : 0;
        rc = ensure_scratch(h, plan_scratch(1, t, h->host.nr * (h->host.wide ? 2u : 1u), vec).total);
        if (rc) return rc;
    }
    return SFA_OK;
}

int batch_enqueue(sfa_batch *b, sfa_result *d_out, cudaStream_t s) {
    for (sfa_batch *sub : b->subs) {
        int rc = batch_enqueue(sub, d_out, s);
        if (rc) return rc;
    }
    if (b->reserved || b->total_tiles > 0) {
        CK(cudaMemsetAsync(b->d_scratch, 0, b->plan.zero, s));
        // reserved plans launch every resident CTA: the tile count is read on
        // the device, so the launch does not depend on the work list
        const uint32_t grid_tiles = b->reserved ? 0xffffffffu : b->total_tiles;
        int rc = launch_kernel(b->kernel, b->shape.threads, b->smem, grid_tiles, b->shape.max_ctas, s, Tables{},
                               TextDesc{}, nullptr, nullptr, reinterpret_cast<const Tables *>(b->d_mem + b->off_tabs),
                               reinterpret_cast<const TextDesc *>(b->d_mem + b->off_descs),
                               reinterpret_cast<const uint32_t *>(b->d_mem + b->off_tt), b->S, d_out);
        if (rc) return rc;
    }
    for (size_t i = 0; i < b->sim_index.size(); ++i) {
        int rc = match_impl(b->sim_handle[i], b->sim_text[i], b->sim_len[i], d_out + b->sim_index[i], s, nullptr,
                            false);
        if (rc) return rc;
    }
    return SFA_OK;
}

// kernels one launch of the plan enqueues
uint64_t batch_launches(const sfa_batch *b) {
    uint64_t n = (b->reserved || b->total_tiles > 0 ? 1 : 0) + b->sim_index.size();
    for (const sfa_batch *sub : b->subs) n += batch_launches(sub);
    return n;
}

void batch_free(sfa_batch *b) {
    for (sfa_batch *sub : b->subs) {
        batch_free(sub);
        delete sub;
    }
    b->subs.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->d_scratch) cudaFree(b->d_scratch);
    for (int i = 0; i < 2; ++i) {
        if (b->h_stage[i]) cudaFreeHost(b->h_stage[i]);
        if (b->ev_stage[i]) cudaEventDestroy(b->ev_stage[i]);
    }
}

int init_shape(sfa_batch *b, const sfa_launch_opts *opts) {
    Shape &sh = b->shape;
    sh.threads = 512;   // two CTAs per SM for automata up to ~150 states
    sh.chains = 1;
    if (b->want_simnq) {
        // the single-text simulation shapes; the caller's options do not apply
        sh.threads = b->want_simnq > 64 ? 256 : 128;
        sh.simnq = b->want_simnq;
        if (opts && opts->timeout_us) sh.timeout_us = opts->timeout_us;
        if (opts) sh.debug = opts->debug_flags;
        b->kernel = kernel_for(sh.threads, 1, b->want_simnq, true);
        return b->kernel ? SFA_OK : SFA_ERR_UNSUPPORTED;
    }
    if (opts) {
        if (opts->block_threads) sh.threads = (int)opts->block_threads;
        if (opts->chains) sh.chains = (int)opts->chains;
        if (opts->timeout_us) sh.timeout_us = opts->timeout_us;
        sh.debug = opts->debug_flags;
        sh.max_ctas = (int)opts->max_ctas;
        if (opts->chunk_bytes > MAX_CHUNK) return SFA_ERR_INVALID;
        if (opts->tiling > SFA_TILING_WARP) return SFA_ERR_INVALID;
        if (opts->tiling == SFA_TILING_WARP) return SFA_ERR_UNSUPPORTED;   // batches take CTA tiles
    }
    b->kernel = kernel_for(sh.threads, sh.chains, 0, true);
    return b->kernel ? SFA_OK : SFA_ERR_UNSUPPORTED;
}

int alloc_device(sfa_batch *b) {
    set_layout(b);
    const uint32_t nrm = std::max<uint32_t>(b->nr_max, 1);
    // simulation plans: a chunk vector of nr_max bytes per chunk
    const uint64_t vec = b->want_simnq ? b->cap_tiles * (uint64_t)b->shape.threads * b->shape.chains * nrm : 0;
    b->plan = plan_scratch((uint32_t)std::max(b->cap_texts, 1), b->cap_tiles, nrm, vec);
    CK(cudaMalloc(&b->d_mem, b->mem_bytes));
    CK(cudaMalloc(&b->d_scratch, b->plan.total));
    b->S = make_scratch(b->d_scratch, b->plan, nrm, 0, b->shape);
    b->smem = smem_bytes(b->shape.threads, b->shape.chains, nrm, b->want_simnq);
    blocks_per_sm(b->kernel, b->shape.threads, b->smem);   // cached before any capture
    return SFA_OK;
}

// An exact plan over the texts of kind `simnq` (see sfa_batch::want_simnq).
int create_plan(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens, int32_t k,
                const sfa_launch_opts *opts, int dev, int simnq, sfa_batch **out) {
    sfa_batch *b = new (std::nothrow) sfa_batch();
    if (!b) return SFA_ERR_OOM;
    b->device = dev;
    b->want_simnq = simnq;
    int rc = init_shape(b, opts);
    if (rc) {
        delete b;
        return rc;
    }
    auto mine = [&](int32_t i) {
        const bool sim = hs[i]->host.mode == SFA_MODE_SIM;
        return simnq ? sim && simnq_for((uint32_t)hs[i]->host.nr) == simnq : !sim && !hs[i]->host.wide;
    };
    const uint64_t cpt = (uint64_t)b->shape.threads * b->shape.chains;
    uint64_t total_bytes = 0;
    for (int32_t i = 0; i < k; ++i) {
        if (!mine(i)) continue;
        b->nr_max = std::max<uint32_t>(b->nr_max, (uint32_t)hs[i]->host.nr);
        total_bytes += lens[i];
    }
    // chunk length: D-SFA texts as for one text of the batch's total size
    // (six tiles per resident CTA); simulation texts with one tile per
    // resident CTA and at least 4 KiB, as for a single text (every chunk
    // pays the vector phase)
    b->chunk = !simnq && opts && opts->chunk_bytes ? opts->chunk_bytes : 0;
    if (!b->chunk) {
        const size_t smem = smem_bytes(b->shape.threads, b->shape.chains, std::max<uint32_t>(b->nr_max, 1), simnq);
        const int bps = blocks_per_sm(b->kernel, b->shape.threads, smem);
        const uint64_t ctas = (uint64_t)std::max(1, bps) * std::max(1, device_props(dev).sms);
        if (simnq)
            b->chunk = std::min<uint64_t>(MAX_CHUNK, std::max<uint64_t>(4096, align_up(total_bytes / (ctas * cpt), 64)));
        else
            b->chunk = std::min<uint64_t>(4096, std::max<uint64_t>(256, align_up(total_bytes / (ctas * 6 * cpt), 16)));
    }
    uint64_t tiles = 0;
    for (int32_t i = 0; i < k; ++i)
        if (mine(i)) tiles += text_tiles(lens[i], b->chunk, cpt);
    if (tiles >= (1ull << 30)) {
        delete b;
        return SFA_ERR_INVALID;
    }
    b->cap_texts = std::max(k, 1);
    b->cap_tiles = tiles;
    rc = alloc_device(b);
    std::vector<uint8_t> img;
    if (!rc) {
        img.assign(b->mem_bytes, 0);
        rc = fill_worklist(b, hs, d_texts, lens, k, img.data());
    }
    if (!rc) rc = cuda_err(cudaMemcpy(b->d_mem, img.data(), b->mem_bytes, cudaMemcpyHostToDevice));
    if (!rc) rc = size_sim_scratch(b);
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return SFA_OK;
}

}  // namespace

extern "C" {

int sfa_batch_create(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens, int32_t k,
                     const sfa_launch_opts *opts, sfa_batch_t *out) {
    if (!out) return SFA_ERR_INVALID;
    *out = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int rc = check_inputs(hs, d_texts, lens, k, dev);
    if (rc) return rc;
    sfa_batch *b = nullptr;
    rc = create_plan(hs, d_texts, lens, k, opts, dev, 0, &b);
    // one sub-plan per vector size of the simulation-mode texts
    for (int nq : {16, 32, 64, 128, 256}) {
        bool any = false;
        for (int32_t i = 0; i < k && !any; ++i)
            any = hs[i]->host.mode == SFA_MODE_SIM && simnq_for((uint32_t)hs[i]->host.nr) == nq;
        if (rc || !any) continue;
        sfa_batch *sub = nullptr;
        rc = create_plan(hs, d_texts, lens, k, opts, dev, nq, &sub);
        if (!rc) b->subs.push_back(sub);
    }
    if (rc) {
        if (b) {
            batch_free(b);
            delete b;
        }
        return rc;
    }
    *out = b;
    return SFA_OK;
}

int sfa_batch_reserve(int32_t max_texts, uint64_t max_tiles, uint32_t nr_max, const sfa_launch_opts *opts,
                      sfa_batch_t *out) {
    if (!out || max_texts < 1 || max_tiles < 1 || max_tiles >= (1ull << 30) || nr_max < 1 || nr_max > 256)
        return SFA_ERR_INVALID;
    *out = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    sfa_batch *b = new (std::nothrow) sfa_batch();
    if (!b) return SFA_ERR_OOM;
    b->device = dev;
    b->reserved = true;
    int rc = init_shape(b, opts);
    b->chunk = opts && opts->chunk_bytes ? opts->chunk_bytes : 1024;
    b->cap_texts = max_texts;
    b->cap_tiles = max_tiles;
    b->nr_max = nr_max;
    if (!rc) rc = alloc_device(b);
    if (!rc) rc = cuda_err(cudaMemset(b->d_mem, 0, b->mem_bytes));   // empty work list
    for (int i = 0; i < 2 && !rc; ++i) {
        rc = cuda_err(cudaHostAlloc(reinterpret_cast<void **>(&b->h_stage[i]), b->mem_bytes, cudaHostAllocDefault));
        if (!rc) rc = cuda_err(cudaEventCreateWithFlags(&b->ev_stage[i], cudaEventDisableTiming));
    }
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return SFA_OK;
}

}  // extern "C"

namespace {

// sfa_batch_update, and (ng > 0) the copy-in of ng texts by one kernel:
// gd[i] and gu[i] (first unit of text i; gu[ng] = all units) are staged with
// the work list and the copy kernel runs before the work list upload
int update_impl(sfa_batch_t b, const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                int32_t k, cudaStream_t s, const GatherDesc *gd, const uint32_t *gu, uint32_t ng) {
    if (!b || !b->reserved) return SFA_ERR_INVALID;
    if (k > b->cap_texts || ng > (uint32_t)b->cap_texts) return SFA_ERR_INVALID;
    int rc = check_inputs(hs, d_texts, lens, k, b->device);
    if (rc) return rc;
    const int st = b->stage ^ 1;
    // the staging buffer may still be the source of the copy two updates ago
    CK(cudaEventSynchronize(b->ev_stage[st]));
    if (ng) {
        uint8_t *h = b->h_stage[st];
        std::memcpy(h + b->off_gd, gd, (size_t)ng * sizeof(GatherDesc));
        std::memcpy(h + b->off_gu, gu, (size_t)(ng + 1) * 4);
        CK(cudaMemcpyAsync(b->d_mem + b->off_gd, h + b->off_gd, b->off_gu - b->off_gd + (size_t)(ng + 1) * 4,
                           cudaMemcpyHostToDevice, s));
        rc = launch_gather(reinterpret_cast<const GatherDesc *>(b->d_mem + b->off_gd),
                           reinterpret_cast<const uint32_t *>(b->d_mem + b->off_gu), ng, gu[ng], s);
        if (rc) return rc;
    }
    const size_t prev_sims = b->sim_index.size();
    rc = fill_worklist(b, hs, d_texts, lens, k, b->h_stage[st]);
    if (rc) return rc;
    if (!b->sim_index.empty() || prev_sims) {
        rc = size_sim_scratch(b);
        if (rc) return rc;
        if (b->exec) {   // the captured launch no longer matches the work list
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    uint8_t *h = b->h_stage[st];
    if (b->used_tabs) CK(cudaMemcpyAsync(b->d_mem + b->off_tabs, h + b->off_tabs, b->used_tabs, cudaMemcpyHostToDevice, s));
    if (b->used_descs)
        CK(cudaMemcpyAsync(b->d_mem + b->off_descs, h + b->off_descs, b->used_descs, cudaMemcpyHostToDevice, s));
    if (b->used_maps)
        CK(cudaMemcpyAsync(b->d_mem + b->off_maps, h + b->off_maps, b->used_maps, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->d_mem + b->off_tt, h + b->off_tt, b->used_tt, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(b->ev_stage[st], s));
    b->stage = st;
    return SFA_OK;
}

}  // namespace

extern "C" {

int sfa_batch_update(sfa_batch_t b, const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                     int32_t k, sfa_stream_t stream) {
    return update_impl(b, hs, d_texts, lens, k, (cudaStream_t)stream, nullptr, nullptr, 0);
}

int sfa_batch_update_host(sfa_batch_t b, const sfa_handle_t *hs, const uint8_t *const *h_texts,
                          uint8_t *const *d_dst, const uint64_t *lens, int32_t k, sfa_stream_t stream) {
    if (!b || !b->reserved || k < 0 || k > b->cap_texts) return SFA_ERR_INVALID;
    if (k > 0 && (!h_texts || !d_dst || !lens)) return SFA_ERR_INVALID;
    for (int32_t i = 0; i < k; ++i)
        if (lens[i] && (!h_texts[i] || !d_dst[i])) return SFA_ERR_INVALID;
    int rc = check_inputs(hs, reinterpret_cast<const uint8_t *const *>(d_dst), lens, k, b->device);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // texts in host memory the device can read: one copy kernel for all;
    // the others: one cudaMemcpyAsync each
    std::vector<GatherDesc> gd;
    std::vector<uint32_t> gu;
    uint64_t units = 0;
    ReadableRange rr;   // this call's texts stay allocated until it returns
    for (int32_t i = 0; i < k; ++i) {
        if (!lens[i]) continue;
        const uint8_t *src = device_readable(h_texts[i], &rr);
        if (src) {
            gu.push_back((uint32_t)units);
            gd.push_back(GatherDesc{src, d_dst[i], lens[i]});
            units += (lens[i] + GATHER_UNIT - 1) / GATHER_UNIT;
        } else {
            CK(cudaMemcpyAsync(d_dst[i], h_texts[i], lens[i], cudaMemcpyHostToDevice, s));
        }
    }
    if (units >= (1ull << 32)) return SFA_ERR_INVALID;
    gu.push_back((uint32_t)units);
    return update_impl(b, hs, reinterpret_cast<const uint8_t *const *>(d_dst), lens, k, s, gd.data(), gu.data(),
                       (uint32_t)gd.size());
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
    g_launches.fetch_add(batch_launches(b), std::memory_order_relaxed);
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
