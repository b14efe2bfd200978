// Continuous-batching match server: the serving loop around the batched
// kernel, in native code.  Requests (automaton, host text) are queued,
// admitted first in, first out while the device text arena has room and a
// batch slot is free, copied into the arena and matched in one persistent
// launch per batch on the slot's stream (sfa_batch_update_host +
// sfa_batch_launch on a reserved plan: nothing is allocated per request);
// finished batches are found by event queries.  No call waits for the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "api_internal.h"

namespace {

constexpr uint64_t ARENA_ALIGN = 256;
// A request's text sits in its arena range at the same offset modulo 16 as
// its host copy, so that the copy kernel moves 16-byte vectors on both sides;
// ranges are TEXT_PAD bytes longer than their text for that.
constexpr uint64_t TEXT_PAD = 15;

uint64_t arena_round(uint64_t n) {
    return std::max<uint64_t>(ARENA_ALIGN, (n + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN);
}

}  // namespace

// First-fit allocator of byte ranges of a fixed arena (offsets only), ranges
// rounded up to 256 bytes, free neighbours merged.
struct sfa_arena {
    uint64_t size = 0, used = 0;
    std::map<uint64_t, uint64_t> free;   // start -> length

    explicit sfa_arena(uint64_t n) : size(n) {
        if (n) free[0] = n;
    }
    bool alloc(uint64_t n, uint64_t &off) {
        n = arena_round(n);
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < n) continue;
            off = it->first;
            const uint64_t rest = it->second - n;
            free.erase(it);
            if (rest) free[off + n] = rest;
            used += n;
            return true;
        }
        return false;
    }
    bool release(uint64_t off, uint64_t n) {
        n = arena_round(n);
        if (off + n > size || n > used) return false;
        auto it = free.lower_bound(off);
        if (it != free.end() && it->first < off + n) return false;   // overlaps a free range
        if (it != free.begin() && std::prev(it)->first + std::prev(it)->second > off) return false;
        used -= n;
        it = free.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
        return true;
    }
};

namespace {

struct Req {
    int32_t automaton;
    const uint8_t *text;
    uint64_t len;
    uint64_t tag;
    uint64_t off;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t t_copy = nullptr, t_match = nullptr, t_end = nullptr;   // SFA_SERVER_TIMING
    uint64_t bytes = 0;
    sfa_batch_t plan = nullptr;
    sfa_result *d_out = nullptr;
    sfa_result *h_out = nullptr;   // pinned
    std::vector<Req> reqs;
    bool busy = false;
};

}  // namespace

struct sfa_server {
    int device = -1;
    std::vector<sfa_handle_t> automata;
    uint8_t *d_arena = nullptr;
    sfa_arena *arena = nullptr;
    int32_t max_batch = 0;
    std::vector<Slot> slots;
    std::deque<Req> queue;
    std::deque<sfa_completion> done;
    bool timing = false;
    cudaEvent_t t_origin = nullptr;
    std::deque<sfa_batch_span> spans;
    uint64_t batches = 0, requests = 0;
    std::vector<sfa_handle_t> hs;
    std::vector<const uint8_t *> src;
    std::vector<uint8_t *> dst;
    std::vector<uint64_t> lens;
};

namespace {

void server_free(sfa_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.plan) sfa_batch_destroy(sl.plan);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.ev) cudaEventDestroy(sl.ev);
        for (cudaEvent_t e : {sl.t_copy, sl.t_match, sl.t_end})
            if (e) cudaEventDestroy(e);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->t_origin) cudaEventDestroy(s->t_origin);
    if (s->d_arena) cudaFree(s->d_arena);
    delete s->arena;
    delete s;
}

// finished batches -> completions, their arena ranges released
int server_reap(sfa_server *s) {
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return sfa_impl::cuda_err(q);
        if (s->timing) {
            sfa_batch_span sp{};
            sp.slot = (int32_t)(&sl - s->slots.data());
            sp.requests = (int32_t)sl.reqs.size();
            sp.bytes = sl.bytes;
            cudaEventElapsedTime(&sp.copy_start_ms, s->t_origin, sl.t_copy);
            cudaEventElapsedTime(&sp.copy_end_ms, s->t_origin, sl.t_match);
            cudaEventElapsedTime(&sp.match_end_ms, s->t_origin, sl.t_end);
            s->spans.push_back(sp);
        }
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            s->done.push_back(sfa_completion{sl.reqs[i].tag, sl.h_out[i]});
            if (sl.reqs[i].len) s->arena->release(sl.reqs[i].off, sl.reqs[i].len + TEXT_PAD);
        }
        sl.reqs.clear();
        sl.busy = false;
    }
    return SFA_OK;
}

// queued requests -> free slots, FIFO, while the arena has room
int server_admit(sfa_server *s) {
    for (Slot &sl : s->slots) {
        if (s->queue.empty()) break;
        if (sl.busy) continue;
        sl.reqs.clear();
        while (!s->queue.empty() && (int32_t)sl.reqs.size() < s->max_batch) {
            Req r = s->queue.front();
            if (r.len && !s->arena->alloc(r.len + TEXT_PAD, r.off)) break;
            s->queue.pop_front();
            sl.reqs.push_back(r);
        }
        if (sl.reqs.empty()) break;   // the head of the queue waits for memory
        const int32_t k = (int32_t)sl.reqs.size();
        s->hs.resize(k);
        s->src.resize(k);
        s->dst.resize(k);
        s->lens.resize(k);
        for (int32_t i = 0; i < k; ++i) {
            const Req &r = sl.reqs[i];
            s->hs[i] = s->automata[r.automaton];
            s->src[i] = r.text;
            s->dst[i] = r.len ? s->d_arena + r.off + (reinterpret_cast<uintptr_t>(r.text) & 15u) : nullptr;
            s->lens[i] = r.len;
        }
        sl.bytes = 0;
        for (int32_t i = 0; i < k; ++i) sl.bytes += s->lens[i];
        int rc = SFA_OK;
        if (s->timing) rc = sfa_impl::cuda_err(cudaEventRecord(sl.t_copy, sl.stream));
        if (!rc)
            rc = sfa_batch_update_host(sl.plan, s->hs.data(), s->src.data(), s->dst.data(), s->lens.data(), k,
                                       sl.stream);
        if (!rc && s->timing) rc = sfa_impl::cuda_err(cudaEventRecord(sl.t_match, sl.stream));
        if (!rc) rc = sfa_batch_launch(sl.plan, sl.d_out, sl.stream);
        if (!rc && s->timing) rc = sfa_impl::cuda_err(cudaEventRecord(sl.t_end, sl.stream));
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)k * sizeof(sfa_result),
                                            cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
            if (e != cudaSuccess) {
                // the batch may still run, but its completion cannot be
                // observed: wait for the stream before the arena is reused
                cudaStreamSynchronize(sl.stream);
                rc = sfa_impl::cuda_err(e);
            }
        }
        if (rc) {
            // put the requests back at the head of the queue, in order
            for (int32_t i = k - 1; i >= 0; --i) {
                if (sl.reqs[i].len) s->arena->release(sl.reqs[i].off, sl.reqs[i].len + TEXT_PAD);
                s->queue.push_front(sl.reqs[i]);
            }
            sl.reqs.clear();
            return rc;
        }
        sl.busy = true;
        ++s->batches;
        s->requests += (uint64_t)k;
    }
    return SFA_OK;
}

}  // namespace

extern "C" {

int sfa_server_create(const sfa_handle_t *automata, int32_t n, const sfa_server_opts *opts, sfa_server_t *out) {
    if (!out || n < 1 || !automata) return SFA_ERR_INVALID;
    *out = nullptr;
    sfa_server_opts o{};
    if (opts) o = *opts;
    const uint64_t budget = o.hbm_budget ? o.hbm_budget : (4ull << 30);
    const int32_t max_batch = o.max_batch > 0 ? o.max_batch : 256;
    const int32_t nslots = o.slots > 0 ? o.slots : 3;
    const uint32_t chunk = o.chunk_bytes ? o.chunk_bytes : 1024;
    const uint32_t threads = o.block_threads ? o.block_threads : 512;
    if (max_batch > (1 << 20) || nslots > 64 || budget > sfa_impl::MAX_TEXT) return SFA_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SFA_ERR_NO_DEVICE;
    uint32_t nr_max = 1;
    for (int32_t i = 0; i < n; ++i) {
        if (!automata[i]) return SFA_ERR_INVALID;
        if (!automata[i]->on_device) return SFA_ERR_HOST_ONLY;
        if (automata[i]->device != dev) return SFA_ERR_INVALID;
        // batch plans hold byte-wide state ids
        if (automata[i]->host.wide) return SFA_ERR_UNSUPPORTED;
        nr_max = std::max<uint32_t>(nr_max, automata[i]->host.nr);
    }
    sfa_server *s = new (std::nothrow) sfa_server;
    if (!s) return SFA_ERR_OOM;
    s->device = dev;
    s->automata.assign(automata, automata + n);
    s->max_batch = max_batch;
    s->timing = (o.flags & SFA_SERVER_TIMING) != 0;
    if (s->timing && (cudaEventCreate(&s->t_origin) != cudaSuccess || cudaEventRecord(s->t_origin, 0) != cudaSuccess ||
                      cudaEventSynchronize(s->t_origin) != cudaSuccess)) {
        cudaGetLastError();
        server_free(s);
        return SFA_ERR_CUDA;
    }
    s->arena = new (std::nothrow) sfa_arena(budget);
    if (!s->arena || cudaMalloc(&s->d_arena, budget) != cudaSuccess) {
        cudaGetLastError();
        server_free(s);
        return SFA_ERR_OOM;
    }
    // a batch's texts all sit in the arena: at most max_batch + budget /
    // (threads * chunk) tiles
    sfa_launch_opts lo{};
    lo.chunk_bytes = chunk;
    lo.block_threads = threads;
    lo.chains = 1;
    const uint64_t max_tiles = (uint64_t)max_batch + budget / ((uint64_t)threads * chunk) + 1;
    s->slots.resize(nslots);
    for (Slot &sl : s->slots) {
        int rc = sfa_batch_reserve(max_batch, max_tiles, nr_max, &lo, &sl.plan);
        if (!rc && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) rc = SFA_ERR_CUDA;
        if (!rc && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) rc = SFA_ERR_CUDA;
        if (!rc && s->timing)
            for (cudaEvent_t *e : {&sl.t_copy, &sl.t_match, &sl.t_end})
                if (!rc && cudaEventCreate(e) != cudaSuccess) rc = SFA_ERR_CUDA;
        if (!rc && cudaMalloc(&sl.d_out, (size_t)max_batch * sizeof(sfa_result)) != cudaSuccess) rc = SFA_ERR_OOM;
        if (!rc && cudaMallocHost(&sl.h_out, (size_t)max_batch * sizeof(sfa_result)) != cudaSuccess)
            rc = SFA_ERR_OOM;
        if (rc) {
            cudaGetLastError();
            server_free(s);
            return rc;
        }
    }
    *out = s;
    return SFA_OK;
}

int sfa_server_submit(sfa_server_t s, int32_t automaton, const uint8_t *h_text, uint64_t len, uint64_t tag) {
    if (!s || automaton < 0 || automaton >= (int32_t)s->automata.size()) return SFA_ERR_INVALID;
    if ((len && !h_text) || len + TEXT_PAD > s->arena->size) return SFA_ERR_INVALID;
    s->queue.push_back(Req{automaton, h_text, len, tag, 0});
    return SFA_OK;
}

int sfa_server_submit_many(sfa_server_t s, int32_t k, const int32_t *automata, const uint8_t *const *h_texts,
                           const uint64_t *lens, const uint64_t *tags) {
    if (!s || k < 0 || (k > 0 && (!automata || !h_texts || !lens || !tags))) return SFA_ERR_INVALID;
    for (int32_t i = 0; i < k; ++i) {   // all or nothing
        if (automata[i] < 0 || automata[i] >= (int32_t)s->automata.size()) return SFA_ERR_INVALID;
        if ((lens[i] && !h_texts[i]) || lens[i] + TEXT_PAD > s->arena->size) return SFA_ERR_INVALID;
    }
    for (int32_t i = 0; i < k; ++i) s->queue.push_back(Req{automata[i], h_texts[i], lens[i], tags[i], 0});
    return SFA_OK;
}

int sfa_server_progress(sfa_server_t s, sfa_completion *done, int32_t cap, int32_t *n_done) {
    if (!s || !n_done || cap < 0 || (cap > 0 && !done)) return SFA_ERR_INVALID;
    *n_done = 0;
    int rc = server_reap(s);
    if (!rc) rc = server_admit(s);
    int32_t k = 0;
    while (k < cap && !s->done.empty()) {
        done[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_done = k;
    return rc;
}

int sfa_server_spans(sfa_server_t s, sfa_batch_span *out, int32_t cap, int32_t *n) {
    if (!s || !n || cap < 0 || (cap > 0 && !out)) return SFA_ERR_INVALID;
    int32_t m = 0;
    while (m < cap && !s->spans.empty()) {
        out[m++] = s->spans.front();
        s->spans.pop_front();
    }
    *n = m;
    return SFA_OK;
}

int sfa_server_stats(sfa_server_t s, sfa_server_stats_t *out) {
    if (!s || !out) return SFA_ERR_INVALID;
    out->queued = s->queue.size();
    uint64_t inflight = 0;
    for (const Slot &sl : s->slots) inflight += sl.reqs.size();
    out->in_flight = inflight;
    out->completed_waiting = s->done.size();
    out->batches = s->batches;
    out->requests = s->requests;
    out->arena_used = s->arena->used;
    return SFA_OK;
}

void sfa_server_destroy(sfa_server_t s) {
    if (s) server_free(s);
}

sfa_arena_t sfa_arena_create(uint64_t size) { return new (std::nothrow) sfa_arena(size); }

int sfa_arena_alloc(sfa_arena_t a, uint64_t n, uint64_t *off) {
    if (!a || !off) return SFA_ERR_INVALID;
    return a->alloc(n, *off) ? SFA_OK : SFA_ERR_OOM;
}

int sfa_arena_release(sfa_arena_t a, uint64_t off, uint64_t n) {
    if (!a) return SFA_ERR_INVALID;
    return a->release(off, n) ? SFA_OK : SFA_ERR_INVALID;
}

uint64_t sfa_arena_used(sfa_arena_t a) { return a ? a->used : 0; }

void sfa_arena_destroy(sfa_arena_t a) { delete a; }

}  // extern "C"
