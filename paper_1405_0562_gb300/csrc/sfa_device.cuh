// Device side of the SFA matcher for sm_103a: one persistent kernel template
// that runs Alg. 5 (parallel computation of a D-SFA) over tiles of chunks,
// combines the chunk mappings with warp / block / grid scans of the reverse
// composition (Lemma 1, Theorem 3) and counts the accepting prefixes.
//
// Vocabulary used below
//   chunk    a contiguous piece of one text, run from f_I by one thread
//   tile     THREADS*CH consecutive chunks, processed by one CTA
//   state id D-SFA state: id c < nr is the constant mapping onto DFA state c
//            (its SFA row is the DFA row of c), id >= nr a non-constant one
//   group    32 consecutive chunks of a tile (one warp, one round)
//
// Text staging: a chunk's 16-byte-aligned body arrives in shared memory by
// asynchronous copies completed on one mbarrier per warp and stage, SLICE
// bytes per chunk per step and STAGES steps in flight: one 2-D tensor copy per
// warp moves the slice of its 32 chunks at once (the text seen as rows of the
// chunk length); chunks that are not full rows use 1-D bulk copies; unaligned
// head and tail bytes are read singly.  The copies bypass the load/store data
// path, which the table lookups need for themselves.
//
// Acceptance bookkeeping (the count): while a chunk runs from f_I its state
// f is known only as a mapping, so for position j the final-ness of
// f(s_in) depends on the still unknown entering state s_in exactly when f is
// "mixed" (final for some kept q, not for others).  Pass 1 counts the
// positions whose mapping is final for every q and remembers the last mixed
// position; once s_in is known, pass 2 reruns the DFA (Alg. 2) from s_in
// over the prefix up to that position.  For synchronising automata (all
// literal automata) that prefix is at most the longest literal.
#pragma once

#include <cuda.h>

#include <cstdint>
#include <type_traits>

#include "sfa.h"
#include "sfa_types.h"

namespace sfa_dev {

// ---------------------------------------------------------------------------
// memory-model, timer and async-copy helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// a self-contained descriptor (an inclusive prefix): its readers read nothing
// else that it would have to order
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// fetch-and-add that orders this thread's earlier writes before it and its
// later reads after it
__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint4 ldg128(const uint8_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_copy(uint32_t dst, const uint8_t *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// 2-D tensor copy of the box at (x, y) of `map` into shared memory, completing
// its bytes (the whole box, out-of-range elements included) on the mbarrier
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// order earlier generic writes of a tensor map in global memory before the
// TMA unit reads it
__device__ __forceinline__ void tensormap_acquire(const void *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for a non-zero descriptor.  Gives up after timeout_us (wall
// clock) or 2^22 polls, or at once when another CTA already gave up; on
// giving up it raises the launch error and returns a PREFIX descriptor so
// that the caller continues (its results are then flagged invalid).
static __device__ __noinline__ uint64_t wait_descriptor(const uint64_t *p, uint32_t *err, uint32_t timeout_us) {
    uint64_t v = ld_acquire(p);
    if (v) return v;
    const uint64_t t0 = globaltimer();
    const uint64_t limit = (uint64_t)timeout_us * 1000ull;
    for (uint32_t it = 1;; ++it) {
        __nanosleep(128);
        v = ld_acquire(p);
        if (v) return v;
        if ((it & 31u) == 0) {
            if (*(volatile uint32_t *)err || globaltimer() - t0 > limit || it > (1u << 22)) {
                atomicOr(err, 1u);
                return ST_PREFIX;
            }
        }
    }
}

// Bounded wait for the completion of an mbarrier phase (a stage of bulk
// copies).  Gives up after timeout_us or 2^24 polls, or soon after another
// wait of the launch gave up; on giving up it raises the launch error and
// returns (the stage's bytes are then not trusted, the results flagged).
static __device__ __noinline__ void wait_stage_slow(uint32_t bar, uint32_t parity, uint32_t *err,
                                                    uint32_t timeout_us) {
    const uint64_t t0 = globaltimer();
    const uint64_t limit = (uint64_t)timeout_us * 1000ull;
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return;
        if ((it & 63u) == 0 &&
            (*(volatile uint32_t *)err || globaltimer() - t0 > limit || it > (1u << 24))) {
            atomicOr(err, 1u);
            return;
        }
    }
}

// After a launch error: before a warp leaves, a bounded wait for the last
// phase of each of its stages (the one a wait may have given up on), so that
// its bulk copies do not land in shared memory after the CTA has exited.
static __device__ __noinline__ void drain_stages(uint32_t bar0, uint32_t parity, int stages, uint32_t timeout_us) {
    const uint64_t limit = (uint64_t)timeout_us * 1000ull;
    for (int st = 0; st < stages; ++st) {
        const uint32_t last = ((parity >> st) & 1u) ^ 1u;
        const uint64_t t0 = globaltimer();
        for (uint32_t it = 1; !mbar_try_wait(bar0 + 8 * st, last); ++it)
            if ((it & 63u) == 0 && (globaltimer() - t0 > limit || it > (1u << 24))) break;
    }
}
__device__ __forceinline__ void wait_stage(uint32_t bar, uint32_t parity, uint32_t *err, uint32_t timeout_us) {
    if (!mbar_try_wait(bar, parity)) wait_stage_slow(bar, parity, err, timeout_us);
}

// ---------------------------------------------------------------------------
// per-chunk state of pass 1
// ---------------------------------------------------------------------------
struct Chain {
    uint32_t f;       // state id
    uint32_t cnt;     // positions whose mapping is final for every kept q
    uint32_t snap;    // cnt at the last mixed position
    int32_t lm;       // offset of the last mixed position, -1 if none
};

// offset of (state q, byte b) in the shared-memory DFA rows
__device__ __forceinline__ uint32_t didx(uint32_t q, uint32_t b) { return q * ROWB + b; }

// DFA-row lookups in shared memory: the transitions of the constant
// mappings, and of the live state of a point mapping.
//   byte ids (up to 256 kept states): one row of all 256 byte columns per
//   state, ROWB bytes apart;
//   16-bit ids (WIDE): one row of ncls 16-bit entries per state, indexed by
//   the byte's class (the class table is in shared memory too).
template <bool WIDE>
struct Rows;
template <>
struct Rows<false> {
    const uint8_t *d;
    __device__ __forceinline__ uint32_t next(uint32_t q, uint32_t b) const { return d[q * ROWB + b]; }
};
template <>
struct Rows<true> {
    const uint16_t *d;
    const uint8_t *cls;
    uint32_t ncls;
    __device__ __forceinline__ uint32_t next(uint32_t q, uint32_t b) const { return d[q * ncls + cls[b]]; }
};

// Fields of a point-mapping entry NC_POINT | s << PT_SHIFT | p: byte ids
// carry 8-bit states, 16-bit ids 12-bit ones.
template <bool WIDE>
struct Pt {
    static constexpr uint32_t SHIFT = WIDE ? 12u : 8u;
    static constexpr uint32_t MASK = (1u << SHIFT) - 1u;
    static constexpr uint32_t KEEP = NC_POINT | NC_SET | ((1u << (2 * SHIFT)) - 1u);   // the flags and both fields
};

// q in the source set sid of a set-point mapping
__device__ __forceinline__ bool in_set(const Tables &T, uint32_t sid, uint32_t q) {
    return (__ldg(T.setbits + (size_t)sid * T.set_words + (q >> 5)) >> (q & 31u)) & 1u;
}

// The point source a chunk keeps for pass 2 (16 bits): its source state s,
// or PS_SET | the id of its source set; 0xffff: none.
template <bool WIDE>
__device__ __forceinline__ uint32_t point_source_of(uint32_t f) {
    const uint32_t fld = (f >> Pt<WIDE>::SHIFT) & Pt<WIDE>::MASK;
    return f & NC_SET ? PS_SET | fld : fld;
}

// one symbol of Alg. 5 in the D-SFA: f <- delta_s[f, sigma].
// Point mappings {s -> p, others -> sink}: f = NC_POINT | s << SHIFT | p, and
// f . delta^sigma = {s -> delta(p, sigma), others -> sink} is one DFA-row
// lookup.  Entering one sets the last mixed position to the entering byte,
// so that pass 2 reruns the DFA up to there; after it cnt counts the final
// p, which are the final positions for the entering state s alone (for any
// other entering state the chunk is in the non-final sink).  A chunk stays a
// point mapping to its end, also once p is the sink (then {s -> sink} is
// the constant sink).
template <bool WIDE>
__device__ __forceinline__ void sfa_step(Chain &s, uint32_t b, int32_t j, const Rows<WIDE> &R,
                                         const uint8_t *s_cls, const uint32_t *nc, uint32_t nr,
                                         uint32_t ncls, uint32_t first_accept) {
    using P = Pt<WIDE>;
    if (s.f & NC_POINT) {
        const uint32_t p = R.next(s.f & P::MASK, b);
        s.cnt += p >= first_accept;
        s.f = (s.f & ~P::MASK) | p;
    } else if (s.f >= nr) {
        const uint32_t e = __ldg(nc + (size_t)(s.f - nr) * ncls + s_cls[b]);
        // the class bits, without divergent branches
        const uint32_t a = e >> 30;
        const bool pt = (e & NC_POINT) != 0u;
        const bool mark = a == ACC_MIXED || pt;
        s.f = e & (pt ? P::KEEP : NC_ID_MASK);
        s.cnt += a == ACC_ALL;
        s.lm = mark ? j : s.lm;
        s.snap = mark ? s.cnt : s.snap;
    } else {
        s.f = R.next(s.f, b);
        s.cnt += s.f >= first_accept;
    }
}

// The count of a chunk entered in state v, from its pass-1 record: the DFA
// rerun over [lo, lo + lm] (rerun: its value, or 0 when it is added later),
// then the positions after lm -- all of them if the chunk never became a
// point mapping, else only for the entering state ps (or a state of the
// source set, PS_SET | sid).
__device__ __forceinline__ uint32_t chunk_count_after(const Chain &c, uint32_t v, uint32_t ps, const Tables &T) {
    const bool live = ps == NO_POINT || (ps & PS_SET ? in_set(T, ps & ~PS_SET, v) : v == ps);
    return live ? c.cnt - c.snap : 0u;
}

// 4 symbols of a constant-state chunk, keeping the largest state seen
template <bool WIDE>
__device__ __forceinline__ void dfa_word_max(uint32_t &q, uint32_t &m, uint32_t w, const Rows<WIDE> &R) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q = R.next(q, __byte_perm(w, 0, 0x4440 | j));
        m = max(m, q);
    }
}

// 4 symbols (one text word) of a constant-state chunk: the DFA row lookups
template <bool WIDE>
__device__ __forceinline__ void dfa_word(uint32_t &q, uint32_t &cnt, uint32_t w, const Rows<WIDE> &R,
                                         uint32_t first_accept) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q = R.next(q, __byte_perm(w, 0, 0x4440 | j));
        cnt += q >= first_accept;
    }
}

// ---------------------------------------------------------------------------
// simulation mode: the |Q|-vector T[q] of Alg. 3.  While T has many distinct
// entries it is kept whole, four states per register (SIM_FULL).  Once at
// most 8 distinct values are left it is kept as those values U[0..7] and, for
// each q, the slot of T[q] among them (SIM_COMPACT): a byte then costs 8
// lookups instead of NQ.  With one value left T is constant (SIM_CONST) and
// the chunk runs on the DFA rows.  The representation is re-examined every
// 16 bytes; the vector it stands for is the same in every form.
// ---------------------------------------------------------------------------
enum : uint32_t { SIM_FULL = 0, SIM_COMPACT = 1, SIM_CONST = 2 };

template <int NQ>
struct SimChain {
    // Vectors of up to 64 entries stay in registers (w); longer ones live in
    // shared memory (ws), word i of this thread at ws[32 * i]: the 32 lanes
    // of a warp touch word i of their own vectors in 32 distinct banks.
    static constexpr bool SMEM = NQ > 64;
    uint32_t w[SMEM ? 1 : NQ / 4];   // SIM_FULL: T[q]; SIM_COMPACT: slot of T[q]
    uint32_t *ws;
    uint32_t u0, u1;      // SIM_COMPACT: U[0..7] (slots past d repeat U[0])
    uint32_t d;           // SIM_COMPACT: number of distinct values
    uint32_t mode;
    __device__ __forceinline__ uint32_t get(int i) const {
        if constexpr (SMEM) return ws[32 * i];
        else return w[i];
    }
    __device__ __forceinline__ void set(int i, uint32_t v) {
        if constexpr (SMEM) ws[32 * i] = v;
        else w[i] = v;
    }
};

// the successors of four packed states on byte b, packed
__device__ __forceinline__ uint32_t step4(uint32_t x, uint32_t b, const uint8_t *s_dfa) {
    const uint32_t y0 = s_dfa[__byte_perm(x, 0, 0x4440) * ROWB + b];
    const uint32_t y1 = s_dfa[__byte_perm(x, 0, 0x4441) * ROWB + b];
    const uint32_t y2 = s_dfa[__byte_perm(x, 0, 0x4442) * ROWB + b];
    const uint32_t y3 = s_dfa[__byte_perm(x, 0, 0x4443) * ROWB + b];
    return __byte_perm(__byte_perm(y0, y1, 0x0040), __byte_perm(y2, y3, 0x0040), 0x5410);
}

// final for all, some or none of the entries, from packed minima and maxima
__device__ __forceinline__ void acc_update(Chain &s, uint32_t mn, uint32_t mx, int32_t j, uint32_t first_accept) {
    mn = __vminu4(mn, mn >> 16);
    mn = __vminu4(mn, mn >> 8) & 0xffu;
    mx = __vmaxu4(mx, mx >> 16);
    mx = __vmaxu4(mx, mx >> 8) & 0xffu;
    if (mn >= first_accept) {
        s.cnt++;
    } else if (mx >= first_accept) {
        s.lm = j;
        s.snap = s.cnt;
    }
}

template <int NQ>
__device__ __forceinline__ void sim_byte(SimChain<NQ> &T, Chain &s, uint32_t b, int32_t j, const uint8_t *s_dfa,
                                         uint32_t first_accept) {
    if (T.mode == SIM_CONST) {
        s.f = s_dfa[didx(s.f, b)];
        s.cnt += s.f >= first_accept;
        return;
    }
    uint32_t mn, mx;
    if (T.mode == SIM_FULL) {
        mn = 0xffffffffu;
        mx = 0;
        if constexpr (SimChain<NQ>::SMEM) {
#pragma unroll 4
            for (int i = 0; i < NQ / 4; ++i) {
                const uint32_t y = step4(T.ws[32 * i], b, s_dfa);
                T.ws[32 * i] = y;
                mn = __vminu4(mn, y);
                mx = __vmaxu4(mx, y);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NQ / 4; ++i) {
                const uint32_t y = step4(T.w[i], b, s_dfa);
                T.w[i] = y;
                mn = __vminu4(mn, y);
                mx = __vmaxu4(mx, y);
            }
        }
    } else {
        T.u0 = step4(T.u0, b, s_dfa);
        T.u1 = step4(T.u1, b, s_dfa);
        mn = __vminu4(T.u0, T.u1);
        mx = __vmaxu4(T.u0, T.u1);
    }
    acc_update(s, mn, mx, j, first_accept);
}

// The set of distinct values of a chunk vector (state ids < NQ), as a bit
// mask of NQ bits in 64-bit words.  Register arrays are only indexed by
// compile-time constants (a value's word is selected, not addressed), so the
// mask stays in registers for every NQ.
template <int NQ>
struct VSet {
    static constexpr int W = NQ <= 64 ? 1 : NQ / 64;
    uint64_t m[W];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int w = 0; w < W; ++w) m[w] = 0;
    }
    __device__ __forceinline__ void add(uint32_t v) {
        if (W == 1) {
            m[0] |= 1ull << v;
        } else {
            const uint64_t bit = 1ull << (v & 63u);
#pragma unroll
            for (int w = 0; w < W; ++w) m[w] |= (v >> 6) == (uint32_t)w ? bit : 0ull;
        }
    }
    __device__ __forceinline__ int count() const {
        int c = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) c += __popcll(m[w]);
        return c;
    }
    // number of values in the set below v
    __device__ __forceinline__ uint32_t rank(uint32_t v) const {
        if (W == 1) return (uint32_t)__popcll(m[0] & ((1ull << v) - 1ull));
        const uint32_t wv = v >> 6;
        const uint64_t below = (1ull << (v & 63u)) - 1ull;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < W; ++w)
            r += (uint32_t)w < wv ? (uint32_t)__popcll(m[w]) : ((uint32_t)w == wv ? (uint32_t)__popcll(m[w] & below) : 0u);
        return r;
    }
    // the smallest value (the set is not empty)
    __device__ __forceinline__ uint32_t first() const {
        uint32_t v = 0xffffffffu;
#pragma unroll
        for (int w = W - 1; w >= 0; --w)
            if (m[w]) v = 64u * w + (uint32_t)__ffsll((long long)m[w]) - 1u;
        return v;
    }
    // the (at most 8) values in ascending order, four per word, padded with
    // the first
    __device__ __forceinline__ void values8(uint32_t &u0, uint32_t &u1) const {
        uint64_t mm[W];
#pragma unroll
        for (int w = 0; w < W; ++w) mm[w] = m[w];
        const uint32_t f = first();
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t x = 0xffffffffu;
#pragma unroll
            for (int w = 0; w < W; ++w)
                if (x == 0xffffffffu && mm[w]) {
                    x = 64u * w + (uint32_t)__ffsll((long long)mm[w]) - 1u;
                    mm[w] &= mm[w] - 1ull;
                }
            v[k] = x == 0xffffffffu ? f : x;
        }
        u0 = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
        u1 = v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24);
    }
    // the ranks of the four values packed in x, packed
    __device__ __forceinline__ uint32_t rank4(uint32_t x) const {
        return rank(x & 0xffu) | (rank((x >> 8) & 0xffu) << 8) | (rank((x >> 16) & 0xffu) << 16) |
               (rank(x >> 24) << 24);
    }
};

// selector of __byte_perm that picks U[slot] for the four slots of a word
__device__ __forceinline__ uint32_t slots_sel(uint32_t x) {
    return (x & 0x7u) | ((x >> 4) & 0x70u) | ((x >> 8) & 0x700u) | ((x >> 12) & 0x7000u);
}

// re-examine the representation (every 16 bytes)
template <int NQ>
__device__ __forceinline__ void sim_compact(SimChain<NQ> &T, Chain &s) {
    if (T.mode == SIM_FULL) {
        VSet<NQ> m;
        m.clear();
        if constexpr (SimChain<NQ>::SMEM) {
#pragma unroll 4
            for (int i = 0; i < NQ / 4; ++i) {
                const uint32_t x = T.ws[32 * i];
#pragma unroll
                for (int k = 0; k < 4; ++k) m.add((x >> (8 * k)) & 0xffu);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NQ / 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) m.add((T.w[i] >> (8 * k)) & 0xffu);
        }
        const int dd = m.count();
        if (dd == 1) {
            T.mode = SIM_CONST;
            s.f = m.first();
            return;
        }
        if (dd > 8) return;
        if constexpr (SimChain<NQ>::SMEM) {
#pragma unroll 4
            for (int i = 0; i < NQ / 4; ++i) T.ws[32 * i] = m.rank4(T.ws[32 * i]);
        } else {
#pragma unroll
            for (int i = 0; i < NQ / 4; ++i) T.w[i] = m.rank4(T.w[i]);
        }
        m.values8(T.u0, T.u1);
        T.d = (uint32_t)dd;
        T.mode = SIM_COMPACT;
    } else if (T.mode == SIM_COMPACT) {
        VSet<NQ> m;
        m.clear();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            m.add((T.u0 >> (8 * k)) & 0xffu);
            m.add((T.u1 >> (8 * k)) & 0xffu);
        }
        const int dd = m.count();
        if (dd == 1) {
            T.mode = SIM_CONST;
            s.f = T.u0 & 0xffu;
            return;
        }
        if ((uint32_t)dd == T.d) return;
        // old slot k moves to the rank of U[k] among the values left
        const uint32_t n0 = m.rank4(T.u0), n1 = m.rank4(T.u1);
        if constexpr (SimChain<NQ>::SMEM) {
#pragma unroll 4
            for (int i = 0; i < NQ / 4; ++i) T.ws[32 * i] = __byte_perm(n0, n1, slots_sel(T.ws[32 * i]));
        } else {
#pragma unroll
            for (int i = 0; i < NQ / 4; ++i) T.w[i] = __byte_perm(n0, n1, slots_sel(T.w[i]));
        }
        m.values8(T.u0, T.u1);
        T.d = (uint32_t)dd;
    }
}

// the four entries T[4i..4i+3] of a non-constant chain
template <int NQ>
__device__ __forceinline__ uint32_t sim_word(const SimChain<NQ> &T, int i) {
    const uint32_t x = T.get(i);
    return T.mode == SIM_FULL ? x : __byte_perm(T.u0, T.u1, slots_sel(x));
}

// mapping applied to a state: constant ids are their own value
__device__ __forceinline__ uint32_t apply_map(uint32_t f, uint32_t v, const uint8_t *mtab, uint32_t nr) {
    return f < nr ? f : (uint32_t)mtab[(size_t)(f - nr) * nr + v];
}
// 16-bit ids: a chunk may also end as a point mapping {s -> p, others ->
// sink} or a set-point mapping {S -> p, others -> sink}, kept in its encoded
// form (neither is stored)
__device__ __forceinline__ uint32_t apply_map(uint32_t f, uint32_t v, const uint16_t *mtab, uint32_t nr,
                                              uint32_t sink, const Tables &T) {
    if (f < nr) return f;
    if (f & NC_POINT) {
        const uint32_t fld = (f >> Pt<true>::SHIFT) & Pt<true>::MASK;
        const bool live = f & NC_SET ? in_set(T, fld, v) : v == fld;
        return live ? (f & Pt<true>::MASK) : sink;
    }
    return mtab[(size_t)(f - nr) * nr + v];
}

// Alg. 2 from state q over [p, e) of the text, counting final states
template <bool WIDE>
__device__ __forceinline__ uint32_t dfa_count(const uint8_t *text, uint64_t p, uint64_t e, uint32_t q,
                                              const Rows<WIDE> &R, uint32_t first_accept) {
    uint32_t c = 0;
    while (p < e && (reinterpret_cast<uintptr_t>(text + p) & 15)) {
        q = R.next(q, text[p]);
        c += q >= first_accept;
        ++p;
    }
    // 16-byte words, the next two loaded while the current two are counted
    // (a long rerun reads its text from HBM)
    auto word16 = [&](const uint4 &v) {
        dfa_word<WIDE>(q, c, v.x, R, first_accept);
        dfa_word<WIDE>(q, c, v.y, R, first_accept);
        dfa_word<WIDE>(q, c, v.z, R, first_accept);
        dfa_word<WIDE>(q, c, v.w, R, first_accept);
    };
    if (p + 32 <= e) {
        uint4 v0 = ldg128(text + p), v1 = ldg128(text + p + 16);
        for (; p + 64 <= e; p += 32) {
            const uint4 n0 = ldg128(text + p + 32), n1 = ldg128(text + p + 48);
            word16(v0);
            word16(v1);
            v0 = n0;
            v1 = n1;
        }
        word16(v0);
        word16(v1);
        p += 32;
    }
    for (; p + 16 <= e; p += 16) word16(ldg128(text + p));
    for (; p < e; ++p) {
        q = R.next(q, text[p]);
        c += q >= first_accept;
    }
    return c;
}

// ---------------------------------------------------------------------------
// tile bookkeeping shared by CTA tiles and warp tiles (run by one thread)
// ---------------------------------------------------------------------------
// The entering state of tile gt of a text: the start state q0 for its first
// tile (with carry: the previous call's final state, Lemma 1), else the
// decoupled look-back: walk back to the nearest inclusive prefix, then apply
// the aggregates in between in order.
template <bool WIDE = false>
__device__ __forceinline__ uint32_t tile_entering_state(const Scratch &S, const Tables &T, const TextDesc &d,
                                                        const sfa_result *out, TextState *ts, uint32_t gt,
                                                        uint32_t local, uint32_t nr, uint32_t nr_max) {
    using SID = typename std::conditional<WIDE, uint16_t, uint8_t>::type;
    if (local == 0) {
        if (!d.carry) return T.q0;
        const sfa_result prev = out[d.out_index];
        if (prev.status || prev.final_state >= T.nq_in || T.kept_of[prev.final_state] < 0) {
            atomicOr(&ts->err, 1u);
            return T.q0;
        }
        return (uint32_t)T.kept_of[prev.final_state];
    }
    const uint32_t base = d.tile_base;
    uint32_t j = gt - 1;
    uint64_t w;
    for (;;) {
        w = wait_descriptor(S.status + j, &S.hdr->err, S.timeout_us);
        if ((w >> 62) == 2u || j == base) break;
        --j;
    }
    uint32_t v = (uint32_t)(w & 0xffffffffu);
    if ((w >> 62) != 2u) v = T.q0;   // unreachable: tile 0 of a text always publishes a prefix
    if (v >= nr) v = 0;              // only after a timeout
    for (uint32_t i = j + 1; i < gt; ++i) {
        const uint64_t wi = ld_acquire(S.status + i);
        if ((wi >> 62) == 2u) {
            v = (uint32_t)(wi & 0xffffffffu);
            if (v >= nr) v = 0;
        } else {
            v = reinterpret_cast<const SID *>(S.agg)[(size_t)i * nr_max + v];
        }
    }
    return v;
}

// Part of a tile's count (and the final state if it is the text's last
// tile), for a text of several tiles.
__device__ __forceinline__ void add_tile_count(const TextDesc &d, TextState *ts, unsigned long long sum,
                                               uint32_t local, uint32_t incl) {
    if (sum) atomicAdd(&ts->count, sum);
    if (local == d.ntiles - 1) ts->final_state = incl;
}

// A tile is done: add its count, record the final state if it is the text's
// last tile, and let the last tile of the text to finish write the result.
// A text of one tile writes it at once.  counted: the count and final state
// were added already (add_tile_count).
__device__ __forceinline__ void finish_tile(const Scratch &S, const Tables &T, const TextDesc &d, TextState *ts,
                                            sfa_result *out, unsigned long long sum, uint32_t local, uint32_t incl,
                                            bool counted = false) {
    unsigned long long total = sum;
    uint32_t fin = incl;
    if (d.ntiles > 1) {
        if (!counted) add_tile_count(d, ts, sum, local, incl);
        // release: this tile's count and final state before its `done`;
        // acquire: every other tile's before the reads of the last one
        const uint32_t prev = atomic_add_acq_rel(&ts->done, 1u);
        if (prev != d.ntiles - 1) return;
        total = atomicAdd(&ts->count, 0ull);
        fin = *(volatile uint32_t *)&ts->final_state;
    }
    const uint32_t err = *(volatile uint32_t *)&ts->err | *(volatile uint32_t *)&S.hdr->err;
    sfa_result r;
    r.final_state = (uint32_t)T.orig_of[fin < T.nr ? fin : 0];
    r.accept_final = fin >= T.first_accept ? 1 : 0;
    r.status = err ? SFA_STATUS_TIMEOUT : SFA_STATUS_OK;
    r.reserved = 0;
    r.count = (d.carry ? out[d.out_index].count : 0ull) + total;
    out[d.out_index] = r;
}

// A tile whose count still lacks the recount of its first chunk over
// [lo, lo + lm] from the tile's entering state (a constant tile whose first
// chunk is constant: nothing else depends on the entering state).  Resolved
// by the CTA after its next tile has streamed, when the look-back no longer
// waits; the recount reads the DFA rows in global memory (the shared copy may
// hold another automaton by then).
// (kept by thread 0 in the CTA's Misc record)
template <bool BATCH>
__device__ __noinline__ void resolve_deferred(Misc *m, const Scratch &S, const Tables &tab, const TextDesc &desc,
                                              const Tables *tabs, const TextDesc *descs, sfa_result *out) {
    const uint32_t gt = m->dfr_gt, ti = m->dfr_ti;
    const TextDesc d = BATCH ? descs[ti] : desc;
    const Tables T = BATCH ? tabs[d.table] : tab;
    TextState *ts = S.texts + (BATCH ? ti : 0u);
    const uint32_t local = gt - d.tile_base;
    uint32_t q = tile_entering_state(S, T, d, out, ts, gt, local, T.nr, S.nr_max);
    unsigned long long c = 0;
    const uint64_t lo = m->dfr_lo, e = lo + (uint64_t)m->dfr_lm;
    for (uint64_t p = lo; p <= e; ++p) {
        q = __ldg(T.dfa + (size_t)q * 256 + d.text[p]);
        c += q >= T.first_accept;
    }
    if (c) atomicAdd(&ts->count, c);
    finish_tile(S, T, d, ts, out, 0ull, local, 0u, true);
    m->dfr_valid = 0;
}

// ---------------------------------------------------------------------------
// the persistent kernel
//   SIMNQ = 0: D-SFA mode; SIMNQ = 16/32/64/128/256: simulation mode with
//   vectors of that many entries (the kept states, padded)
//   BATCH: tables and texts come from device arrays, else from `tab`/`desc`
//   WT: warp tiles.  Every warp takes its own tiles of 32 chunks, publishes
//   its own look-back descriptor and finishes its own tiles, with no CTA
//   barrier after the tables are staged: a warp's scan and look-back overlap
//   the other warps' lookups, and slower warps take fewer tiles.  One text,
//   one chunk per thread.  Without WT a tile is the CTA's THREADS * CH chunks.
// ---------------------------------------------------------------------------
// CTAs per SM asked of the register allocator (0: none asked): the batch
// instances with one chunk per thread must run 1024 threads per SM (two CTAs
// of 512, ...), which their allocator does not choose by itself; the others
// are left to it (a bound there measured 4 % slower on the single-text kernel
// at the same register count)
template <int THREADS, int CH, int SIMNQ, bool BATCH>
constexpr int min_ctas_per_sm() {
    return BATCH && SIMNQ == 0 && CH == 1 && THREADS <= 1024 ? 1024 / THREADS : 0;
}

//   WIDE: 16-bit state ids (more than 256 kept states): class-indexed DFA
//   rows, point mappings never stored (kept encoded to the chunk's end).
//   Single texts, CTA tiles, D-SFA mode.
template <int THREADS, int CH, int SIMNQ, bool BATCH, bool WT = false, bool WIDE = false>
__global__ void __launch_bounds__(THREADS, (min_ctas_per_sm<THREADS, CH, SIMNQ, BATCH>()))
    sfa_match_kernel(Tables tab, TextDesc desc, const __grid_constant__ CUtensorMap tmap,
                     const __grid_constant__ CUtensorMap tmap_b, const Tables *tabs, const TextDesc *descs,
                     const uint32_t *tile_text, Scratch S, sfa_result *out) {
    using L = SmemLayout<THREADS, CH, SIMNQ, WIDE>;
    using SID = typename std::conditional<WIDE, uint16_t, uint8_t>::type;   // a state in a vector
    using P = Pt<WIDE>;
    constexpr int CPT = L::CPT, NW = L::NW, G = L::G;
    static_assert(!WT || (!BATCH && CH == 1), "warp tiles: one text, one chunk per thread");
    static_assert(!WIDE || (!WT && !BATCH && SIMNQ == 0), "16-bit ids: single texts, CTA tiles, D-SFA mode");
    constexpr int NQ = SIMNQ > 0 ? SIMNQ : 4;
    constexpr uint32_t NO_PT = 0xffffu;   // "no point source" in the extra rows
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t nr_max = S.nr_max;
    const uint32_t lcls = WIDE ? tab.ncls : 0u;   // class count of the layout (16-bit ids)
    uint8_t *s_dfa = smem + L::dfa_off();
    uint8_t *s_cls = smem + L::cls_off(nr_max, lcls);
    uint32_t *s_f = reinterpret_cast<uint32_t *>(smem + L::f_off(nr_max, lcls));
    uint32_t *s_gval = reinterpret_cast<uint32_t *>(smem + L::gval_off(nr_max, lcls));
    uint32_t *s_gpre = reinterpret_cast<uint32_t *>(smem + L::gpre_off(nr_max, lcls));
    Misc *s_misc = reinterpret_cast<Misc *>(smem + L::misc_off(nr_max, lcls));
    SID *s_gvec = reinterpret_cast<SID *>(smem + L::gvec_off(nr_max, lcls));
    Rows<WIDE> R;
    if constexpr (WIDE) {
        R.d = reinterpret_cast<const uint16_t *>(s_dfa);
        R.cls = s_cls;
        R.ncls = tab.ncls;
    } else {
        R.d = s_dfa;
    }

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    // this warp's stage barriers and staging buffers
    const uint32_t bar0 = smem_addr(smem + L::bar_off(nr_max, lcls)) + (uint32_t)warp * STAGES * 8;
    uint8_t *s_box = smem + L::stage_off(nr_max, lcls) + (size_t)warp * STAGES * CH * BOX;
    uint8_t *s_extra = smem + L::extra_off(nr_max, lcls) + (size_t)warp * STAGES * CH * SLICE;
    uint16_t *s_psrc = reinterpret_cast<uint16_t *>(s_extra);   // point sources after pass 1 ([round][lane])
    // the point source of this lane's chunk of round c (after pass 1)
    auto point_src = [&](int c) -> uint32_t {
        const uint32_t v = s_psrc[c * 32 + lane];
        return v == NO_PT ? NO_POINT : v;
    };
    if (lane == 0)
        for (int s = 0; s < STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
    mbar_init_fence();
    __syncwarp();
    uint32_t parity = 0;             // bit s: phase parity expected next on stage s (warp-uniform)
    uint32_t loaded = 0xffffffffu;   // table index in shared memory (CTA-uniform)
    // stage the DFA rows (ROWB apart) and the class table; all threads
    auto stage_tables = [&](const Tables &T, uint32_t idx) {
        if constexpr (WIDE) {
            const uint16_t *src = T.cdfa;
            uint16_t *dst = reinterpret_cast<uint16_t *>(s_dfa);
            for (uint32_t i = tid; i < T.nr * T.ncls; i += THREADS) dst[i] = __ldg(src + i);
        } else {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(T.dfa);
            for (uint32_t i = tid; i < T.nr * 64; i += THREADS)
                *reinterpret_cast<uint32_t *>(s_dfa + (i >> 6) * ROWB + (i & 63) * 4) = __ldg(src + i);
        }
        if (tid < 16) reinterpret_cast<uint4 *>(s_cls)[tid] = __ldg(reinterpret_cast<const uint4 *>(T.cls) + tid);
        loaded = idx;
        __syncthreads();
    };

    // Two levels: the first CTA to start on an SM takes level-A tiles, later
    // ones level-B tiles (the older CTA of an SM runs faster, so its tiles
    // are longer); each moves to the other level once its own runs out.
    const bool two_levels = !BATCH && !WT && desc.split_tile != 0;
    uint32_t slot = 0;   // thread 0: CTAs that started on this SM before this one
    if (two_levels && tid == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        slot = atomicAdd(&S.hdr->sm_slot[smid & 255u], 1u);
    }
    // deferred first-chunk recounts: batches (a CTA takes many tiles there;
    // single texts take one tile per CTA with automatic chunks)
    constexpr bool DEFER = BATCH && !WT;
    if (tid == 0) s_misc->dfr_valid = 0;
    if (!BATCH && S.single && tid == 0) {
        // the only CTA of the launch: nothing else reads these before the
        // barrier that follows the first grab
        S.hdr->err = 0;
        S.texts[0].err = 0;
    }
    auto grab = [&]() -> uint32_t {
        if (!two_levels) return atomicAdd(&S.hdr->tile_ctr, 1u);
        const uint32_t na = desc.split_tile, all = S.total_tiles;
        uint32_t t;
        if (slot == 0) {
            t = atomicAdd(&S.hdr->tile_ctr, 1u);
            if (t >= na) t = na + atomicAdd(&S.hdr->tile_ctr_b, 1u);
        } else {
            t = na + atomicAdd(&S.hdr->tile_ctr_b, 1u);
            if (t >= all) {
                t = atomicAdd(&S.hdr->tile_ctr, 1u);
                if (t >= na) t = all;
            }
        }
        return t;
    };

    for (;;) {
        uint32_t gt = 0;
        if constexpr (WT) {
            if (lane == 0) gt = atomicAdd(&S.hdr->tile_ctr, 1u);
            gt = __shfl_sync(0xffffffffu, gt, 0);
        } else {
            if (tid == 0) {
                s_misc->tile = !BATCH && S.single ? 0u : grab();
                s_misc->gconst = 0;
            }
            __syncthreads();
            gt = s_misc->tile;
        }
        // a batch reads its tile count from the work list (tile_text[0]), so a
        // plan can be refilled without changing its launch
        const uint32_t total = BATCH ? __ldg(tile_text) : S.total_tiles;
        if (gt >= total) {
            // warp tiles: a warp without a first tile still takes its part in
            // staging the tables (the one CTA barrier of the launch)
            if (WT && loaded != 0u) stage_tables(tab, 0u);
            if (DEFER && tid == 0 && s_misc->dfr_valid) resolve_deferred<BATCH>(s_misc, S, tab, desc, tabs, descs, out);
            if (*(volatile uint32_t *)&S.hdr->err) drain_stages(bar0, parity, STAGES, S.timeout_us);
            break;
        }

        uint32_t ti = 0;
        if (BATCH) {
            gt = __ldg(tile_text + 1 + gt);           // grab position -> tile id
            ti = __ldg(tile_text + 1 + total + gt);   // tile id -> text
        }
        const TextDesc d = BATCH ? descs[ti] : desc;
        const Tables T = BATCH ? tabs[d.table] : tab;
        const uint32_t tabidx = BATCH ? d.table : 0u;
        const uint32_t nr = T.nr, A = T.first_accept;
        const uint32_t local = gt - d.tile_base;
        // the tile's level: its byte range [lbase, lend), chunk length, tile
        // index within the level and full chunks of the level's tensor map
        const bool lvb = d.split_tile != 0 && local >= d.split_tile;
        const uint32_t lt = lvb ? local - d.split_tile : local;
        const uint64_t lbase = lvb ? d.split : 0;
        const uint64_t lend = d.split_tile != 0 && !lvb ? d.split : d.n;
        const uint64_t lchunk = lvb ? d.chunk_b : d.chunk;
        const uint32_t lrows = lvb ? d.rows2d_b : d.rows2d;
        // level A's origin (level B starts on a 16-byte boundary)
        const uint64_t org = lvb ? 0 : d.origin;
        uint64_t nch = d.forced ? d.forced : (lend - lbase > org ? (lend - lbase - org + lchunk - 1) / lchunk : 1);
        if (nch == 0) nch = 1;   // the empty text: one empty chunk
        TextState *ts = S.texts + (BATCH ? ti : 0u);
        const uint8_t *text = d.text;
        // the text's tensor map: the kernel parameter, or (batches) a map in
        // device memory written before the launch, acquired for the TMA unit
        const CUtensorMap *tmap_p = lvb ? &tmap_b : (d.map ? reinterpret_cast<const CUtensorMap *>(d.map) : &tmap);
        if (BATCH && d.map && d.rows2d && lane == 0) tensormap_acquire(d.map);
        const uint8_t *mtab = SIMNQ ? S.chainvec : T.maps;
        // simulation chunk vectors: nr_max bytes apart (one text: nr_max = nr;
        // a batch mixes automata of different sizes)
        const uint32_t vstride = BATCH ? nr_max : nr;
        // a chunk or group mapping applied to a state
        auto amap = [&](uint32_t f, uint32_t v) -> uint32_t {
            if constexpr (WIDE)
                return apply_map(f, v, T.maps16, nr, T.sink, T);
            else if constexpr (SIMNQ > 0 && BATCH)
                return f < nr ? f : (uint32_t)mtab[(size_t)(f - nr) * vstride + v];
            else
                return apply_map(f, v, mtab, nr);
        };
        const uintptr_t tbase = reinterpret_cast<uintptr_t>(text);
        // index within the level of this thread's chunk c, and of the first
        // chunk of the warp's 32 in that round
        auto kidx = [&](int c) -> uint64_t {
            return WT ? (uint64_t)lt * 32 + lane : (uint64_t)lt * CPT + (uint64_t)c * THREADS + tid;
        };
        auto krow0 = [&](int c) -> uint32_t { return WT ? lt * 32u : lt * CPT + c * THREADS + warp * 32; };

        // ---------------- pass 1: every chunk from f_I ----------------
        Chain ch[CH];
        SimChain<NQ> V[CH];          // simulation: the chunk's vector T
        uint64_t lo[CH], hi[CH], ba[CH], bb[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const uint64_t k = kidx(c);
            if (k >= nch) {
                lo[c] = hi[c] = lend;
            } else if (d.forced) {
                lo[c] = k * d.n / d.forced;
                hi[c] = (k + 1) * d.n / d.forced;
            } else {
                lo[c] = k == 0 ? lbase : lbase + org + k * lchunk;
                const uint64_t e = lbase + org + (k + 1) * lchunk;
                hi[c] = e < lend ? e : lend;
            }
            // body: the 16-byte-aligned addresses inside [lo, hi) (empty when
            // there are none: b wraps around when hi < 16 and the boundary
            // below text + hi lies before the text)
            const uint64_t a = (((tbase + lo[c]) + 15) & ~(uintptr_t)15) - tbase;
            const uint64_t b = ((tbase + hi[c]) & ~(uintptr_t)15) - tbase;
            ba[c] = a < hi[c] ? a : hi[c];
            bb[c] = b > ba[c] && b <= hi[c] ? b : ba[c];
            ch[c].f = T.ident;
            ch[c].cnt = 0;
            ch[c].snap = 0;
            ch[c].lm = -1;
            if (SIMNQ) {
                // T = f_I over the kept states; padding entries follow state 0
                if constexpr (SimChain<NQ>::SMEM)
                    V[c].ws = reinterpret_cast<uint32_t *>(smem + L::vec_off(nr_max)) +
                              ((size_t)(c * NW + warp) * (NQ / 4)) * 32 + lane;
#pragma unroll 4
                for (int i = 0; i < NQ / 4; ++i) {
                    uint32_t w = 0;
#pragma unroll
                    for (int b4 = 0; b4 < 4; ++b4) {
                        const uint32_t q = 4 * i + b4;
                        w |= (q < nr ? q : 0u) << (8 * b4);
                    }
                    V[c].set(i, w);
                }
                V[c].u0 = V[c].u1 = 0;
                V[c].d = 0;
                V[c].mode = nr == 1 ? SIM_CONST : SIM_FULL;
                if (nr == 1) ch[c].f = 0;
            }
        }

        // one symbol of either mode
        auto step = [&](int c, uint32_t b, int32_t j) {
            if (SIMNQ)
                sim_byte<NQ>(V[c], ch[c], b, j, s_dfa, A);
            else
                sfa_step<WIDE>(ch[c], b, j, R, s_cls, T.nc, nr, T.ncls, A);
        };
        auto constant = [&](int c) -> bool { return SIMNQ ? V[c].mode == SIM_CONST : ch[c].f < nr; };

        // body: slices through shared memory
        bool reg2d[CH];          // this lane's chunk is a row of the tensor map
        bool direct[CH];         // count every byte (see the fast path)
        uint32_t reps[CH];       // recounted 16-byte groups
        uint32_t nsl_c[CH], blen[CH], boxw = 0;
        uint32_t nsl = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const uint64_t k = kidx(c);
            reg2d[c] = k < lrows;
            direct[c] = false;
            reps[c] = 0;
            if (__ballot_sync(0xffffffffu, reg2d[c])) boxw |= 1u << c;
            blen[c] = (uint32_t)(bb[c] - ba[c]);   // < 2^31: one chunk
            nsl_c[c] = (blen[c] + SLICE - 1) / SLICE;
            nsl = nsl_c[c] > nsl ? nsl_c[c] : nsl;
        }
        // bytes of slice s of chunk c inside the body
        auto slice_len = [&](int c, uint32_t s) -> uint32_t {
            return s < nsl_c[c] ? min((uint32_t)SLICE, blen[c] - s * SLICE) : 0u;
        };
        nsl = __reduce_max_sync(0xffffffffu, nsl);
        const uint32_t nsl_box = (uint32_t)((lchunk + SLICE - 1) / SLICE);
        // staging addresses: box of (stage, round), this lane's 1-D row, and
        // the 16-byte unit g of this lane's slice
        auto box_at = [&](uint32_t st, int c) -> uint8_t * {
            return s_box + ((size_t)(st * CH + c)) * BOX;
        };
        auto row1d = [&](uint32_t st, int c) -> uint8_t * {
            return lrows ? s_extra + (size_t)(st * CH + c) * SLICE : box_at(st, c) + lane * SLICE;
        };
        auto unit = [&](uint32_t st, int c, uint32_t g) -> const uint4 * {
            const uint8_t *p = reg2d[c] ? box_at(st, c) + lane * SLICE + ((g ^ ((uint32_t)(lane >> 1) & 3u)) << 4)
                                        : row1d(st, c) + (g << 4);
            return reinterpret_cast<const uint4 *>(p);
        };
        auto issue = [&](uint32_t s) {
            const uint32_t st = s % STAGES;
            uint32_t sz[CH], tot = 0;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                sz[c] = reg2d[c] ? 0u : slice_len(c, s);
                tot += sz[c];
            }
            tot = __reduce_add_sync(0xffffffffu, tot);
            const bool boxes = s < nsl_box;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (boxes && (boxw >> c) & 1u) tot += BOX;
            if (lane == 0) mbar_arrive_expect_tx(bar0 + 8 * st, tot);
            __syncwarp();
            fence_proxy_async_smem();
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (boxes && ((boxw >> c) & 1u) && lane == 0) {
                    const uint32_t row0 = krow0(c);
                    tma_load_2d(smem_addr(box_at(st, c)), tmap_p, (int)(s * SLICE), (int)row0, bar0 + 8 * st);
                }
                if (sz[c]) bulk_copy(smem_addr(row1d(st, c)), text + ba[c] + (uint64_t)s * SLICE, sz[c], bar0 + 8 * st);
            }
        };
        // the first slices are in flight while the previous tile's deferred
        // recount is resolved and the tables are staged
        for (uint32_t s = 0; s < (uint32_t)STAGES && s < nsl; ++s) issue(s);
        if (DEFER && tid == 0 && s_misc->dfr_valid) resolve_deferred<BATCH>(s_misc, S, tab, desc, tabs, descs, out);
        // (warp tiles: every warp comes here once, in its first tile, or in
        // the exit branch above)
        if (tabidx != loaded) stage_tables(T, tabidx);

        // head bytes
#pragma unroll
        for (int c = 0; c < CH; ++c)
            for (uint64_t p = lo[c]; p < ba[c]; ++p) step(c, text[p], (int32_t)(p - lo[c]));

        for (uint32_t s = 0; s < nsl; ++s) {
            const uint32_t st = s % STAGES;
            wait_stage(bar0 + 8 * st, (parity >> st) & 1u, &S.hdr->err, S.timeout_us);
            parity ^= 1u << st;
            uint32_t len[CH];
            bool allc = true;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                len[c] = slice_len(c, s);
                allc &= constant(c) || len[c] == 0;
            }
            if (allc) {
                // fast path: every chunk of the thread is a constant mapping
                // (a DFA state); one row lookup per byte, chunks interleaved.
                // Per 16 bytes only the largest state is tracked; final
                // states are the ids >= A, so a group with no final state is
                // counted as 0 at once and the rare others are recounted
                // exactly from the group's first state.  A chunk that needs
                // the recount often counts every byte instead.
                auto group = [&](int g, bool guard) {
                    uint4 v[CH];
#pragma unroll
                    for (int c = 0; c < CH; ++c) v[c] = *unit(st, c, g);
                    uint32_t q[CH], m[CH];
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        q[c] = ch[c].f;
                        m[c] = 0;
                    }
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (!guard || (uint32_t)(16 * g) < len[c]) {
                            if (direct[c]) {
                                dfa_word<WIDE>(q[c], ch[c].cnt, v[c].x, R, A);
                                dfa_word<WIDE>(q[c], ch[c].cnt, v[c].y, R, A);
                                dfa_word<WIDE>(q[c], ch[c].cnt, v[c].z, R, A);
                                dfa_word<WIDE>(q[c], ch[c].cnt, v[c].w, R, A);
                            } else {
                                dfa_word_max<WIDE>(q[c], m[c], v[c].x, R);
                                dfa_word_max<WIDE>(q[c], m[c], v[c].y, R);
                                dfa_word_max<WIDE>(q[c], m[c], v[c].z, R);
                                dfa_word_max<WIDE>(q[c], m[c], v[c].w, R);
                                if (m[c] >= A) {
                                    uint32_t qq = ch[c].f;
                                    dfa_word<WIDE>(qq, ch[c].cnt, v[c].x, R, A);
                                    dfa_word<WIDE>(qq, ch[c].cnt, v[c].y, R, A);
                                    dfa_word<WIDE>(qq, ch[c].cnt, v[c].z, R, A);
                                    dfa_word<WIDE>(qq, ch[c].cnt, v[c].w, R, A);
                                    ++reps[c];
                                }
                            }
                            ch[c].f = q[c];
                        }
                };
                // full slices and no chunk counting every byte: the CH chains
                // advance byte by byte in one block, so that their lookups
                // overlap
                auto group_fast = [&](int g) {
                    uint4 v[CH];
                    uint32_t q[CH], m[CH];
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        v[c] = *unit(st, c, g);
                        q[c] = ch[c].f;
                        m[c] = 0;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i)
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const uint32_t w = (i >> 2) == 0 ? v[c].x : (i >> 2) == 1 ? v[c].y : (i >> 2) == 2 ? v[c].z : v[c].w;
                            q[c] = R.next(q[c], __byte_perm(w, 0, 0x4440 | (i & 3)));
                            m[c] = max(m[c], q[c]);
                        }
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        if (m[c] >= A) {
                            uint32_t qq = ch[c].f;
                            dfa_word<WIDE>(qq, ch[c].cnt, v[c].x, R, A);
                            dfa_word<WIDE>(qq, ch[c].cnt, v[c].y, R, A);
                            dfa_word<WIDE>(qq, ch[c].cnt, v[c].z, R, A);
                            dfa_word<WIDE>(qq, ch[c].cnt, v[c].w, R, A);
                            ++reps[c];
                        }
                        ch[c].f = q[c];
                    }
                };
                bool full = true, anydirect = false;
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    full &= len[c] == (uint32_t)SLICE;
                    anydirect |= direct[c];
                }
                if (full && !anydirect) {
#pragma unroll
                    for (int g = 0; g < SLICE / 16; ++g) group_fast(g);
                } else if (full) {
#pragma unroll
                    for (int g = 0; g < SLICE / 16; ++g) group(g, false);
                } else {
#pragma unroll
                    for (int g = 0; g < SLICE / 16; ++g) group(g, true);
                }
#pragma unroll
                for (int c = 0; c < CH; ++c) direct[c] = direct[c] || reps[c] * 8u > 4u * s + 32u;
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    if (!SIMNQ && (ch[c].f & NC_POINT) && len[c] == (uint32_t)SLICE) {
                        // a point mapping over a full slice: its live state
                        // through the DFA rows, the slice's 64 bytes unrolled
                        uint32_t q = ch[c].f & P::MASK, cn = ch[c].cnt;
#pragma unroll
                        for (int g = 0; g < SLICE / 16; ++g) {
                            const uint4 v = *unit(st, c, g);
                            dfa_word<WIDE>(q, cn, v.x, R, A);
                            dfa_word<WIDE>(q, cn, v.y, R, A);
                            dfa_word<WIDE>(q, cn, v.z, R, A);
                            dfa_word<WIDE>(q, cn, v.w, R, A);
                        }
                        ch[c].cnt = cn;
                        ch[c].f = (ch[c].f & ~P::MASK) | q;
                        continue;
                    }
                    const int32_t j0 = (int32_t)(ba[c] + (uint64_t)s * SLICE - lo[c]);
                    for (uint32_t g = 0; 16 * g < len[c]; ++g) {
                        const uint4 v = *unit(st, c, g);
                        if (constant(c)) {
                            uint32_t q = ch[c].f, cn = ch[c].cnt;
                            dfa_word<WIDE>(q, cn, v.x, R, A);
                            dfa_word<WIDE>(q, cn, v.y, R, A);
                            dfa_word<WIDE>(q, cn, v.z, R, A);
                            dfa_word<WIDE>(q, cn, v.w, R, A);
                            ch[c].f = q;
                            ch[c].cnt = cn;
                        } else if (!SIMNQ && (ch[c].f & NC_POINT)) {
                            // a point mapping: its live state p through the
                            // DFA rows, 16 bytes at a time
                            uint32_t q = ch[c].f & P::MASK, cn = ch[c].cnt;
                            dfa_word<WIDE>(q, cn, v.x, R, A);
                            dfa_word<WIDE>(q, cn, v.y, R, A);
                            dfa_word<WIDE>(q, cn, v.z, R, A);
                            dfa_word<WIDE>(q, cn, v.w, R, A);
                            ch[c].cnt = cn;
                            ch[c].f = (ch[c].f & ~P::MASK) | q;
                        } else {
                            const uint32_t ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                step(c, (ws[i >> 2] >> (8 * (i & 3))) & 0xffu, j0 + (int32_t)(16 * g) + i);
                            if (SIMNQ) sim_compact<NQ>(V[c], ch[c]);
                        }
                    }
                }
            }
            if (s + STAGES < nsl) issue(s + STAGES);
        }

        // tail bytes, then the chunk's mapping id
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            for (uint64_t p = bb[c] > lo[c] ? bb[c] : lo[c]; p < hi[c]; ++p) step(c, text[p], (int32_t)(p - lo[c]));
            // a point mapping to the end: its source s kept for pass 2 in
            // the warp's extra rows (idle until the next tile's copies), and
            // its D-SFA id (the constant sink once p is there) for the scan
            uint32_t ps = NO_PT;
            if (!SIMNQ && (ch[c].f & NC_POINT)) {
                ps = point_source_of<WIDE>(ch[c].f);
                const uint32_t p = ch[c].f & P::MASK;
                const uint32_t fld = ps & ~PS_SET;
                // byte ids: the stored id of {ps -> p} or {S -> p}; 16-bit
                // ids keep the encoded form (neither is stored)
                if constexpr (WIDE)
                    ch[c].f = p == T.sink ? p : ch[c].f;
                else
                    ch[c].f = p == T.sink ? p : __ldg((ps & PS_SET ? T.spid : T.pid) + fld * nr + p);
            }
            s_psrc[c * 32 + lane] = (uint16_t)ps;
            if (SIMNQ) sim_compact<NQ>(V[c], ch[c]);
            if (SIMNQ && V[c].mode != SIM_CONST) {
                // keep the vector for the scan: id nr + global chunk index
                const uint64_t gk = WT ? (uint64_t)gt * 32 + lane : (uint64_t)gt * CPT + (uint64_t)c * THREADS + tid;
                uint8_t *dst = S.chainvec + gk * vstride;
#pragma unroll 4
                for (int i = 0; i < NQ / 4; ++i) {
                    const uint32_t x = sim_word<NQ>(V[c], i);
#pragma unroll
                    for (int b4 = 0; b4 < 4; ++b4)
                        if ((uint32_t)(4 * i + b4) < nr) dst[4 * i + b4] = (x >> (8 * b4)) & 0xffu;
                }
                ch[c].f = nr + (uint32_t)gk;
            }
        }

#pragma unroll
        for (int c = 0; c < CH; ++c) s_f[c * THREADS + tid] = ch[c].f;
        __syncwarp();   // chunk vectors of the simulation path written by this warp
        if constexpr (WT) {
            // ---------------- warp tile: summary, look-back, pass 2 ----------------
            const uint32_t fl = ch[0].f;
            const uint32_t cm = __ballot_sync(0xffffffffu, fl < nr);
            uint64_t *st = S.status + gt;
            uint8_t *gv = s_gvec + (size_t)warp * nr;   // this warp's |Q|-vector
            const bool skip = (S.debug & SFA_DEBUG_SKIP_PUBLISH) && local == 1;
            uint32_t tval = 0;
            if (cm) {
                // constant: the last constant chunk composed with the chunks
                // after it; an inclusive prefix at once
                const int lc = 31 - __clz(cm);
                tval = __shfl_sync(0xffffffffu, fl, lc);
                for (int i = lc + 1; i < 32; ++i) tval = amap(__shfl_sync(0xffffffffu, fl, i), tval);
                if (lane == 0 && !skip) st_relaxed(st, ST_PREFIX | tval);
            } else {
                // a |Q|-vector: lanes take the components, every chunk in
                // turn; published as the tile's aggregate
                uint8_t *agg = S.agg + (size_t)gt * nr_max;
                for (uint32_t qb = 0; qb < nr; qb += 32) {
                    const uint32_t q = qb + lane;
                    uint32_t v = q < nr ? q : 0u;
                    for (int i = 0; i < 32; ++i) v = amap(__shfl_sync(0xffffffffu, fl, i), v);
                    if (q < nr) {
                        gv[q] = (uint8_t)v;
                        agg[q] = (uint8_t)v;
                    }
                }
                __threadfence();
                __syncwarp();
                if (lane == 0 && local > 0 && !skip) st_release(st, ST_AGG);
            }
            uint32_t s_in = 0, incl = tval;
            if (lane == 0) {
                s_in = tile_entering_state<WIDE>(S, T, d, out, ts, gt, local, nr, nr_max);
                if (!cm) {
                    incl = gv[s_in];
                    if (!skip) st_relaxed(st, ST_PREFIX | incl);
                }
            }
            s_in = __shfl_sync(0xffffffffu, s_in, 0);
            // entering state of every chunk: the nearest constant chunk below
            // it (or s_in), then the chunks in between; pass 2
            const uint32_t below = cm & lanemask_lt;
            const int j = below ? 31 - __clz(below) : -1;
            uint32_t v = __shfl_sync(0xffffffffu, fl, j < 0 ? 0 : j);
            if (j < 0) v = s_in;
            for (int i = j + 1; i < lane; ++i) v = amap(s_f[warp * 32 + i], v);
            unsigned long long tsum = ch[0].cnt;
            if (ch[0].lm >= 0)
                tsum = dfa_count<WIDE>(text, lo[0], lo[0] + (uint64_t)ch[0].lm + 1, v, R, A) +
                       chunk_count_after(ch[0], v, point_src(0), T);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, o);
            if (lane == 0) finish_tile(S, T, d, ts, out, tsum, local, incl);
            __syncwarp();
            // every warp of the grid had at most one tile: no second grab
            if (!BATCH && S.total_tiles <= gridDim.x * (uint32_t)NW) {
                if (*(volatile uint32_t *)&S.hdr->err) drain_stages(bar0, parity, STAGES, S.timeout_us);
                break;
            }
            continue;
        }

        // ---------------- scan of the chunk mappings inside the tile ----------------
        uint32_t my_gconst = 0;   // bit c: the group of round c is constant (warp-uniform)
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int g = c * NW + warp;
            const uint32_t fl = ch[c].f;
            const uint32_t cm = __ballot_sync(0xffffffffu, fl < nr);
            if (cm) {
                // the group's mapping is constant: its last constant chunk
                // composed with the (non-constant) chunks after it
                const int lc = 31 - __clz(cm);
                uint32_t v = __shfl_sync(0xffffffffu, fl, lc);
                for (int i = lc + 1; i < 32; ++i) v = amap(__shfl_sync(0xffffffffu, fl, i), v);
                if (lane == 0) s_gval[g] = v;
                my_gconst |= 1u << c;
            } else {
                // a |Q|-vector: lanes take the components, every chunk in turn
                for (uint32_t qb = 0; qb < nr; qb += 32) {
                    const uint32_t q = qb + lane;
                    uint32_t v = q < nr ? q : 0u;
                    for (int i = 0; i < 32; ++i) v = amap(__shfl_sync(0xffffffffu, fl, i), v);
                    if (q < nr) s_gvec[(size_t)g * nr + q] = (SID)v;
                }
            }
        }
        if (lane == 0 && my_gconst) {
            uint32_t bits = 0;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (my_gconst & (1u << c)) bits |= 1u << (c * NW + warp);
            atomicOr(&s_misc->gconst, bits);
        }
        __syncthreads();

        // ---------------- tile aggregate, look-back, group prefixes (warp 0) ----------------
        if (warp == 0) {
            const uint32_t gconst = s_misc->gconst & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
            uint64_t *st = S.status + gt;
            SID *agg = reinterpret_cast<SID *>(S.agg) + (size_t)gt * nr_max;
            const bool skip = (S.debug & SFA_DEBUG_SKIP_PUBLISH) && local == 1;
            const bool tconst = gconst != 0;
            uint32_t tval = 0;
            if (tconst) {
                const int gc = 31 - __clz(gconst);
                tval = s_gval[gc];
                for (int g = gc + 1; g < G; ++g) tval = s_gvec[(size_t)g * nr + tval];
                if (lane == 0 && !skip) st_relaxed(st, ST_PREFIX | tval);
                // the slice mapping needs every tile's vector: a constant one
                // maps every state to tval
                if (S.map_mode)
                    for (uint32_t q = lane; q < nr; q += 32) agg[q] = (SID)tval;
            } else {
                for (uint32_t qb = 0; qb < nr; qb += 32) {
                    const uint32_t q = qb + lane;
                    if (q < nr) {
                        uint32_t v = q;
                        for (int g = 0; g < G; ++g) v = s_gvec[(size_t)g * nr + v];
                        agg[q] = (SID)v;
                    }
                }
                __threadfence();
                __syncwarp();
                if (lane == 0 && local > 0 && !skip) st_release(st, ST_AGG);
            }
            // entering state of the tile.  A constant tile whose first chunk
            // is constant needs it only for that chunk's recount: none if the
            // chunk has no mixed position, else (if the CTA will take another
            // tile) deferred until after that tile
            uint32_t s_in = 0;
            if (lane == 0) {
                const bool first_const =
                    DEFER && tconst && local > 0 && ch[0].f < nr && point_src(0) == NO_POINT && total > gridDim.x;
                if (first_const && ch[0].lm < 0) {
                    s_in = 0;   // unused
                } else if (first_const && ch[0].lm < 64) {
                    s_misc->dfr_gt = gt;
                    s_misc->dfr_ti = ti;
                    s_misc->dfr_lo = lo[0];
                    s_misc->dfr_lm = ch[0].lm;
                    s_misc->dfr_valid = 1;
                } else {
                    s_in = tile_entering_state<WIDE>(S, T, d, out, ts, gt, local, nr, nr_max);
                }
                uint32_t incl = tval;
                if (!tconst) {
                    incl = s_in;
                    for (int g = 0; g < G; ++g) incl = s_gvec[(size_t)g * nr + incl];
                    if (!skip) st_relaxed(st, ST_PREFIX | incl);
                }
                s_misc->s_in = s_in;
                s_misc->incl = incl;
            }
            s_in = __shfl_sync(0xffffffffu, s_in, 0);
            // exclusive prefix of every group: the nearest constant group
            // below it, then the vector groups in between
            if (lane < G) {
                const uint32_t below = gconst & lanemask_lt;
                int j;
                uint32_t v;
                if (below) {
                    j = 31 - __clz(below);
                    v = s_gval[j];
                } else {
                    j = -1;
                    v = s_in;
                }
                for (int g = j + 1; g < lane; ++g) v = s_gvec[(size_t)g * nr + v];
                s_gpre[lane] = v;
            }
        }
        __syncthreads();

        // ---------------- entering state of every chunk, pass 2 (count) ----------------
        unsigned long long tsum = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int g = c * NW + warp;
            const uint32_t fl = ch[c].f;
            const uint32_t cm = __ballot_sync(0xffffffffu, fl < nr);
            const uint32_t below = cm & lanemask_lt;
            const int j = below ? 31 - __clz(below) : -1;
            uint32_t v = __shfl_sync(0xffffffffu, fl, j < 0 ? 0 : j);
            if (j < 0) v = s_gpre[g];
            for (int i = j + 1; i < lane; ++i) v = amap(s_f[g * 32 + i], v);
            uint32_t cc = ch[c].cnt;
            if (ch[c].lm >= 0) {
                // the tile's first chunk with a deferred recount: only the
                // positions after its last mixed one now
                const bool deferred = DEFER && c == 0 && tid == 0 && s_misc->dfr_valid;
                cc = (deferred ? 0u : dfa_count<WIDE>(text, lo[c], lo[c] + (uint64_t)ch[c].lm + 1, v, R, A)) +
                     chunk_count_after(ch[c], v, point_src(c), T);
            }
            tsum += cc;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, o);
        if (lane == 0) s_misc->wsum[warp] = tsum;
        __syncthreads();
        if (tid == 0) {
            unsigned long long sum = 0;
            for (int w = 0; w < NW; ++w) sum += s_misc->wsum[w];
            if (DEFER && s_misc->dfr_valid)
                add_tile_count(d, ts, sum, local, s_misc->incl);   // done when the recount is resolved
            else
                finish_tile(S, T, d, ts, out, sum, local, s_misc->incl);
        }
        __syncthreads();
        // every CTA of the grid had at most one tile (each CTA takes one
        // per grab): no second grab
        if (!BATCH && S.total_tiles <= gridDim.x) {
            if (*(volatile uint32_t *)&S.hdr->err) drain_stages(bar0, parity, STAGES, S.timeout_us);
            break;
        }
    }
}

}  // namespace sfa_dev
