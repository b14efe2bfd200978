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
// Acceptance bookkeeping (the count): while a chunk runs from f_I its state
// f is known only as a mapping, so for position j the final-ness of
// f(s_in) depends on the still unknown entering state s_in exactly when f is
// "mixed" (final for some kept q, not for others).  Pass 1 counts the
// positions whose mapping is final for every q and remembers the last mixed
// position; once s_in is known, pass 2 reruns the DFA (Alg. 2) from s_in
// over the prefix up to that position.  For synchronising automata (all
// literal automata) that prefix is at most the longest literal.
#pragma once

#include <cstdint>

#include "sfa.h"
#include "sfa_types.h"

namespace sfa_dev {

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint4 ldg128(const uint8_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
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

// ---------------------------------------------------------------------------
// per-chunk state of pass 1
// ---------------------------------------------------------------------------
struct Chain {
    uint32_t f;       // state id
    uint32_t cnt;     // positions whose mapping is final for every kept q
    uint32_t snap;    // cnt at the last mixed position
    int32_t lm;       // offset of the last mixed position, -1 if none
};

// one symbol of Alg. 5 in the D-SFA: f <- delta_s[f, sigma]
__device__ __forceinline__ void sfa_step(Chain &s, uint32_t b, int32_t j, const uint8_t *s_dfa,
                                         const uint8_t *s_cls, const uint32_t *nc, uint32_t nr,
                                         uint32_t ncls, uint32_t first_accept) {
    if (s.f >= nr) {
        const uint32_t e = __ldg(nc + (size_t)(s.f - nr) * ncls + s_cls[b]);
        s.f = e & NC_ID_MASK;
        const uint32_t a = e >> 30;
        if (a == ACC_ALL) {
            s.cnt++;
        } else if (a == ACC_MIXED) {
            s.lm = j;
            s.snap = s.cnt;
        }
    } else {
        s.f = s_dfa[(s.f << 8) | b];
        s.cnt += s.f >= first_accept;
    }
}

// 16 symbols of a constant-state chunk: the DFA row lookups.  The table
// offset (q << 8) | byte is one byte permute of the text word and q.
__device__ __forceinline__ void dfa_word(uint32_t &q, uint32_t &cnt, uint32_t w, const uint8_t *s_dfa,
                                         uint32_t first_accept) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q = s_dfa[__byte_perm(w, q, 0x5540 | j)];
        cnt += q >= first_accept;
    }
}

// ---------------------------------------------------------------------------
// simulation mode: the |Q|-vector T[q] of Alg. 3, packed four states per word
// ---------------------------------------------------------------------------
template <int NQ>
struct SimVec {
    uint32_t w[NQ / 4];
};

template <int NQ>
__device__ __forceinline__ void sim_step(SimVec<NQ> &T, Chain &s, uint32_t b, int32_t j,
                                         const uint8_t *s_dfa, uint32_t first_accept) {
    uint32_t mn = 0xffffffffu, mx = 0;
#pragma unroll
    for (int i = 0; i < NQ / 4; ++i) {
        const uint32_t x = T.w[i];
        const uint32_t y0 = s_dfa[__byte_perm(x, b, 0x5504)];
        const uint32_t y1 = s_dfa[__byte_perm(x, b, 0x5514)];
        const uint32_t y2 = s_dfa[__byte_perm(x, b, 0x5524)];
        const uint32_t y3 = s_dfa[__byte_perm(x, b, 0x5534)];
        const uint32_t y = __byte_perm(__byte_perm(y0, y1, 0x0040), __byte_perm(y2, y3, 0x0040), 0x5410);
        T.w[i] = y;
        mn = __vminu4(mn, y);
        mx = __vmaxu4(mx, y);
    }
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
__device__ __forceinline__ bool sim_constant(const SimVec<NQ> &T) {
    const uint32_t splat = (T.w[0] & 0xffu) * 0x01010101u;
    bool c = true;
#pragma unroll
    for (int i = 0; i < NQ / 4; ++i) c &= T.w[i] == splat;
    return c;
}

// mapping applied to a state: constant ids are their own value
__device__ __forceinline__ uint32_t apply_map(uint32_t f, uint32_t v, const uint8_t *mtab, uint32_t nr) {
    return f < nr ? f : (uint32_t)mtab[(size_t)(f - nr) * nr + v];
}

// Alg. 2 from state q over [p, e) of the text, counting final states
__device__ __forceinline__ uint32_t dfa_count(const uint8_t *text, uint64_t p, uint64_t e, uint32_t q,
                                              const uint8_t *s_dfa, uint32_t first_accept) {
    uint32_t c = 0;
    while (p < e && (reinterpret_cast<uintptr_t>(text + p) & 15)) {
        q = s_dfa[(q << 8) | text[p]];
        c += q >= first_accept;
        ++p;
    }
    for (; p + 16 <= e; p += 16) {
        const uint4 v = ldg128(text + p);
        dfa_word(q, c, v.x, s_dfa, first_accept);
        dfa_word(q, c, v.y, s_dfa, first_accept);
        dfa_word(q, c, v.z, s_dfa, first_accept);
        dfa_word(q, c, v.w, s_dfa, first_accept);
    }
    for (; p < e; ++p) {
        q = s_dfa[(q << 8) | text[p]];
        c += q >= first_accept;
    }
    return c;
}

// ---------------------------------------------------------------------------
// the persistent kernel
//   SIMNQ = 0: D-SFA mode; SIMNQ = 16/32/64: simulation mode with vectors of
//   that many entries (the kept states, padded)
//   BATCH: tables and texts come from device arrays, else from `tab`/`desc`
// ---------------------------------------------------------------------------
template <int THREADS, int CH, int SIMNQ, bool BATCH>
__global__ void __launch_bounds__(THREADS)
    sfa_match_kernel(Tables tab, TextDesc desc, const Tables *tabs, const TextDesc *descs,
                     const uint32_t *tile_text, Scratch S, sfa_result *out) {
    using L = SmemLayout<THREADS, CH>;
    constexpr int CPT = L::CPT, NW = L::NW, G = L::G;
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t nr_max = S.nr_max;
    uint8_t *s_dfa = smem + L::dfa_off();
    uint8_t *s_cls = smem + L::cls_off(nr_max);
    uint32_t *s_f = reinterpret_cast<uint32_t *>(smem + L::f_off(nr_max));
    uint32_t *s_gval = reinterpret_cast<uint32_t *>(smem + L::gval_off(nr_max));
    uint32_t *s_gpre = reinterpret_cast<uint32_t *>(smem + L::gpre_off(nr_max));
    Misc *s_misc = reinterpret_cast<Misc *>(smem + L::misc_off(nr_max));
    uint8_t *s_gvec = smem + L::gvec_off(nr_max);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    uint32_t loaded = 0xffffffffu;   // table index in shared memory (CTA-uniform)

    for (;;) {
        if (tid == 0) {
            s_misc->tile = atomicAdd(&S.hdr->tile_ctr, 1u);
            s_misc->gconst = 0;
        }
        __syncthreads();
        const uint32_t gt = s_misc->tile;
        if (gt >= S.total_tiles) break;

        uint32_t ti = 0;
        if (BATCH) ti = __ldg(tile_text + gt);
        const TextDesc d = BATCH ? descs[ti] : desc;
        const Tables T = BATCH ? tabs[d.table] : tab;
        const uint32_t tabidx = BATCH ? d.table : 0u;
        if (tabidx != loaded) {
            // stage the DFA rows and the class table in shared memory
            const uint4 *src = reinterpret_cast<const uint4 *>(T.dfa);
            uint4 *dst = reinterpret_cast<uint4 *>(s_dfa);
            for (uint32_t i = tid; i < T.nr * 16; i += THREADS) dst[i] = __ldg(src + i);
            if (tid < 16) reinterpret_cast<uint4 *>(s_cls)[tid] = __ldg(reinterpret_cast<const uint4 *>(T.cls) + tid);
            loaded = tabidx;
            __syncthreads();
        }
        const uint32_t nr = T.nr, A = T.first_accept;
        const uint32_t local = gt - d.tile_base;
        const uint64_t nch = num_chunks(d);
        TextState *ts = S.texts + (BATCH ? ti : 0u);
        const uint8_t *text = d.text;
        const uint8_t *mtab = SIMNQ ? S.chainvec : T.maps;

        // ---------------- pass 1: every chunk from f_I ----------------
        Chain ch[CH];
        uint64_t lo[CH], hi[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const uint64_t k = (uint64_t)local * CPT + (uint64_t)c * THREADS + tid;
            if (k >= nch) {
                lo[c] = hi[c] = d.n;
            } else if (d.forced) {
                lo[c] = k * d.n / d.forced;
                hi[c] = (k + 1) * d.n / d.forced;
            } else {
                lo[c] = k * d.chunk;
                hi[c] = lo[c] + d.chunk < d.n ? lo[c] + d.chunk : d.n;
            }
            ch[c].f = T.ident;
            ch[c].cnt = 0;
            ch[c].snap = 0;
            ch[c].lm = -1;
        }
        uint64_t pos[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            uint64_t p = lo[c];
            const uint64_t e = hi[c];
            Chain s = ch[c];
            if (SIMNQ == 0) {
                // head bytes until 16-byte alignment, then whole words while
                // the mapping is not constant
                while (p < e && (reinterpret_cast<uintptr_t>(text + p) & 15)) {
                    sfa_step(s, text[p], (int32_t)(p - lo[c]), s_dfa, s_cls, T.nc, nr, T.ncls, A);
                    ++p;
                }
                while (s.f >= nr && p + 16 <= e) {
                    const uint4 v = ldg128(text + p);
                    const uint32_t ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        sfa_step(s, (ws[i >> 2] >> (8 * (i & 3))) & 0xffu, (int32_t)(p - lo[c]) + i, s_dfa,
                                 s_cls, T.nc, nr, T.ncls, A);
                    p += 16;
                }
                if (s.f >= nr)
                    for (; p < e; ++p)
                        sfa_step(s, text[p], (int32_t)(p - lo[c]), s_dfa, s_cls, T.nc, nr, T.ncls, A);
            } else {
                constexpr int NQ = SIMNQ > 0 ? SIMNQ : 4;
                SimVec<NQ> V;
#pragma unroll
                for (int i = 0; i < NQ / 4; ++i) {
                    uint32_t w = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t q = 4 * i + b;
                        w |= (q < nr ? q : 0u) << (8 * b);
                    }
                    V.w[i] = w;
                }
                bool con = nr == 1;
                while (!con && p < e && (reinterpret_cast<uintptr_t>(text + p) & 15)) {
                    sim_step<NQ>(V, s, text[p], (int32_t)(p - lo[c]), s_dfa, A);
                    ++p;
                    con = sim_constant<NQ>(V);
                }
                while (!con && p + 16 <= e) {
                    const uint4 v = ldg128(text + p);
                    const uint32_t ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        sim_step<NQ>(V, s, (ws[i >> 2] >> (8 * (i & 3))) & 0xffu, (int32_t)(p - lo[c]) + i,
                                     s_dfa, A);
                    p += 16;
                    con = sim_constant<NQ>(V);
                }
                while (!con && p < e) {
                    sim_step<NQ>(V, s, text[p], (int32_t)(p - lo[c]), s_dfa, A);
                    ++p;
                    con = sim_constant<NQ>(V);
                }
                if (con) {
                    s.f = V.w[0] & 0xffu;
                } else {
                    // keep the vector for the scan: id nr + global chunk index
                    const uint64_t gk = (uint64_t)gt * CPT + (uint64_t)c * THREADS + tid;
                    uint8_t *dst = S.chainvec + gk * nr;
#pragma unroll
                    for (int i = 0; i < NQ / 4; ++i)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if ((uint32_t)(4 * i + b) < nr) dst[4 * i + b] = (V.w[i] >> (8 * b)) & 0xffu;
                    s.f = nr + (uint32_t)gk;
                }
            }
            // a constant chunk now only needs the DFA rows: reach 16-byte
            // alignment for the fast loop (simulation chunks can converge at
            // any byte, and a one-state automaton starts constant)
            if (s.f < nr) {
                while (p < e && (reinterpret_cast<uintptr_t>(text + p) & 15)) {
                    s.f = s_dfa[(s.f << 8) | text[p]];
                    s.cnt += s.f >= A;
                    ++p;
                }
            } else {
                p = e;
            }
            ch[c] = s;
            pos[c] = p;
        }
        // fast loop: all chunks of the thread in lockstep, one DFA lookup per
        // byte, 16-byte loads prefetched one iteration ahead
        {
            uint64_t m = ~0ull;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const uint64_t v = (hi[c] - pos[c]) >> 4;
                m = v < m ? v : m;
            }
            uint32_t q[CH], cn[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                q[c] = ch[c].f;
                cn[c] = ch[c].cnt;
            }
            if (m > 0) {
                uint4 cur[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) cur[c] = ldg128(text + pos[c]);
                for (uint64_t it = 0; it < m; ++it) {
                    uint4 nxt[CH];
                    if (it + 1 < m) {
#pragma unroll
                        for (int c = 0; c < CH; ++c) nxt[c] = ldg128(text + pos[c] + 16 * (it + 1));
                    }
#pragma unroll
                    for (int c = 0; c < CH; ++c) dfa_word(q[c], cn[c], cur[c].x, s_dfa, A);
#pragma unroll
                    for (int c = 0; c < CH; ++c) dfa_word(q[c], cn[c], cur[c].y, s_dfa, A);
#pragma unroll
                    for (int c = 0; c < CH; ++c) dfa_word(q[c], cn[c], cur[c].z, s_dfa, A);
#pragma unroll
                    for (int c = 0; c < CH; ++c) dfa_word(q[c], cn[c], cur[c].w, s_dfa, A);
#pragma unroll
                    for (int c = 0; c < CH; ++c) cur[c] = nxt[c];
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                uint64_t p = pos[c] + 16 * m;
                uint32_t qq = q[c], cc = cn[c];
                for (; p + 16 <= hi[c]; p += 16) {
                    const uint4 v = ldg128(text + p);
                    dfa_word(qq, cc, v.x, s_dfa, A);
                    dfa_word(qq, cc, v.y, s_dfa, A);
                    dfa_word(qq, cc, v.z, s_dfa, A);
                    dfa_word(qq, cc, v.w, s_dfa, A);
                }
                for (; p < hi[c]; ++p) {
                    qq = s_dfa[(qq << 8) | text[p]];
                    cc += qq >= A;
                }
                ch[c].f = qq;
                ch[c].cnt = cc;
            }
        }

        // ---------------- scan of the chunk mappings inside the tile ----------------
#pragma unroll
        for (int c = 0; c < CH; ++c) s_f[c * THREADS + tid] = ch[c].f;
        __syncwarp();   // chunk vectors of the simulation path written by this warp
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
                for (int i = lc + 1; i < 32; ++i) v = apply_map(__shfl_sync(0xffffffffu, fl, i), v, mtab, nr);
                if (lane == 0) s_gval[g] = v;
                my_gconst |= 1u << c;
            } else {
                // a |Q|-vector: lanes take the components, every chunk in turn
                for (uint32_t qb = 0; qb < nr; qb += 32) {
                    const uint32_t q = qb + lane;
                    uint32_t v = q < nr ? q : 0u;
                    for (int i = 0; i < 32; ++i) v = apply_map(__shfl_sync(0xffffffffu, fl, i), v, mtab, nr);
                    if (q < nr) s_gvec[(size_t)g * nr + q] = (uint8_t)v;
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
            uint8_t *agg = S.agg + (size_t)gt * nr_max;
            const bool skip = (S.debug & SFA_DEBUG_SKIP_PUBLISH) && local == 1;
            bool tconst = gconst != 0;
            uint32_t tval = 0;
            if (tconst) {
                const int gc = 31 - __clz(gconst);
                tval = s_gval[gc];
                for (int g = gc + 1; g < G; ++g) tval = s_gvec[(size_t)g * nr + tval];
                if (lane == 0 && !skip) st_release(st, ST_PREFIX | tval);
            } else {
                for (uint32_t q0 = 0; q0 < nr; q0 += 32) {
                    const uint32_t q = q0 + lane;
                    if (q < nr) {
                        uint32_t v = q;
                        for (int g = 0; g < G; ++g) v = s_gvec[(size_t)g * nr + v];
                        agg[q] = (uint8_t)v;
                    }
                }
                __threadfence();
                __syncwarp();
                if (lane == 0 && local > 0 && !skip) st_release(st, ST_AGG);
            }
            // entering state of the tile
            uint32_t s_in = 0;
            if (lane == 0) {
                if (local == 0) {
                    if (d.carry) {
                        const sfa_result prev = out[d.out_index];
                        if (prev.status || prev.final_state >= T.nq_in || T.kept_of[prev.final_state] < 0) {
                            atomicOr(&ts->err, 1u);
                            s_in = T.q0;
                        } else {
                            s_in = (uint32_t)T.kept_of[prev.final_state];
                        }
                    } else {
                        s_in = T.q0;
                    }
                } else {
                    // decoupled look-back: walk back to the nearest inclusive
                    // prefix, then apply the aggregates in between in order
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
                            v = S.agg[(size_t)i * nr_max + v];
                        }
                    }
                    s_in = v;
                }
                uint32_t incl = tval;
                if (!tconst) {
                    incl = s_in;
                    for (int g = 0; g < G; ++g) incl = s_gvec[(size_t)g * nr + incl];
                    if (!skip) st_release(st, ST_PREFIX | incl);
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
            for (int i = j + 1; i < lane; ++i) v = apply_map(s_f[g * 32 + i], v, mtab, nr);
            uint32_t total = ch[c].cnt;
            if (ch[c].lm >= 0) {
                total = dfa_count(text, lo[c], lo[c] + (uint64_t)ch[c].lm + 1, v, s_dfa, A) + ch[c].cnt - ch[c].snap;
            }
            tsum += total;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, o);
        if (lane == 0) s_misc->wsum[warp] = tsum;
        __syncthreads();
        if (tid == 0) {
            unsigned long long sum = 0;
            for (int w = 0; w < NW; ++w) sum += s_misc->wsum[w];
            if (sum) atomicAdd(&ts->count, sum);
            if (local == d.ntiles - 1) ts->final_state = s_misc->incl;
            __threadfence();
            const uint32_t prev = atomicAdd(&ts->done, 1u);
            if (prev == d.ntiles - 1) {
                // the last tile of this text to finish writes its result
                __threadfence();
                const unsigned long long total = atomicAdd(&ts->count, 0ull);
                const uint32_t fin = *(volatile uint32_t *)&ts->final_state;
                const uint32_t err = *(volatile uint32_t *)&ts->err | *(volatile uint32_t *)&S.hdr->err;
                sfa_result r;
                r.final_state = (uint32_t)T.orig_of[fin < nr ? fin : 0];
                r.accept_final = fin >= A ? 1 : 0;
                r.status = err ? SFA_STATUS_TIMEOUT : SFA_STATUS_OK;
                r.reserved = 0;
                r.count = (d.carry ? out[d.out_index].count : 0ull) + total;
                out[d.out_index] = r;
            }
        }
        __syncthreads();
    }
}

}  // namespace sfa_dev
