// The short-text form of Alg. 5: one CTA matches a text of up to
// SMALL_THREADS * SMALL_CHUNK bytes with no scratch memory, no tensor maps
// and no look-back, for the latency of single short matches.  Each thread
// loads its chunk into shared memory (word k of thread t at k * SMALL_THREADS
// + t, so that a warp's reads of one word are conflict-free), runs the SFA
// from f_I over it, and after the CTA's scan of the chunk mappings (Lemma 1)
// recounts the prefix whose acceptance depended on the entering state.  D-SFA
// handles with byte state ids only.  Every loop over text bytes is rolled: a
// launch of a few microseconds lands on an SM whose instruction cache does
// not hold this kernel, so its code is kept short.  The launch's latency is
// a chain of dependent loads, so the tables arrive by asynchronous copies
// issued together with the text's loads: the non-constant rows, staged in
// shared memory when they fit (pass 1 then never waits on L2), by one bulk
// copy on an mbarrier (a bounded wait), the other tables by cp.async; and
// the scans and the final sum use warp ballots and shuffles instead of loops
// over shared memory.
//
// Past one CTA's 64 KiB (and for latency already past 16 KiB) the same
// kernel runs as a thread-block cluster of up to 16 CTAs, each matching a
// contiguous run of chunks: every CTA composes its groups into its aggregate
// (a constant, f_I, or a |Q|-vector), and after a cluster barrier reads the
// aggregates of the CTAs before it from their shared memory (Lemma 1 across
// CTAs, no global scratch and no wait on a flag); the counts are added into
// CTA 0's shared memory, which writes the result after a second barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "api_internal.h"
#include "sfa_device.cuh"

namespace sfa_dev {

constexpr int SMALL_THREADS = 1024;
constexpr int SMALL_CHUNK = 64;               // bytes per chunk at most (chunk 0: up to 15 more)
constexpr int SMALL_WORDS = (SMALL_CHUNK + 16) / 4;
constexpr int SMALL_CLUSTER_MAX = 16;         // CTAs of a cluster at most (a non-portable size)
constexpr uint32_t SMALL_WAIT_US = 2000000;   // bound of the one wait (for the bulk copy)

struct SmallLayout {
    static constexpr int G = SMALL_THREADS / 32;
    static SFA_HD size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static SFA_HD size_t cls_off(uint32_t nr) { return a16((size_t)nr * ROWB); }
    static SFA_HD size_t f_off(uint32_t nr) { return cls_off(nr) + 256; }
    static SFA_HD size_t gval_off(uint32_t nr) { return f_off(nr) + SMALL_THREADS * 4; }
    static SFA_HD size_t gpre_off(uint32_t nr) { return gval_off(nr) + G * 4; }
    static SFA_HD size_t red_off(uint32_t nr) { return gpre_off(nr) + G * 4; }
    static SFA_HD size_t misc_off(uint32_t nr) { return red_off(nr) + G * 8; }
    // cluster exchange: aggregate kind and value, final state, count (u64);
    // then the mbarrier of the bulk copy of the non-constant rows
    static SFA_HD size_t clu_off(uint32_t nr) { return misc_off(nr) + 16; }
    static SFA_HD size_t txt_off(uint32_t nr) { return clu_off(nr) + 32; }
    static SFA_HD size_t gvec_off(uint32_t nr) { return txt_off(nr) + (size_t)SMALL_WORDS * SMALL_THREADS * 4; }
    static SFA_HD size_t aggv_off(uint32_t nr) { return gvec_off(nr) + (size_t)G * nr; }   // the CTA's vector
    static SFA_HD size_t orig_off(uint32_t nr) { return a16(aggv_off(nr) + nr); }
    static SFA_HD size_t nc_off(uint32_t nr) { return a16(orig_off(nr) + (size_t)nr * 4); }
    static SFA_HD size_t bytes(uint32_t nr) { return nc_off(nr); }
    // with the non-constant rows (nc_words 32-bit entries) staged
    static SFA_HD size_t bytes(uint32_t nr, uint64_t nc_words) { return a16(nc_off(nr) + nc_words * 4); }
};
static_assert(SmallLayout::G == 32, "the group scans are one warp wide");

constexpr uint32_t GV_IDENT = 0xfffffffeu;    // a group of f_I chunks (past the text)
constexpr uint32_t GV_VEC = 0xffffffffu;      // a group summarised by a |Q|-vector
// kinds of a CTA's aggregate in a cluster
constexpr uint32_t AGG_IDENT = 0, AGG_CONST = 1, AGG_VEC = 2;

// asynchronous global -> shared copies (no register holds the data)
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// byte b of a text word
__device__ __forceinline__ uint32_t wbyte(uint32_t x, uint32_t b) { return __byte_perm(x, 0, 0x4440 | b); }

// sfa_step over byte ids, given the byte's class, with a generic load of the
// non-constant row entry (the rows are in shared or in global memory)
__device__ __forceinline__ void small_step(Chain &s, uint32_t b, uint32_t cl, int32_t j, const Rows<false> &R,
                                           const uint32_t *nc, uint32_t nr, uint32_t ncls, uint32_t first_accept) {
    using P = Pt<false>;
    if (s.f & NC_POINT) {
        const uint32_t p = R.next(s.f & P::MASK, b);
        s.cnt += p >= first_accept;
        s.f = (s.f & ~P::MASK) | p;
    } else if (s.f >= nr) {
        const uint32_t e = nc[(size_t)(s.f - nr) * ncls + cl];
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

__global__ void __launch_bounds__(SMALL_THREADS, 1) sfa_small_kernel(Tables T, const uint8_t *text, uint64_t n,
                                                                  uint32_t chunk, uint32_t origin, uint32_t carry,
                                                                  uint32_t nc_words, sfa_result *out) {
    using L = SmallLayout;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t nr = T.nr, A = T.first_accept;
    uint8_t *s_dfa = smem;
    uint8_t *s_cls = smem + L::cls_off(nr);
    uint32_t *s_f = reinterpret_cast<uint32_t *>(smem + L::f_off(nr));
    uint32_t *s_gval = reinterpret_cast<uint32_t *>(smem + L::gval_off(nr));
    uint32_t *s_gpre = reinterpret_cast<uint32_t *>(smem + L::gpre_off(nr));
    unsigned long long *s_red = reinterpret_cast<unsigned long long *>(smem + L::red_off(nr));
    uint32_t *s_misc = reinterpret_cast<uint32_t *>(smem + L::misc_off(nr));
    uint32_t *s_txt = reinterpret_cast<uint32_t *>(smem + L::txt_off(nr));
    uint8_t *s_gvec = smem + L::gvec_off(nr);
    int32_t *s_orig = reinterpret_cast<int32_t *>(smem + L::orig_off(nr));
    uint32_t *s_clu = reinterpret_cast<uint32_t *>(smem + L::clu_off(nr));
    unsigned long long *s_total = reinterpret_cast<unsigned long long *>(smem + L::clu_off(nr) + 16);
    uint8_t *s_aggv = smem + L::aggv_off(nr);
    namespace cg = cooperative_groups;
    const cg::cluster_group cluster = cg::this_cluster();
    const uint32_t crank = cluster.block_rank(), csize = cluster.num_blocks();
    const uint32_t gt = crank * SMALL_THREADS + (uint32_t)threadIdx.x;   // this thread's chunk
    uint32_t *s_nc = reinterpret_cast<uint32_t *>(smem + L::nc_off(nr));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    Rows<false> R;
    R.d = s_dfa;

    // This thread's window of the text, from a 16-byte boundary: offsets are
    // taken from the boundary at or below text[0] (head bytes before it).
    // Chunk 0 is [0, origin + chunk) (window bytes [head, 16 + chunk)), chunk
    // t > 0 is [origin + t * chunk, origin + (t + 1) * chunk) (Theorem 3: any
    // division); window bytes [jlo, jhi) are the chunk's.
    const uint32_t head = origin ? 16u - origin : 0u, o16 = head + origin;
    const uint64_t vs = gt == 0 ? 0 : (uint64_t)o16 + (uint64_t)gt * chunk;
    const uint64_t ve_c = (uint64_t)o16 + (uint64_t)(gt + 1) * chunk, ve_t = (uint64_t)head + n;
    const uint64_t ve = ve_c < ve_t ? ve_c : ve_t;
    const uint32_t jlo = gt == 0 ? head : 0u;
    const uint32_t jhi = ve > vs ? (uint32_t)(ve - vs) : 0u;

    // the non-constant rows by one bulk copy (the largest table; the copy
    // engine moves it faster than per-thread copies would)
    uint32_t *s_err = s_misc + 3;   // a bounded wait gave up
    const uint32_t bar = smem_addr(smem + L::clu_off(nr) + 24);
    const uint32_t nc16 = (nc_words + 3) / 4;
    if (tid == 0) {
        *s_err = 0;
        if (nc16) {
            mbar_init(bar, 1);
            mbar_init_fence();
            mbar_arrive_expect_tx(bar, nc16 * 16);
            bulk_copy(smem_addr(s_nc), reinterpret_cast<const uint8_t *>(T.nc), nc16 * 16, bar);
        }
    }
    // the chunk's full 16-byte units into registers
    uint4 tx[SMALL_WORDS / 4];
#pragma unroll
    for (uint32_t u = 0; u < (uint32_t)SMALL_WORDS / 4; ++u) {
        const uint32_t a = 16 * u;
        tx[u] = make_uint4(0, 0, 0, 0);
        if (jlo <= a && a + 16 <= jhi) tx[u] = ldg128(text + (vs + a - head));
    }
    // the other tables by asynchronous copies: DFA rows in 8-byte pieces (rows
    // ROWB apart, not all 16-byte aligned), the class table, the caller's
    // state ids
#pragma unroll 1
    for (uint32_t i = tid; i < nr * 32; i += SMALL_THREADS)
        cp_async8(s_dfa + (i >> 5) * ROWB + (i & 31) * 8, T.dfa + (size_t)i * 8);
    if (tid < 16) cp_async16(s_cls + tid * 16, T.cls + tid * 16);
    if ((uint32_t)tid < nr) cp_async4(s_orig + tid, T.orig_of + tid);
    const uint32_t *ncp = nc_words ? s_nc : T.nc;
    // the text's first or last partial 16 bytes (chunk 0 and the last chunk)
#pragma unroll 1
    for (uint32_t u = 0; u < (uint32_t)SMALL_WORDS / 4; ++u) {
        const uint32_t a = 16 * u;
        if (!(jlo <= a && a + 16 <= jhi) && a < jhi && a + 16 > jlo) {
            uint32_t wd[4] = {0, 0, 0, 0};
#pragma unroll
            for (uint32_t b = 0; b < 16; ++b)
                if (a + b >= jlo && a + b < jhi) wd[b >> 2] |= (uint32_t)__ldg(text + (vs + a + b - head)) << (8 * (b & 3));
            s_txt[(4 * u + 0) * SMALL_THREADS + tid] = wd[0];
            s_txt[(4 * u + 1) * SMALL_THREADS + tid] = wd[1];
            s_txt[(4 * u + 2) * SMALL_THREADS + tid] = wd[2];
            s_txt[(4 * u + 3) * SMALL_THREADS + tid] = wd[3];
        }
    }
#pragma unroll
    for (uint32_t u = 0; u < (uint32_t)SMALL_WORDS / 4; ++u) {
        const uint32_t a = 16 * u;
        if (jlo <= a && a + 16 <= jhi) {
            s_txt[(4 * u + 0) * SMALL_THREADS + tid] = tx[u].x;
            s_txt[(4 * u + 1) * SMALL_THREADS + tid] = tx[u].y;
            s_txt[(4 * u + 2) * SMALL_THREADS + tid] = tx[u].z;
            s_txt[(4 * u + 3) * SMALL_THREADS + tid] = tx[u].w;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // the non-constant rows (the staged region is 256-byte aligned and padded
    // in global memory: whole 16-byte units are read); a bounded wait
    if (nc16) wait_stage(bar, 0u, s_err, SMALL_WAIT_US);

    // pass 1: the chunk from f_I, one word (4 bytes) per iteration; a word
    // entered with a constant mapping is four DFA-row lookups
    Chain ch;
    ch.f = T.ident;
    ch.cnt = 0;
    ch.snap = 0;
    ch.lm = -1;
    const uint32_t kend = (jhi + 3) >> 2;
#pragma unroll 1
    for (uint32_t k = jlo >> 2; k < kend; ++k) {
        const uint32_t x = s_txt[k * SMALL_THREADS + tid];
        const uint32_t j0 = 4 * k;
        if (j0 >= jlo && j0 + 4 <= jhi && ch.f < nr) {
            uint32_t q = ch.f, c = 0;
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                q = R.next(q, wbyte(x, b));
                c += q >= A;
            }
            ch.f = q;
            ch.cnt += c;
        } else {
            uint32_t cl[4];
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) cl[b] = s_cls[wbyte(x, b)];
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                const uint32_t j = j0 + b;
                if (j >= jlo && j < jhi) small_step(ch, wbyte(x, b), cl[b], (int32_t)j, R, ncp, nr, T.ncls, A);
            }
        }
    }
    uint32_t ps = NO_POINT;
    if (ch.f & NC_POINT) {
        ps = point_source_of<false>(ch.f);
        const uint32_t p = ch.f & 0xffu;
        ch.f = p == T.sink ? p : __ldg((ps & PS_SET ? T.spid : T.pid) + (ps & ~PS_SET) * nr + p);
    }
    const uint32_t fl = ch.f;
    s_f[tid] = fl;

    // group (warp) summaries: a constant, f_I (every chunk past the text), or
    // a |Q|-vector with lanes over states; compositions skip f_I chunks
    const uint32_t am = __ballot_sync(0xffffffffu, fl != T.ident);
    const uint32_t cm = __ballot_sync(0xffffffffu, fl < nr);
    if (cm) {
        const int lc = 31 - __clz(cm);
        uint32_t v = __shfl_sync(0xffffffffu, fl, lc);
        uint32_t m = am & ~((2u << lc) - 1u);
#pragma unroll 1
        while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1u;
            v = apply_map(__shfl_sync(0xffffffffu, fl, i), v, T.maps, nr);
        }
        if (lane == 0) s_gval[warp] = v;
    } else if (!am) {
        if (lane == 0) s_gval[warp] = GV_IDENT;
    } else {
#pragma unroll 1
        for (uint32_t qb = 0; qb < nr; qb += 32) {
            const uint32_t q = qb + lane;
            uint32_t v = q < nr ? q : 0u;
            uint32_t m = am;
#pragma unroll 1
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1u;
                v = apply_map(__shfl_sync(0xffffffffu, fl, i), v, T.maps, nr);
            }
            if (q < nr) s_gvec[(size_t)warp * nr + q] = (uint8_t)v;
        }
        if (lane == 0) s_gval[warp] = GV_VEC;
    }
    // the entering state of the text: q0, or the carried result's state
    if (tid == 0) {
        uint32_t s_in = T.q0, bad = 0;
        if (carry) {
            const sfa_result prev = *out;
            if (prev.status || prev.final_state >= T.nq_in || T.kept_of[prev.final_state] < 0)
                bad = 1;
            else
                s_in = (uint32_t)T.kept_of[prev.final_state];
        }
        s_misc[0] = s_in;
        s_misc[1] = bad;
        if (crank == 0) *s_total = 0;
    }
    __syncthreads();
    if (csize > 1) {
        // this CTA's aggregate (warp 0): its groups composed in order
        if (warp == 0) {
            const uint32_t gv = s_gval[lane];
            const uint32_t cgm = __ballot_sync(0xffffffffu, gv < GV_IDENT);
            const uint32_t vgm = __ballot_sync(0xffffffffu, gv == GV_VEC);
            if (cgm) {
                const int j = 31 - __clz(cgm);
                uint32_t v = __shfl_sync(0xffffffffu, gv, j);
                uint32_t m = vgm & ~((2u << j) - 1u);
#pragma unroll 1
                while (m) {
                    const int g = __ffs(m) - 1;
                    m &= m - 1u;
                    v = s_gvec[(size_t)g * nr + v];
                }
                if (lane == 0) {
                    s_clu[0] = AGG_CONST;
                    s_clu[1] = v;
                }
            } else if (!vgm) {
                if (lane == 0) s_clu[0] = AGG_IDENT;
            } else {
#pragma unroll 1
                for (uint32_t q = lane; q < nr; q += 32) {
                    uint32_t v = q, m = vgm;
#pragma unroll 1
                    while (m) {
                        const int g = __ffs(m) - 1;
                        m &= m - 1u;
                        v = s_gvec[(size_t)g * nr + v];
                    }
                    s_aggv[q] = (uint8_t)v;
                }
                if (lane == 0) s_clu[0] = AGG_VEC;
            }
        }
        cluster.sync();   // every aggregate written
        // the state entering this CTA (warp 0; lane j reads CTA j's kind):
        // the last constant aggregate before it, then the vectors after that
        if (warp == 0) {
            uint32_t kind = AGG_IDENT, val = 0;
            if ((uint32_t)lane < crank) {
                const uint32_t *rc = cluster.map_shared_rank(s_clu, (int)lane);
                kind = rc[0];
                val = rc[1];
            }
            const uint32_t ccm = __ballot_sync(0xffffffffu, kind == AGG_CONST);
            const uint32_t cvm = __ballot_sync(0xffffffffu, kind == AGG_VEC);
            const int j = ccm ? 31 - __clz(ccm) : -1;
            const uint32_t vj = __shfl_sync(0xffffffffu, val, j < 0 ? 0 : j);
            uint32_t st = j < 0 ? s_misc[0] : vj;
            uint32_t m = cvm & (j < 0 ? 0xffffffffu : ~((2u << j) - 1u));
#pragma unroll 1
            while (m) {
                const int r = __ffs(m) - 1;
                m &= m - 1u;
                st = cluster.map_shared_rank(s_aggv, r)[st];
            }
            if (lane == 0) s_misc[0] = st;
        }
        __syncthreads();
    }
    // exclusive prefix of every group (warp 0, lane g for group g): the
    // nearest constant group below it, then the vector groups in between
    if (warp == 0) {
        const uint32_t gv = s_gval[lane];
        const uint32_t cgm = __ballot_sync(0xffffffffu, gv < GV_IDENT);
        const uint32_t vgm = __ballot_sync(0xffffffffu, gv == GV_VEC);
        const uint32_t below = cgm & lanemask_lt;
        const int j = below ? 31 - __clz(below) : -1;
        const uint32_t vj = __shfl_sync(0xffffffffu, gv, j < 0 ? 0 : j);
        uint32_t v = j < 0 ? s_misc[0] : vj;
        uint32_t m = vgm & lanemask_lt & (j < 0 ? 0xffffffffu : ~((2u << j) - 1u));
#pragma unroll 1
        while (m) {
            const int g = __ffs(m) - 1;
            m &= m - 1u;
            v = s_gvec[(size_t)g * nr + v];
        }
        s_gpre[lane] = v;
    }
    __syncthreads();

    // entering state of this chunk, pass 2 from shared memory, the state after it
    const uint32_t below = cm & lanemask_lt;
    const int jc = below ? 31 - __clz(below) : -1;
    uint32_t v = __shfl_sync(0xffffffffu, fl, jc < 0 ? 0 : jc);
    if (jc < 0) v = s_gpre[warp];
    uint32_t mb = am & lanemask_lt & (jc < 0 ? 0xffffffffu : ~((2u << jc) - 1u));
#pragma unroll 1
    while (mb) {
        const int i = __ffs(mb) - 1;
        mb &= mb - 1u;
        v = apply_map(s_f[warp * 32 + i], v, T.maps, nr);
    }
    unsigned long long cnt = ch.cnt;
    if (ch.lm >= 0) {
        const uint32_t lm = (uint32_t)ch.lm;
        uint32_t q = v, c = 0;
#pragma unroll 1
        for (uint32_t k = jlo >> 2; 4 * k <= lm; ++k) {
            const uint32_t x = s_txt[k * SMALL_THREADS + tid];
            const uint32_t j0 = 4 * k;
            if (j0 >= jlo && j0 + 3 <= lm) {
#pragma unroll
                for (uint32_t b = 0; b < 4; ++b) {
                    q = R.next(q, wbyte(x, b));
                    c += q >= A;
                }
            } else {
#pragma unroll
                for (uint32_t b = 0; b < 4; ++b) {
                    const uint32_t j = j0 + b;
                    if (j >= jlo && j <= lm) {
                        q = R.next(q, wbyte(x, b));
                        c += q >= A;
                    }
                }
            }
        }
        cnt = c + chunk_count_after(ch, v, ps, T);
    }
    if (tid == SMALL_THREADS - 1) s_misc[2] = fl == T.ident ? v : apply_map(fl, v, T.maps, nr);   // after the text
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_red[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        unsigned long long total = s_red[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(0xffffffffu, total, o);
        if (lane == 0) {
            if (csize > 1) {
                // into CTA 0: the count, a wait that gave up, and from the
                // last CTA the state after the text
                atomicAdd(cluster.map_shared_rank(s_total, 0), total);
                if (*(volatile uint32_t *)s_err) atomicOr(cluster.map_shared_rank(s_err, 0), 1u);
                if (crank == csize - 1) *cluster.map_shared_rank(s_clu + 2, 0) = s_misc[2];
            } else {
                *s_total = total;
                s_clu[2] = s_misc[2];
            }
        }
    }
    if (csize > 1) cluster.sync();   // every count added; no CTA leaves while others read its memory
    if (crank == 0 && tid == 0) {
        const uint32_t fin = s_clu[2];
        sfa_result r;
        r.final_state = (uint32_t)s_orig[fin < nr ? fin : 0];
        r.accept_final = fin >= A ? 1 : 0;
        r.status = s_misc[1] || *(volatile uint32_t *)s_err ? SFA_STATUS_TIMEOUT : SFA_STATUS_OK;
        r.reserved = 0;
        r.count = (carry ? out->count : 0ull) + *s_total;
        *out = r;
    }
    // a wait that gave up: the bulk copy may still be landing; a bounded wait
    // for it before the CTA's shared memory is released
    if (tid == 0 && nc16 && *(volatile uint32_t *)s_err) drain_stages(bar, 1u, 1, SMALL_WAIT_US);
}

}  // namespace sfa_dev

namespace sfa_impl {

namespace {

constexpr uint64_t CLUSTER_FROM = 16 << 10;   // longer texts take a cluster of CTAs,
constexpr uint64_t CTA_BYTES = 8 << 10;       // about this many bytes each

// whether clusters of c CTAs of this shape can be resident on the device,
// asked once per (device, c, shared-memory size)
bool cluster_fits(int dev, int c, size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, int>, std::pair<size_t, bool>>> known;
    std::lock_guard<std::mutex> lock(mu);
    for (auto &e : known)
        if (e.first.first == dev && e.first.second == c && e.second.first == smem) return e.second.second;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3(sfa_dev::SMALL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, reinterpret_cast<const void *>(&sfa_dev::sfa_small_kernel),
                                                   &cfg) == cudaSuccess &&
                    nclusters > 0;
    if (!ok) cudaGetLastError();
    known.push_back({{dev, c}, {smem, ok}});
    return ok;
}

}  // namespace

bool small_fits(uint64_t n) {
    return n <= (uint64_t)sfa_dev::SMALL_CLUSTER_MAX * sfa_dev::SMALL_THREADS * sfa_dev::SMALL_CHUNK;
}

size_t small_smem(uint32_t nr) { return sfa_dev::SmallLayout::bytes(nr); }

int launch_small(const sfa_dev::Tables &T, uint64_t n_nc, const uint8_t *text, uint64_t n, bool carry,
                 sfa_result *out, cudaStream_t s) {
    if (!small_fits(n) || T.nr > 255) return SFA_ERR_UNSUPPORTED;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SFA_ERR_UNSUPPORTED;
    const size_t optin = device_props(dev).smem_optin;
    // the kernel's shared-memory limit and cluster size, raised once per device
    static std::atomic<uint8_t> attr_done[64];
    if (!attr_done[dev].load(std::memory_order_acquire)) {
        const void *k = reinterpret_cast<const void *>(&sfa_dev::sfa_small_kernel);
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)optin));
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_done[dev].store(1, std::memory_order_release);
    }
    // the non-constant rows go to shared memory when they fit
    const uint64_t nc_words = n_nc * T.ncls;
    const bool stage = nc_words && sfa_dev::SmallLayout::bytes(T.nr, nc_words) <= optin;
    const size_t smem = stage ? sfa_dev::SmallLayout::bytes(T.nr, nc_words) : small_smem(T.nr);
    // CTAs: one up to CLUSTER_FROM bytes, then about CTA_BYTES each (fewer if
    // a cluster that large cannot be resident, while every chunk stays within
    // SMALL_CHUNK bytes)
    const uint32_t origin = n ? sfa_dev::text_origin(text) : 0u;
    const uint64_t body = n > origin ? n - origin : 0;
    int c = n <= CLUSTER_FROM ? 1
                              : (int)std::min<uint64_t>(sfa_dev::SMALL_CLUSTER_MAX, (n + CTA_BYTES - 1) / CTA_BYTES);
    const uint64_t cap_cta = (uint64_t)sfa_dev::SMALL_THREADS * sfa_dev::SMALL_CHUNK;
    while (c > 1 && !cluster_fits(dev, c, smem)) {
        if ((uint64_t)(c - 1) * cap_cta < body + 16) return SFA_ERR_UNSUPPORTED;   // the persistent kernel takes it
        --c;
    }
    // chunk bodies from the first 16-byte boundary, in 16-byte multiples
    const uint64_t threads = (uint64_t)c * sfa_dev::SMALL_THREADS;
    uint32_t chunk = (uint32_t)((body + threads - 1) / threads);
    chunk = std::max<uint32_t>(16, (chunk + 15) & ~15u);
    if (chunk > (uint32_t)sfa_dev::SMALL_CHUNK) return SFA_ERR_UNSUPPORTED;
    const uint32_t nc_arg = stage ? (uint32_t)nc_words : 0u, carry_arg = carry ? 1u : 0u;
    if (c == 1) {
        sfa_dev::sfa_small_kernel<<<1, sfa_dev::SMALL_THREADS, smem, s>>>(T, text, n, chunk, origin, carry_arg,
                                                                         nc_arg, out);
    } else {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(sfa_dev::SMALL_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, &sfa_dev::sfa_small_kernel, T, text, n, chunk, origin, carry_arg, nc_arg, out));
    }
    CK(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

}  // namespace sfa_impl
