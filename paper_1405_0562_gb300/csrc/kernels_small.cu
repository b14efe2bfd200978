// The short-text form of Alg. 5: one CTA matches a text of up to
// SMALL_THREADS * SMALL_CHUNK bytes with no scratch memory, no bulk copies
// and no look-back, for the latency of single short matches.  Each thread
// loads its chunk into shared memory (word k of thread t at k * SMALL_THREADS
// + t, so that a warp's reads of one word are conflict-free), runs the SFA
// from f_I over it, and after the CTA's scan of the chunk mappings (Lemma 1)
// recounts the prefix whose acceptance depended on the entering state.  D-SFA
// handles with byte state ids only.  Every loop over text bytes is rolled: a
// launch of a few microseconds lands on an SM whose instruction cache does
// not hold this kernel, so its code is kept short.
#include <algorithm>

#include "api_internal.h"
#include "sfa_device.cuh"

namespace sfa_dev {

constexpr int SMALL_THREADS = 1024;
constexpr int SMALL_CHUNK = 64;               // bytes per chunk at most (chunk 0: up to 15 more)
constexpr int SMALL_WORDS = (SMALL_CHUNK + 16) / 4;

struct SmallLayout {
    static constexpr int G = SMALL_THREADS / 32;
    static SFA_HD size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static SFA_HD size_t cls_off(uint32_t nr) { return a16((size_t)nr * ROWB); }
    static SFA_HD size_t f_off(uint32_t nr) { return cls_off(nr) + 256; }
    static SFA_HD size_t gval_off(uint32_t nr) { return f_off(nr) + SMALL_THREADS * 4; }
    static SFA_HD size_t gpre_off(uint32_t nr) { return gval_off(nr) + G * 4; }
    static SFA_HD size_t red_off(uint32_t nr) { return gpre_off(nr) + G * 4; }
    static SFA_HD size_t misc_off(uint32_t nr) { return red_off(nr) + G * 8; }
    static SFA_HD size_t txt_off(uint32_t nr) { return misc_off(nr) + 16; }
    static SFA_HD size_t gvec_off(uint32_t nr) { return txt_off(nr) + (size_t)SMALL_WORDS * SMALL_THREADS * 4; }
    static SFA_HD size_t bytes(uint32_t nr) { return a16(gvec_off(nr) + (size_t)G * nr); }
};

__global__ void __launch_bounds__(SMALL_THREADS) sfa_small_kernel(Tables T, const uint8_t *text, uint64_t n,
                                                                  uint32_t chunk, uint32_t origin, uint32_t carry,
                                                                  sfa_result *out) {
    using L = SmallLayout;
    constexpr int G = L::G;
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
    const uint64_t vs = tid == 0 ? 0 : (uint64_t)o16 + (uint64_t)tid * chunk;
    const uint64_t ve_c = (uint64_t)o16 + (uint64_t)(tid + 1) * chunk, ve_t = (uint64_t)head + n;
    const uint64_t ve = ve_c < ve_t ? ve_c : ve_t;
    const uint32_t jlo = tid == 0 ? head : 0u;
    const uint32_t jhi = ve > vs ? (uint32_t)(ve - vs) : 0u;
#pragma unroll
    for (uint32_t u = 0; u < (uint32_t)SMALL_WORDS / 4; ++u) {
        const uint32_t a = 16 * u;
        uint4 x = make_uint4(0, 0, 0, 0);
        if (jlo <= a && a + 16 <= jhi) {
            x = ldg128(text + (vs + a - head));
        } else if (a < jhi && a + 16 > jlo) {   // the text's first or last partial 16 bytes
            uint32_t wd[4] = {0, 0, 0, 0};
#pragma unroll
            for (uint32_t b = 0; b < 16; ++b)
                if (a + b >= jlo && a + b < jhi) wd[b >> 2] |= (uint32_t)__ldg(text + (vs + a + b - head)) << (8 * (b & 3));
            x = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
        if (a < jhi) {
            s_txt[(4 * u + 0) * SMALL_THREADS + tid] = x.x;
            s_txt[(4 * u + 1) * SMALL_THREADS + tid] = x.y;
            s_txt[(4 * u + 2) * SMALL_THREADS + tid] = x.z;
            s_txt[(4 * u + 3) * SMALL_THREADS + tid] = x.w;
        }
    }
    // the DFA rows (ROWB apart) and the class table, every load in flight
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(T.dfa);
        const uint32_t n16 = nr * 16;
        uint4 v[2];
#pragma unroll
        for (uint32_t u = 0; u < 2; ++u) {
            const uint32_t i = u * SMALL_THREADS + tid;
            if (i < n16) v[u] = __ldg(src + i);
        }
#pragma unroll 1
        for (uint32_t i = 2 * SMALL_THREADS + tid; i < n16; i += SMALL_THREADS) {
            const uint4 x = __ldg(src + i);
            uint2 *dst = reinterpret_cast<uint2 *>(s_dfa + (i >> 4) * ROWB + (i & 15) * 16);
            dst[0] = make_uint2(x.x, x.y);
            dst[1] = make_uint2(x.z, x.w);
        }
#pragma unroll
        for (uint32_t u = 0; u < 2; ++u) {
            const uint32_t i = u * SMALL_THREADS + tid;
            if (i < n16) {
                uint2 *dst = reinterpret_cast<uint2 *>(s_dfa + (i >> 4) * ROWB + (i & 15) * 16);
                dst[0] = make_uint2(v[u].x, v[u].y);
                dst[1] = make_uint2(v[u].z, v[u].w);
            }
        }
        if (tid < 16) reinterpret_cast<uint4 *>(s_cls)[tid] = __ldg(reinterpret_cast<const uint4 *>(T.cls) + tid);
    }
    __syncthreads();

    // pass 1: the chunk from f_I, one word (4 bytes) per iteration
    Chain ch;
    ch.f = T.ident;
    ch.cnt = 0;
    ch.snap = 0;
    ch.lm = -1;
    const uint32_t kend = (jhi + 3) >> 2;
#pragma unroll 1
    for (uint32_t k = jlo >> 2; k < kend; ++k) {
        const uint32_t x = s_txt[k * SMALL_THREADS + tid];
#pragma unroll
        for (uint32_t b = 0; b < 4; ++b) {
            const uint32_t j = 4 * k + b;
            if (j >= jlo && j < jhi) sfa_step<false>(ch, (x >> (8 * b)) & 0xffu, (int32_t)j, R, s_cls, T.nc, nr, T.ncls, A);
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

    // group (warp) summaries: a constant, or a |Q|-vector with lanes over states
    // (the chunks of threads past the end of the text are f_I, which every
    // composition below skips)
    auto amap = [&](uint32_t f, uint32_t v) -> uint32_t { return f == T.ident ? v : apply_map(f, v, T.maps, nr); };
    const uint32_t cm = __ballot_sync(0xffffffffu, fl < nr);
    if (cm) {
        const int lc = 31 - __clz(cm);
        uint32_t v = __shfl_sync(0xffffffffu, fl, lc);
#pragma unroll 1
        for (int i = lc + 1; i < 32; ++i) v = amap(__shfl_sync(0xffffffffu, fl, i), v);
        if (lane == 0) s_gval[warp] = v;
    } else {
#pragma unroll 1
        for (uint32_t qb = 0; qb < nr; qb += 32) {
            const uint32_t q = qb + lane;
            uint32_t v = q < nr ? q : 0u;
#pragma unroll 1
            for (int i = 0; i < 32; ++i) v = amap(__shfl_sync(0xffffffffu, fl, i), v);
            if (q < nr) s_gvec[(size_t)warp * nr + q] = (uint8_t)v;
        }
        if (lane == 0) s_gval[warp] = 0xffffffffu;   // marks a vector group
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
    }
    __syncthreads();
    // exclusive prefix of every group (warp 0): the nearest constant group
    // below it, then the vector groups in between
    if (warp == 0 && lane < G) {
        uint32_t below = 0;
#pragma unroll 1
        for (int g = 0; g < lane; ++g)
            if (s_gval[g] != 0xffffffffu) below |= 1u << g;
        int j;
        uint32_t v;
        if (below) {
            j = 31 - __clz(below);
            v = s_gval[j];
        } else {
            j = -1;
            v = s_misc[0];
        }
#pragma unroll 1
        for (int g = j + 1; g < lane; ++g) v = s_gvec[(size_t)g * nr + v];
        s_gpre[lane] = v;
    }
    __syncthreads();

    // entering state of this chunk, pass 2 from shared memory, the state after it
    const uint32_t below = cm & lanemask_lt;
    const int jc = below ? 31 - __clz(below) : -1;
    uint32_t v = __shfl_sync(0xffffffffu, fl, jc < 0 ? 0 : jc);
    if (jc < 0) v = s_gpre[warp];
#pragma unroll 1
    for (int i = jc + 1; i < lane; ++i) v = amap(s_f[warp * 32 + i], v);
    unsigned long long cnt = ch.cnt;
    if (ch.lm >= 0) {
        const uint32_t lm = (uint32_t)ch.lm;
        uint32_t q = v, c = 0;
#pragma unroll 1
        for (uint32_t k = jlo >> 2; 4 * k <= lm; ++k) {
            const uint32_t x = s_txt[k * SMALL_THREADS + tid];
#pragma unroll
            for (uint32_t b = 0; b < 4; ++b) {
                const uint32_t j = 4 * k + b;
                if (j >= jlo && j <= lm) {
                    q = R.next(q, (x >> (8 * b)) & 0xffu);
                    c += q >= A;
                }
            }
        }
        cnt = c + chunk_count_after(ch, v, ps, T);
    }
    if (tid == SMALL_THREADS - 1) s_misc[2] = amap(fl, v);   // the state after the text
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_red[warp] = cnt;
    __syncthreads();
    if (tid == 0) {
        unsigned long long total = 0;
#pragma unroll 1
        for (int g = 0; g < G; ++g) total += s_red[g];
        const uint32_t fin = s_misc[2];
        sfa_result r;
        r.final_state = (uint32_t)T.orig_of[fin < nr ? fin : 0];
        r.accept_final = fin >= A ? 1 : 0;
        r.status = s_misc[1] ? SFA_STATUS_TIMEOUT : SFA_STATUS_OK;
        r.reserved = 0;
        r.count = (carry ? out->count : 0ull) + total;
        *out = r;
    }
}

}  // namespace sfa_dev

namespace sfa_impl {

bool small_fits(uint64_t n) { return n <= (uint64_t)sfa_dev::SMALL_THREADS * sfa_dev::SMALL_CHUNK; }

size_t small_smem(uint32_t nr) { return sfa_dev::SmallLayout::bytes(nr); }

int launch_small(const sfa_dev::Tables &T, const uint8_t *text, uint64_t n, bool carry, sfa_result *out,
                 cudaStream_t s) {
    if (!small_fits(n) || T.nr > 255) return SFA_ERR_UNSUPPORTED;
    // chunk bodies from the first 16-byte boundary, in 16-byte multiples
    const uint32_t origin = n ? sfa_dev::text_origin(text) : 0u;
    const uint64_t body = n > origin ? n - origin : 0;
    uint32_t chunk = (uint32_t)((body + sfa_dev::SMALL_THREADS - 1) / sfa_dev::SMALL_THREADS);
    chunk = std::max<uint32_t>(16, (chunk + 15) & ~15u);
    if (chunk > (uint32_t)sfa_dev::SMALL_CHUNK) return SFA_ERR_UNSUPPORTED;
    static const bool attr = [] {
        int dev = 0;
        cudaGetDevice(&dev);
        return cudaFuncSetAttribute(reinterpret_cast<const void *>(&sfa_dev::sfa_small_kernel),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)device_props(dev).smem_optin) == cudaSuccess;
    }();
    if (!attr) return SFA_ERR_CUDA;
    const size_t smem = small_smem(T.nr);
    sfa_dev::sfa_small_kernel<<<1, sfa_dev::SMALL_THREADS, smem, s>>>(T, text, n, chunk, origin, carry ? 1u : 0u, out);
    CK(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return SFA_OK;
}

}  // namespace sfa_impl
