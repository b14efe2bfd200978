// Data layouts shared by the host launcher and the kernels: table and text
// descriptors, per-launch scratch, shared-memory layout of a CTA.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define SFA_HD __host__ __device__
#else
#define SFA_HD
#endif

namespace sfa_dev {

// A non-constant row entry: next id | acceptance class << 30.  On the device
// an entry whose target is a point mapping {s -> p, every other q -> sink}
// (sink: an absorbing non-final state) carries NC_POINT | s << 8 | p instead
// of the id: the chunk then follows p through the DFA rows (one shared-memory
// lookup per byte) until it ends or p falls into the sink.
constexpr uint32_t NC_ID_MASK = 0x1fffffffu;
constexpr uint32_t NC_POINT = 1u << 29;
// With NC_POINT, NC_SET marks a set-point mapping {q in S -> p, every other
// q -> sink} (|S| >= 2): the source field holds the id of the set S (a row
// of Tables::setbits) instead of a state.
constexpr uint32_t NC_SET = 1u << 28;
constexpr uint32_t NO_SINK = 0xffffffffu;
constexpr uint32_t NO_POINT = 0xffffffffu;   // a chunk's point source: none (0xffff when kept in 16 bits)
constexpr uint32_t PS_SET = 0x8000u;         // a kept point source that is a set id
constexpr uint32_t ACC_ALL = 1, ACC_MIXED = 2;

// look-back descriptor: flag in bits 62..63, value (a kept DFA state) below
constexpr uint64_t ST_AGG = 1ull << 62;
constexpr uint64_t ST_PREFIX = 2ull << 62;

struct Tables {
    const uint8_t *dfa;        // [nr*256]     kept DFA, final states last
    const uint8_t *cls;        // [256]        byte -> class
    const uint32_t *nc;        // [n_nc*ncls]  non-constant SFA rows
    const uint8_t *maps;       // [n_nc*nr]    mappings of non-constant states
    const int32_t *orig_of;    // [nr]
    const int32_t *kept_of;    // [nq_in]
    const uint32_t *pid;       // [nr*nr] id of the point mapping {s -> p} at s*nr + p (sink != NO_SINK)
    const uint32_t *setbits;   // [n_sets*set_words] the source set of each set-point id, bit q of q
    const uint32_t *spid;      // byte ids: [n_sets*nr] id of the set-point mapping {S -> p} at sid*nr + p
    uint32_t set_words;        // 32-bit words per set: (nr + 31) / 32
    // more than 256 kept states (16-bit ids): dfa and maps are unused
    const uint16_t *cdfa;      // [nr*ncls] kept DFA over byte classes
    const uint16_t *maps16;    // [n_nc*nr]  stored non-constant mappings
    uint32_t nr, ncls, first_accept, q0, ident, nq_in, mode;
    uint32_t sink;             // the sink of the point mappings, or NO_SINK
};

struct TextDesc {
    const uint8_t *text;
    uint64_t n;
    uint64_t chunk;            // bytes per chunk when forced == 0 (level A)
    const void *map;           // batches: this text's tensor map in device
                               // memory (NULL: the kernel's parameter)
    // Two levels (split_tile != 0): tiles [0, split_tile) cover [0, split)
    // in chunks of `chunk` bytes, the others [split, n) in chunks of
    // chunk_b bytes, rows of the kernel's second tensor map (rows2d_b full
    // ones).  split_tile == 0: one level, [0, n) in chunks of `chunk`.
    uint64_t split;
    uint64_t chunk_b;
    uint32_t split_tile;
    uint32_t rows2d_b;
    uint32_t forced;           // exact number of chunks, or 0
    uint32_t ntiles;
    uint32_t tile_base;        // first global tile of the text
    uint32_t table;            // index into the table array (batches)
    uint32_t out_index;
    uint32_t carry;            // 1: continue from out[out_index] (Lemma 1)
    uint32_t rows2d;           // chunks [0, rows2d) are rows of the kernel's
                               // tensor map (their bodies: full chunks that
                               // start on a 16-byte boundary); 0: no map
    // bytes before the text's first 16-byte boundary (0 with forced chunk
    // counts): level A's chunk 0 is [0, origin + chunk), chunk k >= 1 is
    // [origin + k*chunk, origin + (k+1)*chunk), so that every chunk body
    // starts on a 16-byte boundary (Theorem 3: any division of the text
    // gives the same result)
    uint32_t origin;
};

struct TextState {             // zeroed before each launch
    unsigned long long count;
    uint32_t done;
    uint32_t final_state;
    uint32_t err;
    uint32_t pad[3];
};

struct LaunchHeader {          // zeroed before each launch
    uint32_t tile_ctr;         // next tile (two levels: next level-A tile)
    uint32_t err;
    uint32_t tile_ctr_b;       // two levels: next level-B tile
    uint32_t pad[13];
    uint32_t sm_slot[256];     // two levels: CTAs started so far on each SM
};

struct Scratch {
    LaunchHeader *hdr;
    TextState *texts;
    uint64_t *status;          // [total tiles]
    uint8_t *agg;              // [total tiles * nr_max]   tile aggregates
    uint8_t *chainvec;         // [total tiles * CPT * nr]  chunk vectors (simulation only)
    uint32_t nr_max;
    uint32_t timeout_us;
    uint32_t debug;
    uint32_t total_tiles;
    uint32_t map_mode;         // 1: every tile leaves its aggregate as a
                               // |Q|-vector in agg (constant tiles too), for
                               // the slice mapping of sfa_match_map
    uint32_t single;           // 1: one text of one tile on one CTA; the CTA
                               // clears the error words itself and takes
                               // tile 0 without the counter, so the launch
                               // needs no zeroed scratch
};

// chunks of a one-level text (the empty text, and one shorter than its
// origin, have one chunk)
SFA_HD inline uint64_t num_chunks(const TextDesc &d) {
    if (d.forced) return d.forced;
    const uint64_t body = d.n > d.origin ? d.n - d.origin : 0;
    uint64_t c = (body + d.chunk - 1) / d.chunk;
    return c ? c : 1;
}

// the origin of a text that starts at p
SFA_HD inline uint32_t text_origin(const uint8_t *p) {
    return (uint32_t)((16u - ((uint32_t)(uintptr_t)p & 15u)) & 15u);
}

// ---------------------------------------------------------------------------
// shared memory of one CTA
// ---------------------------------------------------------------------------
// DFA rows in shared memory are ROWB = 264 bytes apart: byte b of state q sits
// in bank (2q + b/4) mod 32, so lanes reading the same byte value in different
// states hit different banks (a 256-byte stride would put them all in one),
// and the few words a small alphabet uses in each row spread over all 32
// banks (a 260-byte stride, bank (q + b/4) mod 32, crowds neighbouring
// states into neighbouring banks: a bank-conflict model of the lanes of the
// workloads counts 1.95 instead of 1.98 wavefronts per lookup for literal
// automata on base64 text, 2.0 instead of 3.2 for 16-state automata over 16
// symbols).
constexpr uint32_t ROWB = 264;
// Text staging, SLICE bytes of every chunk per step, STAGES steps in flight.
// For each warp, stage and round of chunks there is a BOX of 32 rows x SLICE
// bytes: one 2-D tensor copy fills it with the next slice of the warp's 32
// chunks (rows of the text viewed as [chunk][chunk length]), 64-byte
// swizzled, so that 16-byte reads of 8 consecutive lanes hit distinct banks.
// Chunks that are not a full row (the text's ragged last chunk) take a 1-D
// bulk copy into the EXTRA row of the warp instead; without a tensor map
// (forced chunk counts, chunk lengths that are not multiples of 16) every
// lane copies its own slice into its row of the box, unswizzled.  After
// pass 1 the EXTRA rows hold each chunk's point source for pass 2.
constexpr int SLICE = 64;
constexpr int STAGES = 2;
constexpr int BOX = 32 * SLICE;
static_assert(SLICE == 64, "the read pattern assumes the 64-byte swizzle");

// WIDE: 16-bit state ids; the DFA rows are indexed by byte class (ncls
// 16-bit entries per state) and the group vectors hold 16-bit states.  Every
// offset takes the table's state count nr_max and, for WIDE, its class count.
template <int THREADS, int CH, int SIMNQ = 0, bool WIDE = false>
struct SmemLayout {
    static constexpr int CPT = THREADS * CH;   // chunks per tile
    static constexpr int NW = THREADS / 32;
    static constexpr int G = CPT / 32;         // groups per tile
    static constexpr size_t IDB = WIDE ? 2 : 1;   // bytes per state id
    static_assert(G <= 32, "at most 1024 chunks per tile");
    // offsets in bytes from the start of dynamic shared memory
    static SFA_HD size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static SFA_HD size_t dfa_off() { return 0; }
    static SFA_HD size_t cls_off(uint32_t nr_max, uint32_t ncls = 0) {
        return a16(WIDE ? (size_t)nr_max * ncls * 2 : (size_t)nr_max * ROWB);
    }
    static SFA_HD size_t f_off(uint32_t nr_max, uint32_t ncls = 0) { return cls_off(nr_max, ncls) + 256; }
    static SFA_HD size_t gval_off(uint32_t nr_max, uint32_t ncls = 0) { return f_off(nr_max, ncls) + CPT * 4; }
    static SFA_HD size_t gpre_off(uint32_t nr_max, uint32_t ncls = 0) { return gval_off(nr_max, ncls) + 32 * 4; }
    static SFA_HD size_t misc_off(uint32_t nr_max, uint32_t ncls = 0) { return gpre_off(nr_max, ncls) + 32 * 4; }
    static SFA_HD size_t gvec_off(uint32_t nr_max, uint32_t ncls = 0) { return misc_off(nr_max, ncls) + 512; }
    static SFA_HD size_t bar_off(uint32_t nr_max, uint32_t ncls = 0) {
        return a16(gvec_off(nr_max, ncls) + (size_t)G * nr_max * IDB);
    }
    // boxes: [warp][stage][round] x BOX, 1024-byte aligned (the swizzle
    // pattern repeats every 512 bytes); extra rows: [warp][stage][round] x SLICE
    static SFA_HD size_t stage_off(uint32_t nr_max, uint32_t ncls = 0) {
        return (bar_off(nr_max, ncls) + (size_t)NW * STAGES * 8 + 1023) & ~(size_t)1023;
    }
    static SFA_HD size_t extra_off(uint32_t nr_max, uint32_t ncls = 0) {
        return stage_off(nr_max, ncls) + (size_t)NW * STAGES * CH * BOX;
    }
    // simulation vectors of more than 64 entries: SIMNQ bytes per chunk,
    // [round][warp][word][lane] (see SimChain)
    static SFA_HD size_t vec_off(uint32_t nr_max, uint32_t ncls = 0) {
        return a16(extra_off(nr_max, ncls) + (size_t)NW * STAGES * CH * SLICE);
    }
    static SFA_HD size_t bytes(uint32_t nr_max, uint32_t ncls = 0) {
        return vec_off(nr_max, ncls) + (SIMNQ > 64 ? (size_t)CPT * SIMNQ : 0);
    }
};

struct Misc {
    uint32_t tile;          // global tile being processed
    uint32_t gconst;        // bit g: group g is a constant mapping
    uint32_t s_in;          // entering state of the tile
    uint32_t incl;          // state after the tile
    // thread 0: a tile whose first chunk's recount is deferred (valid != 0)
    uint32_t dfr_gt, dfr_ti, dfr_valid;
    int32_t dfr_lm;
    unsigned long long dfr_lo;
    unsigned long long pad;
    unsigned long long wsum[32];
};
static_assert(sizeof(Misc) <= 512, "misc region");

}  // namespace sfa_dev
