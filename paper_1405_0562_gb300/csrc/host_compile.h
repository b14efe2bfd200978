// Host-side construction of the D-SFA tables (no CUDA in this unit).
#pragma once

#include <cstdint>
#include <vector>

namespace sfa_impl {

// acceptance class of a mapping f over the kept states: whether f(q) is final
// for no q, for every q, or for some q only ("mixed")
enum AccClass : uint32_t { ACC_NONE = 0, ACC_ALL = 1, ACC_MIXED = 2 };

constexpr uint32_t NC_ID_MASK = 0x1fffffffu;   // bit 29 is the device's point flag
constexpr uint32_t NC_POINT = 1u << 29;
constexpr uint32_t NC_SET = 1u << 28;           // with NC_POINT: the source field is a set id
constexpr int NC_ACC_SHIFT = 30;
constexpr uint32_t DEFAULT_CAP = 65536;
constexpr int SIM_MAX_STATES = 256;
constexpr int NARROW_MAX_STATES = 256;         // byte-wide state ids
constexpr int WIDE_MAX_STATES = 4095;          // 16-bit ids; a point entry holds two 12-bit states
constexpr int WIDE_POINT_SHIFT = 12;

struct HostTables {
    int32_t nq_in = 0;             // states given by the caller
    int32_t nr = 0;                // states reachable from q0 (kept)
    int32_t q0 = 0;                // kept numbering
    int32_t first_accept = 0;      // kept ids [first_accept, nr) are final
    int32_t ncls = 0;              // byte classes
    uint8_t cls[256] = {};         // class of each byte
    std::vector<int32_t> orig_of;  // [nr]     caller id of a kept state
    std::vector<int32_t> kept_of;  // [nq_in]  kept id of a caller state, -1 if unreachable
    std::vector<uint8_t> dfa;      // [nr*256] kept DFA over bytes
    int32_t mode = 0;              // SFA_MODE_SFA or SFA_MODE_SIM
    uint32_t ident = 0;            // D-SFA id of f_I (nr when nr > 1, else 0)
    uint64_t n_nc = 0;             // non-constant D-SFA states
    std::vector<uint32_t> nc;      // [n_nc*ncls] next id | acc class of next << 30
    std::vector<uint8_t> maps;     // [n_nc*nr]   f(q) of each non-constant state
    uint64_t n_const = 0;          // constant mappings reachable from f_I
    double seconds = 0.0;
    // More than 256 kept states ("wide"): 16-bit ids, a class-indexed DFA,
    // and point mappings {s -> p, every other state -> sink} never stored:
    // a row entry whose target is one carries NC_POINT | s << 12 | p.  The
    // u8 tables above (dfa, maps) are then empty.
    bool wide = false;
    int32_t sink = -1;             // wide: the absorbing non-final state, or -1
    std::vector<uint16_t> cdfa;    // wide: [nr*ncls] kept DFA over classes
    std::vector<uint16_t> maps16;  // wide: [n_nc*nr] f(q) of each stored non-constant state
    uint64_t n_points = 0;         // wide: point and set-point mappings reachable from f_I (not stored)
    // wide: the source sets of the set-point mappings {q in S -> p, others ->
    // sink} (|S| >= 2; entries NC_POINT | NC_SET | sid << 12 | p), bit q of
    // set sid at setbits[sid * set_words + q / 32]
    std::vector<uint32_t> setbits;
    uint32_t set_words = 0;
};

// Returns SFA_OK or an SFA_ERR_* code (see sfa.h for the rules).  tune_banks:
// number the kept states against shared-memory bank conflicts, modelled on
// `sample` (host bytes) when it is long enough, else on bytes drawn uniformly
// from the bytes that can change a state.
int build_tables(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                 uint32_t cap, int32_t force_mode, HostTables &out, bool tune_banks = false,
                 const uint8_t *sample = nullptr, uint64_t sample_len = 0);

// The search of bank_layout.cpp: new id of every kept id (a permutation that
// keeps [0, first_accept) and [first_accept, nr) in place as sets).
std::vector<int32_t> bank_numbering(const std::vector<uint8_t> &dfa, int nr, int first_accept, int q0,
                                    const uint8_t *sample, uint64_t sample_len);

}  // namespace sfa_impl
