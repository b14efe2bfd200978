// Numbering of the kept DFA states against shared-memory bank conflicts (no
// CUDA in this unit).
//
// The kernel keeps the kept DFA in shared memory, row q at q * ROWB: a lane in
// state q that reads byte b touches the 4-byte word (ROWB/4) q + b/4, in bank
// ((ROWB/4) q + b/4) mod 32, and a warp's lookup takes as many wavefronts as
// the largest number of distinct words any one bank gets.  Which lanes sit in
// which states is a property of the automaton and the text, so the state ids
// -- free up to "final states last" -- decide how many of those collide.
//
// The search models lanes: LANES lanes run the DFA over a text source (a
// caller's sample, else bytes drawn uniformly from the bytes whose column is
// not constant, i.e. the bytes that can change a state's fate) for WARM bytes
// from q0, then STEPS bytes are recorded; each step of 32 consecutive lanes is
// one warp's lookup.  Its cost is the mean of the per-lookup wavefront counts.
// A local search then swaps the ids of two states of the same kind (both
// final or both not), one of them among the most visited states, keeping a
// swap only if the modelled cost falls.  Every numbering is exact (the
// matching results do not depend on it); only the speed does.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "host_compile.h"
#include "sfa_types.h"

namespace sfa_impl {

namespace {

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

constexpr int LANES = 256, STEPS = 300, WARM = 64, HOT = 32, ITERS = 1000;

}  // namespace

std::vector<int32_t> bank_numbering(const std::vector<uint8_t> &dfa, int nr, int first_accept, int q0,
                                    const uint8_t *sample, uint64_t sample_len) {
    std::vector<int32_t> id(nr);
    std::iota(id.begin(), id.end(), 0);
    if (nr < 3) return id;
    const uint32_t stride = (uint32_t)(sfa_dev::ROWB / 4) & 31u;   // bank step from one row to the next
    auto bank = [&](int32_t i, uint32_t w) -> uint32_t { return (stride * (uint32_t)i + w) & 31u; };

    // text source
    std::vector<uint8_t> sig;
    for (int b = 0; b < 256; ++b) {
        bool varies = false;
        for (int q = 1; q < nr && !varies; ++q) varies = dfa[(size_t)q * 256 + b] != dfa[b];
        if (varies) sig.push_back((uint8_t)b);
    }
    const bool from_sample = sample && sample_len >= 4ull * (WARM + STEPS);
    if (sig.empty() && !from_sample) return id;
    uint64_t rng = 0x1405056215ull;

    // lanes: the state and the word within the row of every lookup
    std::vector<uint16_t> st((size_t)STEPS * LANES);
    std::vector<uint8_t> wd((size_t)STEPS * LANES);
    for (int l = 0; l < LANES; ++l) {
        uint64_t pos = from_sample ? splitmix64(rng) % (sample_len - WARM - STEPS) : 0;
        auto next = [&]() -> uint8_t { return from_sample ? sample[pos++] : sig[splitmix64(rng) % sig.size()]; };
        int q = q0;
        for (int j = 0; j < WARM; ++j) q = dfa[(size_t)q * 256 + next()];
        for (int j = 0; j < STEPS; ++j) {
            const uint8_t b = next();
            st[(size_t)j * LANES + l] = (uint16_t)q;
            wd[(size_t)j * LANES + l] = (uint8_t)(b >> 2);
            q = dfa[(size_t)q * 256 + b];
        }
    }

    // warps: the distinct (state, word) pairs of each lookup (two lanes on one
    // pair read one word, a broadcast), listed per state for the updates
    const int G = STEPS * LANES / 32;
    struct Entry {
        uint32_t g;
        uint8_t w;
    };
    std::vector<std::vector<Entry>> of(nr);
    std::vector<uint8_t> hist((size_t)G * 32, 0), gmax(G, 0);
    {
        uint32_t keys[32];
        for (int g = 0; g < G; ++g) {
            const size_t base = (size_t)(g / (LANES / 32)) * LANES + (size_t)(g % (LANES / 32)) * 32;
            for (int i = 0; i < 32; ++i) keys[i] = (uint32_t)st[base + i] << 8 | wd[base + i];
            std::sort(keys, keys + 32);
            for (int i = 0; i < 32; ++i) {
                if (i && keys[i] == keys[i - 1]) continue;
                const int q = (int)(keys[i] >> 8);
                const uint8_t w = (uint8_t)(keys[i] & 0xffu);
                of[q].push_back({(uint32_t)g, w});
                ++hist[(size_t)g * 32 + bank(id[q], w)];
            }
        }
    }
    auto group_max = [&](uint32_t g) -> uint8_t {
        const uint8_t *h = &hist[(size_t)g * 32];
        uint8_t m = 0;
        for (int b = 0; b < 32; ++b) m = std::max(m, h[b]);
        return m;
    };
    int64_t cost = 0;
    for (int g = 0; g < G; ++g) cost += gmax[g] = group_max((uint32_t)g);

    // the most visited states, and the states of each kind
    std::vector<int> hot(nr);
    std::iota(hot.begin(), hot.end(), 0);
    std::stable_sort(hot.begin(), hot.end(), [&](int a, int b) { return of[a].size() > of[b].size(); });
    int nhot = 0;
    while (nhot < std::min(nr, HOT) && !of[hot[nhot]].empty()) ++nhot;
    if (nhot == 0) return id;

    std::vector<uint32_t> stamp(G, 0), touched;
    std::vector<uint8_t> newmax(G, 0);
    uint32_t epoch = 0;
    auto move = [&](int q, int32_t from, int32_t to) {
        for (const Entry &e : of[q]) {
            --hist[(size_t)e.g * 32 + bank(from, e.w)];
            ++hist[(size_t)e.g * 32 + bank(to, e.w)];
        }
    };
    for (int it = 0; it < ITERS; ++it) {
        const int s = hot[splitmix64(rng) % (uint64_t)nhot];
        const bool fin = s >= first_accept;
        const int lo = fin ? first_accept : 0, hi = fin ? nr : first_accept;
        if (hi - lo < 2) continue;
        const int o = lo + (int)(splitmix64(rng) % (uint64_t)(hi - lo));
        if (o == s || bank(id[s], 0) == bank(id[o], 0)) continue;
        const int32_t is = id[s], io = id[o];
        move(s, is, io);
        move(o, io, is);
        ++epoch;
        touched.clear();
        for (int q : {s, o})
            for (const Entry &e : of[q])
                if (stamp[e.g] != epoch) {
                    stamp[e.g] = epoch;
                    touched.push_back(e.g);
                }
        int64_t delta = 0;
        for (uint32_t g : touched) {
            newmax[g] = group_max(g);
            delta += (int64_t)newmax[g] - gmax[g];
        }
        if (delta < 0) {
            for (uint32_t g : touched) gmax[g] = newmax[g];
            cost += delta;
            id[s] = io;
            id[o] = is;
        } else {
            move(s, io, is);
            move(o, is, io);
        }
    }
    return id;
}

}  // namespace sfa_impl
