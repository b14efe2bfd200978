// D-SFA construction on the host: Alg. 4 (correspondence construction) with
// the DFA simplification of Sect. V-A, f_next(q) = delta(f(q), sigma).
//
// Steps (all exact, none changes a match result):
//  1. validate the DFA (Sect. II-B: total table, one initial state);
//  2. keep the states reachable from q0 -- every state a chunk can be
//     entered in is one of them -- and renumber them so that the final
//     states are the ids [first_accept, nr); within each kind the ids are
//     then chosen against shared-memory bank conflicts (bank_layout.cpp);
//  3. merge bytes whose columns of delta are equal into classes (the
//     alphabet Sigma of Alg. 4 becomes the set of classes);
//  4. breadth-first correspondence construction from f_I over the classes,
//     with a FIFO worklist.  Constant mappings q -> c are not stored as
//     rows of their own: their SFA transition is c . delta^sigma, the
//     constant onto delta(c, sigma), i.e. the DFA row of c.  They get the
//     ids 0..nr-1 (the id is the constant's value) and the DFA table serves
//     as their part of the transition table.  Non-constant mappings get ids
//     nr, nr+1, ... in discovery order;
//  5. past `cap` non-constant mappings the handle uses the simulation path
//     of Alg. 3 instead (Theorem 2 bounds the D-SFA only by nr^nr).
#include "host_compile.h"

#include <chrono>
#include <cstring>
#include <string>
#include <unordered_map>

#include "sfa.h"

namespace sfa_impl {

namespace {

struct VecHash {
    size_t operator()(const std::string &s) const noexcept {
        // 64-bit FNV-1a over the mapping bytes
        uint64_t h = 0xcbf29ce484222325ull;
        for (unsigned char c : s) {
            h ^= c;
            h *= 0x100000001b3ull;
        }
        return (size_t)h;
    }
};

uint32_t acc_class(const uint8_t *f, int nr, int first_accept) {
    bool any = false, all = true;
    for (int q = 0; q < nr; ++q) {
        bool fin = f[q] >= first_accept;
        any |= fin;
        all &= fin;
    }
    return all ? ACC_ALL : (any ? ACC_MIXED : ACC_NONE);
}

}  // namespace

namespace {

// Steps 2-4 for more than 256 kept states: 16-bit ids over byte classes, and
// point mappings {s -> p, all other states -> z}, for an absorbing non-final
// state z, kept implicit: Alg. 4 does not enqueue them (their successors are
// again point mappings, or the constant z, one DFA step of p away), and a
// row entry whose target is one carries NC_POINT | s << 12 | p.  Only the
// other non-constant mappings are stored (cap applies to them).  The states
// reachable from f_I are still all counted: the stored ones, the point
// mappings (pairs (s, p) closed under p -> delta(p, sigma)) and the constants.
// There is no simulation path for such automata (UNSUPPORTED past the cap).
int build_wide(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept, uint32_t cap,
               const std::vector<int32_t> &order, HostTables &T, std::chrono::steady_clock::time_point t0) {
    const int nr = (int)order.size();
    T.nq_in = nq;
    T.nr = nr;
    T.wide = true;
    T.mode = SFA_MODE_SFA;
    T.orig_of.clear();
    for (int32_t s : order)
        if (!accept[s]) T.orig_of.push_back(s);
    T.first_accept = (int32_t)T.orig_of.size();
    for (int32_t s : order)
        if (accept[s]) T.orig_of.push_back(s);
    T.kept_of.assign(nq, -1);
    for (int32_t i = 0; i < nr; ++i) T.kept_of[T.orig_of[i]] = i;
    T.q0 = T.kept_of[q0];
    T.dfa.clear();
    T.maps.clear();
    std::vector<uint16_t> d16((size_t)nr * 256);
    for (int i = 0; i < nr; ++i)
        for (int b = 0; b < 256; ++b) d16[(size_t)i * 256 + b] = (uint16_t)T.kept_of[delta[(int64_t)T.orig_of[i] * 256 + b]];
    // byte classes: equal columns of the kept table
    {
        std::unordered_map<std::string, int, VecHash> cols;
        std::string col(2 * (size_t)nr, '\0');
        T.ncls = 0;
        for (int b = 0; b < 256; ++b) {
            for (int i = 0; i < nr; ++i) std::memcpy(&col[2 * (size_t)i], &d16[(size_t)i * 256 + b], 2);
            auto it = cols.find(col);
            if (it == cols.end()) it = cols.emplace(col, T.ncls++).first;
            T.cls[b] = (uint8_t)it->second;
        }
    }
    const int ncls = T.ncls;
    std::vector<uint8_t> rep(ncls);
    for (int b = 255; b >= 0; --b) rep[T.cls[b]] = (uint8_t)b;
    T.cdfa.assign((size_t)nr * ncls, 0);
    for (int i = 0; i < nr; ++i)
        for (int c = 0; c < ncls; ++c) T.cdfa[(size_t)i * ncls + c] = d16[(size_t)i * 256 + rep[c]];
    // the sink: an absorbing non-final kept state
    T.sink = -1;
    for (int q = 0; q < T.first_accept && T.sink < 0; ++q) {
        bool absorbing = true;
        for (int c = 0; c < ncls && absorbing; ++c) absorbing = T.cdfa[(size_t)q * ncls + c] == q;
        if (absorbing) T.sink = q;
    }
    const int z = T.sink;
    // Alg. 4 over the stored (neither constant nor point) mappings
    T.ident = (uint32_t)nr;
    T.n_nc = 0;
    T.nc.clear();
    T.maps16.clear();
    std::unordered_map<std::string, uint32_t, VecHash> ids;
    std::string g(2 * (size_t)nr, '\0');
    std::vector<uint16_t> gv(nr);
    // source sets of set-point mappings (at most 4096: the id is 12 bits)
    T.set_words = ((uint32_t)nr + 31) / 32;
    T.setbits.clear();
    std::unordered_map<std::string, uint32_t, VecHash> set_ids;
    std::vector<uint32_t> sbits(T.set_words);
    for (int q = 0; q < nr; ++q) gv[q] = (uint16_t)q;
    T.maps16.insert(T.maps16.end(), gv.begin(), gv.end());
    ids.emplace(std::string(reinterpret_cast<const char *>(gv.data()), 2 * (size_t)nr), 0);
    T.n_nc = 1;
    for (uint64_t head = 0; head < T.n_nc; ++head) {
        for (int c = 0; c < ncls; ++c) {
            const uint16_t *fm = T.maps16.data() + head * nr;
            int live = 0, src = -1, img = -1;
            bool constant = true, one_image = true;
            std::fill(sbits.begin(), sbits.end(), 0u);
            for (int q = 0; q < nr; ++q) {
                gv[q] = T.cdfa[(size_t)fm[q] * ncls + c];
                constant &= gv[q] == gv[0];
                if ((int)gv[q] != z) {
                    ++live;
                    src = q;
                    one_image &= img < 0 || (int)gv[q] == img;
                    img = gv[q];
                    sbits[q >> 5] |= 1u << (q & 31);
                }
            }
            uint32_t e = 0;
            bool set_point = false;
            if (!constant && z >= 0 && live >= 2 && one_image) {
                const std::string key(reinterpret_cast<const char *>(sbits.data()), sbits.size() * 4);
                auto it = set_ids.find(key);
                if (it == set_ids.end() && set_ids.size() < (1u << WIDE_POINT_SHIFT)) {
                    it = set_ids.emplace(key, (uint32_t)set_ids.size()).first;
                    T.setbits.insert(T.setbits.end(), sbits.begin(), sbits.end());
                }
                if (it != set_ids.end()) {
                    e = NC_POINT | NC_SET | it->second << WIDE_POINT_SHIFT | (uint32_t)img;
                    set_point = true;
                }
            }
            if (set_point) {
            } else if (constant) {
                e = gv[0];
            } else if (z >= 0 && live == 1) {
                e = NC_POINT | (uint32_t)src << WIDE_POINT_SHIFT | gv[src];
            } else {
                std::memcpy(&g[0], gv.data(), 2 * (size_t)nr);
                auto it = ids.find(g);
                if (it == ids.end()) {
                    if (T.n_nc >= cap) return SFA_ERR_UNSUPPORTED;
                    it = ids.emplace(g, (uint32_t)T.n_nc).first;
                    T.maps16.insert(T.maps16.end(), gv.begin(), gv.end());
                    ++T.n_nc;
                }
                e = (uint32_t)nr + it->second;
            }
            T.nc.push_back(e);
        }
    }
    // acceptance class of each target (point mappings: none, the kernel
    // follows their live state instead)
    for (uint32_t &e : T.nc) {
        if (e & NC_POINT) continue;
        const uint32_t id = e;
        uint32_t a;
        if (id < (uint32_t)nr) {
            a = (int)id >= T.first_accept ? ACC_ALL : ACC_NONE;
        } else {
            const uint16_t *f = T.maps16.data() + (size_t)(id - nr) * nr;
            bool any = false, all = true;
            for (int q = 0; q < nr; ++q) {
                const bool fin = f[q] >= T.first_accept;
                any |= fin;
                all &= fin;
            }
            a = all ? ACC_ALL : (any ? ACC_MIXED : ACC_NONE);
        }
        e = id | (a << NC_ACC_SHIFT);
    }
    // reachable constants and point mappings
    std::vector<char> creach(nr, 0);
    std::vector<int> cstack;
    auto cmark = [&](int c) {
        if (!creach[c]) {
            creach[c] = 1;
            cstack.push_back(c);
        }
    };
    // point mappings (s, p) and set-point mappings (S, p): pairs closed
    // under p -> delta(p, sigma) (or the constant sink)
    const size_t nsets = T.set_words ? T.setbits.size() / T.set_words : 0;
    const size_t npair = ((size_t)nr + nsets) * nr;   // sources: states, then sets
    std::vector<uint64_t> preach((npair + 63) / 64, 0);
    std::vector<uint64_t> pstack;
    auto pmark = [&](size_t s_, uint32_t p_) {
        const size_t k = s_ * nr + p_;
        if (!(preach[k >> 6] >> (k & 63) & 1)) {
            preach[k >> 6] |= 1ull << (k & 63);
            pstack.push_back(k);
        }
    };
    for (uint32_t e : T.nc) {
        if (e & NC_POINT)
            pmark((e & NC_SET ? (size_t)nr : 0) + ((e >> WIDE_POINT_SHIFT) & 0xfffu), e & 0xfffu);
        else if ((e & NC_ID_MASK) < (uint32_t)nr)
            cmark((int)(e & NC_ID_MASK));
    }
    T.n_points = 0;
    while (!pstack.empty()) {
        const uint64_t k = pstack.back();
        pstack.pop_back();
        ++T.n_points;
        const size_t s_ = k / nr;
        const uint32_t p_ = (uint32_t)(k % nr);
        for (int c = 0; c < ncls; ++c) {
            const uint32_t np = T.cdfa[(size_t)p_ * ncls + c];
            if ((int)np == z) cmark(z);
            else pmark(s_, np);
        }
    }
    while (!cstack.empty()) {
        const int c0 = cstack.back();
        cstack.pop_back();
        for (int c = 0; c < ncls; ++c) cmark(T.cdfa[(size_t)c0 * ncls + c]);
    }
    T.n_const = 0;
    for (char r : creach) T.n_const += r ? 1 : 0;
    T.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SFA_OK;
}

// Steps 1-5 with the kept states numbered breadth first (final states last),
// then renumbered by `renumber` (new id of every such id) when given.
int build_numbered(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept, uint32_t cap,
                   int32_t force_mode, HostTables &T, const std::vector<int32_t> *renumber) {
    auto t0 = std::chrono::steady_clock::now();
    if (!delta || !accept) return SFA_ERR_INVALID;
    if (nq < 1) return SFA_ERR_INVALID;
    if (nq > WIDE_MAX_STATES) return SFA_ERR_UNSUPPORTED;
    if (q0 < 0 || q0 >= nq) return SFA_ERR_INVALID;
    for (int64_t i = 0; i < (int64_t)nq * 256; ++i)
        if (delta[i] < 0 || delta[i] >= nq) return SFA_ERR_INVALID;
    if (force_mode < SFA_MODE_AUTO || force_mode > SFA_MODE_SIM) return SFA_ERR_INVALID;
    if (cap == 0) cap = DEFAULT_CAP;
    if (cap > NC_ID_MASK - 256) cap = NC_ID_MASK - 256;

    // 2. reachable states, breadth first from q0, then final states last
    std::vector<int32_t> order;
    std::vector<char> seen(nq, 0);
    order.push_back(q0);
    seen[q0] = 1;
    for (size_t i = 0; i < order.size(); ++i)
        for (int b = 0; b < 256; ++b) {
            int32_t t = delta[(int64_t)order[i] * 256 + b];
            if (!seen[t]) {
                seen[t] = 1;
                order.push_back(t);
            }
        }
    if ((int)order.size() > NARROW_MAX_STATES) {
        if (force_mode == SFA_MODE_SIM) return SFA_ERR_UNSUPPORTED;
        return build_wide(delta, nq, q0, accept, cap, order, T, t0);
    }
    T.wide = false;
    T.sink = -1;
    T.cdfa.clear();
    T.maps16.clear();
    T.n_points = 0;
    T.nq_in = nq;
    T.nr = (int32_t)order.size();
    T.orig_of.clear();
    for (int32_t s : order)
        if (!accept[s]) T.orig_of.push_back(s);
    T.first_accept = (int32_t)T.orig_of.size();
    for (int32_t s : order)
        if (accept[s]) T.orig_of.push_back(s);
    const int nr = T.nr;
    auto number = [&]() {
        T.kept_of.assign(nq, -1);
        for (int32_t i = 0; i < nr; ++i) T.kept_of[T.orig_of[i]] = i;
        T.q0 = T.kept_of[q0];
        T.dfa.assign((size_t)nr * 256, 0);
        for (int i = 0; i < nr; ++i)
            for (int b = 0; b < 256; ++b)
                T.dfa[(size_t)i * 256 + b] = (uint8_t)T.kept_of[delta[(int64_t)T.orig_of[i] * 256 + b]];
    };
    if (renumber) {
        std::vector<int32_t> orig(nr);
        for (int i = 0; i < nr; ++i) orig[(*renumber)[i]] = T.orig_of[i];
        T.orig_of = orig;
    }
    number();

    // 3. byte classes: equal columns of the kept table, numbered by first byte
    {
        std::unordered_map<std::string, int, VecHash> cols;
        std::string col(nr, '\0');
        T.ncls = 0;
        for (int b = 0; b < 256; ++b) {
            for (int i = 0; i < nr; ++i) col[i] = (char)T.dfa[(size_t)i * 256 + b];
            auto it = cols.find(col);
            if (it == cols.end()) it = cols.emplace(col, T.ncls++).first;
            T.cls[b] = (uint8_t)it->second;
        }
    }
    const int ncls = T.ncls;
    std::vector<uint8_t> rep(ncls);  // a representative byte of each class
    for (int b = 255; b >= 0; --b) rep[T.cls[b]] = (uint8_t)b;

    T.ident = nr > 1 ? (uint32_t)nr : 0u;
    T.n_nc = 0;
    T.nc.clear();
    T.maps.clear();
    T.n_const = 0;
    T.mode = SFA_MODE_SFA;

    bool sim = force_mode == SFA_MODE_SIM;
    if (!sim && nr > 1) {
        // 4. correspondence construction over the non-constant mappings
        std::unordered_map<std::string, uint32_t, VecHash> ids;
        ids.reserve(1024);
        std::string f(nr, '\0'), g(nr, '\0');
        for (int q = 0; q < nr; ++q) f[q] = (char)q;
        T.maps.insert(T.maps.end(), f.begin(), f.end());
        ids.emplace(f, 0);
        T.n_nc = 1;
        for (uint64_t head = 0; head < T.n_nc && !sim; ++head) {
            for (int c = 0; c < ncls; ++c) {
                const uint8_t *fm = T.maps.data() + head * nr;
                const uint8_t *row_b = T.dfa.data() + rep[c];
                bool constant = true;
                for (int q = 0; q < nr; ++q) {
                    g[q] = (char)row_b[(size_t)fm[q] * 256];
                    constant &= g[q] == g[0];
                }
                uint32_t id;
                if (constant) {
                    id = (uint8_t)g[0];
                } else {
                    auto it = ids.find(g);
                    if (it == ids.end()) {
                        if (T.n_nc >= cap) {
                            sim = true;
                            break;
                        }
                        it = ids.emplace(g, (uint32_t)T.n_nc).first;
                        T.maps.insert(T.maps.end(), g.begin(), g.end());
                        ++T.n_nc;
                    }
                    id = (uint32_t)nr + it->second;
                }
                T.nc.push_back(id);  // class bits added below
            }
        }
        if (sim && force_mode == SFA_MODE_SFA) return SFA_ERR_UNSUPPORTED;
    }
    if (sim) {
        if (nr > SIM_MAX_STATES) return SFA_ERR_UNSUPPORTED;
        T.mode = SFA_MODE_SIM;
        T.n_nc = 0;
        T.nc.clear();
        T.maps.clear();
    } else {
        // acceptance class of each target, packed into the entry
        for (uint64_t i = 0; i < T.nc.size(); ++i) {
            uint32_t id = T.nc[i];
            uint32_t a = id < (uint32_t)nr ? ((int)id >= T.first_accept ? ACC_ALL : ACC_NONE)
                                           : acc_class(T.maps.data() + (size_t)(id - nr) * nr, nr,
                                                       T.first_accept);
            T.nc[i] = id | (a << NC_ACC_SHIFT);
        }
        // constant mappings reachable from f_I: the targets of non-constant
        // rows (or f_I itself when nr = 1), closed under the DFA rows
        std::vector<char> reach(nr, 0);
        std::vector<int> stack;
        auto mark = [&](int c) {
            if (!reach[c]) {
                reach[c] = 1;
                stack.push_back(c);
            }
        };
        if (nr == 1) mark(0);
        for (uint32_t e : T.nc)
            if ((e & NC_ID_MASK) < (uint32_t)nr) mark((int)(e & NC_ID_MASK));
        while (!stack.empty()) {
            int c = stack.back();
            stack.pop_back();
            for (int k = 0; k < ncls; ++k) mark(T.dfa[(size_t)c * 256 + rep[k]]);
        }
        for (char r : reach) T.n_const += r ? 1 : 0;
    }
    T.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SFA_OK;
}

}  // namespace

// The bank-conflict numbering applies to D-SFA handles only: the simulation
// path looks up |Q| rows per byte and lane, which the model does not describe.
int build_tables(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                 uint32_t cap, int32_t force_mode, HostTables &T, bool tune_banks, const uint8_t *sample,
                 uint64_t sample_len) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = build_numbered(delta, nq, q0, accept, cap, force_mode, T, nullptr);
    if (rc || !tune_banks || T.mode != SFA_MODE_SFA || T.nr < 3 || T.wide) return rc;
    const std::vector<int32_t> id = bank_numbering(T.dfa, T.nr, T.first_accept, T.q0, sample, sample_len);
    bool moved = false;
    for (int32_t i = 0; i < T.nr; ++i) moved |= id[i] != i;
    if (moved) rc = build_numbered(delta, nq, q0, accept, cap, force_mode, T, &id);
    T.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // namespace sfa_impl
