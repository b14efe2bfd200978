// Regular-expression front end (no CUDA in this unit): the pipeline of
// Sect. VI -- a regular expression to an NFA by McNaughton and Yamada's
// position construction, to a DFA by the subset construction (Alg. 1), then
// minimised -- whose DFA feeds sfa_compile; and the N-SFA of the position
// automaton (Alg. 4 over correspondences, Definition 1), counted.
//
// Syntax (bytes): literals; escapes \n \t \r \f \v \0 \xHH and \ before any
// other byte; \d \D \w \W \s \S; '.' (every byte but '\n'; every byte with
// SFA_REGEX_DOTALL); classes [...] with ranges, negation [^...] and the
// escapes above; groups (...) and (?:...); alternation |; quantifiers * + ?
// {m} {m,} {m,n}.  The empty pattern and empty alternatives denote the
// empty word.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "sfa.h"

namespace {

constexpr int MAX_POSITIONS = 4096;   // positions of the expanded expression
constexpr int MAX_REPEAT = 1000;      // bound m, n of {m,n}

using Bytes = std::vector<uint8_t>;   // a byte set as 256 flags

struct Node {
    enum Kind { EMPTY, SET, CAT, ALT, STAR, PLUS, OPT } kind = EMPTY;
    Bytes set;          // SET
    int a = -1, b = -1; // children
};

struct Parser {
    const uint8_t *p;
    size_t n, i = 0;
    uint32_t flags;
    std::vector<Node> nodes;
    bool bad = false;
    size_t bad_at = 0;

    int add(Node x) {
        nodes.push_back(std::move(x));
        return (int)nodes.size() - 1;
    }
    int fail() {
        if (!bad) {
            bad = true;
            bad_at = i;
        }
        return -1;
    }
    bool more() const { return i < n; }
    uint8_t peek() const { return p[i]; }

    static void set_range(Bytes &s, int lo, int hi) {
        for (int c = lo; c <= hi; ++c) s[c] = 1;
    }
    static Bytes digits() {
        Bytes s(256, 0);
        set_range(s, '0', '9');
        return s;
    }
    static Bytes words() {
        Bytes s(256, 0);
        set_range(s, '0', '9');
        set_range(s, 'a', 'z');
        set_range(s, 'A', 'Z');
        s['_'] = 1;
        return s;
    }
    static Bytes spaces() {
        Bytes s(256, 0);
        for (int c : {' ', '\t', '\n', '\r', '\f', '\v'}) s[c] = 1;
        return s;
    }
    static Bytes complement(Bytes s) {
        for (auto &x : s) x = !x;
        return s;
    }
    static int hexv(uint8_t c) {
        if (c >= '0' && c <= '9') return c - '0';
        if (c >= 'a' && c <= 'f') return c - 'a' + 10;
        if (c >= 'A' && c <= 'F') return c - 'A' + 10;
        return -1;
    }
    // after a backslash: a byte set (class escapes) or a single byte; false
    // on a malformed escape
    bool escape(Bytes &out) {
        if (!more()) return false;
        const uint8_t c = p[i++];
        out.assign(256, 0);
        switch (c) {
            case 'd': out = digits(); return true;
            case 'D': out = complement(digits()); return true;
            case 'w': out = words(); return true;
            case 'W': out = complement(words()); return true;
            case 's': out = spaces(); return true;
            case 'S': out = complement(spaces()); return true;
            case 'n': out['\n'] = 1; return true;
            case 't': out['\t'] = 1; return true;
            case 'r': out['\r'] = 1; return true;
            case 'f': out['\f'] = 1; return true;
            case 'v': out['\v'] = 1; return true;
            case '0': out[0] = 1; return true;
            case 'x': {
                if (i + 2 > n) return false;
                const int h = hexv(p[i]), l = hexv(p[i + 1]);
                if (h < 0 || l < 0) return false;
                i += 2;
                out[h * 16 + l] = 1;
                return true;
            }
            default:
                if ((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9'))
                    return false;   // an unknown letter escape is an error, not a literal
                out[c] = 1;
                return true;
        }
    }
    int cls() {   // after '['
        Bytes s(256, 0);
        bool neg = false;
        if (more() && peek() == '^') {
            neg = true;
            ++i;
        }
        bool first = true;
        while (more() && (peek() != ']' || first)) {
            first = false;
            Bytes lo_set;
            int lo;
            if (peek() == '\\') {
                ++i;
                if (!escape(lo_set)) return fail();
                int cnt = 0, only = -1;
                for (int c = 0; c < 256; ++c)
                    if (lo_set[c]) {
                        ++cnt;
                        only = c;
                    }
                if (cnt != 1) {   // a class escape: no range from it
                    for (int c = 0; c < 256; ++c) s[c] |= lo_set[c];
                    continue;
                }
                lo = only;
            } else {
                lo = p[i++];
            }
            if (i + 1 < n && peek() == '-' && p[i + 1] != ']') {
                ++i;
                int hi;
                if (peek() == '\\') {
                    ++i;
                    Bytes hs;
                    if (!escape(hs)) return fail();
                    int cnt = 0, only = -1;
                    for (int c = 0; c < 256; ++c)
                        if (hs[c]) {
                            ++cnt;
                            only = c;
                        }
                    if (cnt != 1) return fail();
                    hi = only;
                } else {
                    hi = p[i++];
                }
                if (hi < lo) return fail();
                set_range(s, lo, hi);
            } else {
                s[lo] = 1;
            }
        }
        if (!more()) return fail();
        ++i;   // ']'
        if (neg) s = complement(s);
        Node x;
        x.kind = Node::SET;
        x.set = s;
        return add(x);
    }
    int atom() {
        if (!more()) return fail();
        const uint8_t c = peek();
        if (c == '(') {
            ++i;
            if (i + 1 < n && p[i] == '?' && p[i + 1] == ':') i += 2;
            const int r = alt();
            if (r < 0) return -1;
            if (!more() || peek() != ')') return fail();
            ++i;
            return r;
        }
        if (c == '[') {
            ++i;
            return cls();
        }
        Node x;
        x.kind = Node::SET;
        x.set.assign(256, 0);
        if (c == '.') {
            ++i;
            x.set.assign(256, 1);
            if (!(flags & SFA_REGEX_DOTALL)) x.set['\n'] = 0;
            return add(x);
        }
        if (c == '\\') {
            ++i;
            if (!escape(x.set)) return fail();
            return add(x);
        }
        if (c == ')' || c == '|' || c == '*' || c == '+' || c == '?' || c == '{' || c == ']' || c == '}' ||
            c == '^' || c == '$')
            return fail();   // a stray metacharacter (anchors are not supported)
        ++i;
        x.set[c] = 1;
        return add(x);
    }
    // a copy of the subtree at r (counted repetition: every copy has
    // positions of its own)
    int clone(int r) {
        Node x = nodes[r];
        if (x.a >= 0) x.a = clone(x.a);
        if (x.b >= 0) x.b = clone(x.b);
        return add(x);
    }
    int unary(Node::Kind k, int a) {
        Node x;
        x.kind = k;
        x.a = a;
        return add(x);
    }
    int binary(Node::Kind k, int a, int b) {
        Node x;
        x.kind = k;
        x.a = a;
        x.b = b;
        return add(x);
    }
    bool number(int &v) {
        if (!more() || peek() < '0' || peek() > '9') return false;
        v = 0;
        while (more() && peek() >= '0' && peek() <= '9') {
            v = v * 10 + (p[i++] - '0');
            if (v > MAX_REPEAT) return false;
        }
        return true;
    }
    int repeat() {
        int r = atom();
        if (r < 0) return -1;
        while (more()) {
            const uint8_t c = peek();
            if (c == '*') {
                ++i;
                r = unary(Node::STAR, r);
            } else if (c == '+') {
                ++i;
                r = unary(Node::PLUS, r);
            } else if (c == '?') {
                ++i;
                r = unary(Node::OPT, r);
            } else if (c == '{') {
                ++i;
                int m = 0, mx = 0;
                if (!number(m)) return fail();
                bool unbounded = false;
                if (more() && peek() == ',') {
                    ++i;
                    if (more() && peek() == '}') unbounded = true;
                    else if (!number(mx)) return fail();
                } else {
                    mx = m;
                }
                if (!more() || peek() != '}') return fail();
                ++i;
                if (!unbounded && mx < m) return fail();
                // r{m,n} = r ... r (m copies) then (r (r ...)?)? (n - m
                // optional copies); r{m,} = r ... r r*
                int out = -1;
                for (int k = 0; k < m; ++k) out = out < 0 ? clone(r) : binary(Node::CAT, out, clone(r));
                int tail = -1;
                if (unbounded) {
                    tail = unary(Node::STAR, clone(r));
                } else {
                    for (int k = 0; k < mx - m; ++k)
                        tail = unary(Node::OPT, tail < 0 ? clone(r) : binary(Node::CAT, clone(r), tail));
                }
                if (tail >= 0) out = out < 0 ? tail : binary(Node::CAT, out, tail);
                if (out < 0) out = add(Node{});   // r{0} and r{0,0}: the empty word
                r = out;
            } else {
                break;
            }
            if (nodes.size() > 16u * MAX_POSITIONS) return fail();
        }
        return r;
    }
    int cat() {
        int r = -1;
        while (more() && peek() != '|' && peek() != ')') {
            const int x = repeat();
            if (x < 0) return -1;
            r = r < 0 ? x : binary(Node::CAT, r, x);
        }
        return r < 0 ? add(Node{}) : r;
    }
    int alt() {
        int r = cat();
        if (r < 0) return -1;
        while (more() && peek() == '|') {
            ++i;
            const int x = cat();
            if (x < 0) return -1;
            r = binary(Node::ALT, r, x);
        }
        return r;
    }
};

// a set of NFA states (0 = initial, 1..P = positions) as 64-bit words
struct Bits {
    std::vector<uint64_t> w;
    explicit Bits(int n = 0) : w((n + 63) / 64, 0) {}
    void set(int k) { w[k >> 6] |= 1ull << (k & 63); }
    bool get(int k) const { return w[k >> 6] >> (k & 63) & 1; }
    void operator|=(const Bits &o) {
        for (size_t j = 0; j < w.size(); ++j) w[j] |= o.w[j];
    }
    bool any() const {
        for (uint64_t x : w)
            if (x) return true;
        return false;
    }
};

// McNaughton and Yamada's position automaton of the parsed expression
struct PositionNfa {
    int P = 0;                    // positions; NFA states 0..P
    std::vector<Bytes> sym;       // [P+1] byte set of each position (0 unused)
    std::vector<Bits> follow;     // [P+1] follow(0) = first
    Bits last;                    // final positions (and 0 when the expression is nullable)
    bool search = false;          // state 0 loops on every byte
};

struct Glushkov {
    Parser &ps;
    PositionNfa &A;
    std::vector<int> pos_of;   // node -> position (SET nodes)
    struct Info {
        bool nullable = false;
        std::vector<int> first, last;
    };
    Info walk(int r) {
        const Node &x = ps.nodes[r];
        Info out;
        switch (x.kind) {
            case Node::EMPTY: out.nullable = true; break;
            case Node::SET: {
                const int k = ++A.P;
                A.sym.push_back(x.set);
                A.follow.emplace_back();
                out.first = {k};
                out.last = {k};
                break;
            }
            case Node::CAT: {
                Info a = walk(x.a), b = walk(x.b);
                pending.emplace_back(a.last, b.first);
                out.nullable = a.nullable && b.nullable;
                out.first = a.first;
                if (a.nullable) out.first.insert(out.first.end(), b.first.begin(), b.first.end());
                out.last = b.last;
                if (b.nullable) out.last.insert(out.last.end(), a.last.begin(), a.last.end());
                break;
            }
            case Node::ALT: {
                Info a = walk(x.a), b = walk(x.b);
                out.nullable = a.nullable || b.nullable;
                out.first = a.first;
                out.first.insert(out.first.end(), b.first.begin(), b.first.end());
                out.last = a.last;
                out.last.insert(out.last.end(), b.last.begin(), b.last.end());
                break;
            }
            case Node::STAR:
            case Node::PLUS:
            case Node::OPT: {
                Info a = walk(x.a);
                if (x.kind != Node::OPT) pending.emplace_back(a.last, a.first);
                out.nullable = x.kind == Node::PLUS ? a.nullable : true;
                out.first = a.first;
                out.last = a.last;
                break;
            }
        }
        return out;
    }
    std::vector<std::pair<std::vector<int>, std::vector<int>>> pending;   // follow(p) |= F for p in L
};

int build_nfa(const char *pattern, size_t len, uint32_t flags, PositionNfa &A, size_t *err_pos) {
    if (!pattern && len) return SFA_ERR_INVALID;
    Parser ps{reinterpret_cast<const uint8_t *>(pattern), len, 0, flags, {}, false, 0};
    const int root = ps.alt();
    if (root < 0 || ps.bad || ps.i != len) {
        if (err_pos) *err_pos = ps.bad ? ps.bad_at : ps.i;
        return SFA_ERR_INVALID;
    }
    size_t sets = 0;
    for (const Node &x : ps.nodes) sets += x.kind == Node::SET;
    if (sets > (size_t)MAX_POSITIONS) return SFA_ERR_UNSUPPORTED;
    A = PositionNfa();
    A.sym.emplace_back(256, 0);
    A.follow.emplace_back();
    Glushkov g{ps, A, {}, {}};
    Glushkov::Info top = g.walk(root);
    const int ns = A.P + 1;
    for (auto &f : A.follow) f = Bits(ns);
    for (auto &pr : g.pending)
        for (int p : pr.first)
            for (int q : pr.second) A.follow[p].set(q);
    for (int q : top.first) A.follow[0].set(q);
    A.last = Bits(ns);
    for (int q : top.last) A.last.set(q);
    if (top.nullable) A.last.set(0);
    A.search = (flags & SFA_REGEX_SEARCH) != 0;
    return SFA_OK;
}

// byte classes: bytes in exactly the same positions' sets
int byte_classes(const PositionNfa &A, uint8_t cls[256], std::vector<uint8_t> &rep) {
    std::unordered_map<std::string, int> ids;
    std::string key((A.P + 8) / 8, '\0');
    int ncls = 0;
    for (int b = 0; b < 256; ++b) {
        std::fill(key.begin(), key.end(), '\0');
        for (int q = 1; q <= A.P; ++q)
            if (A.sym[q][b]) key[q >> 3] |= (char)(1 << (q & 7));
        auto it = ids.find(key);
        if (it == ids.end()) {
            it = ids.emplace(key, ncls++).first;
            rep.push_back((uint8_t)b);
        }
        cls[b] = (uint8_t)it->second;
    }
    return ncls;
}

// the successors of a set S of NFA states on class c: the union of follow
// sets (follow(0) = first) of S's states, restricted to the positions of c
// (plus state 0 itself when it loops, in the search form)
void step_set(const PositionNfa &A, const std::vector<Bits> &in_class, const Bits &S, int c, Bits &out) {
    const int ns = A.P + 1;
    out = Bits(ns);
    for (int q = 0; q < ns; ++q)
        if (S.get(q)) out |= A.follow[q];
    for (size_t j = 0; j < out.w.size(); ++j) out.w[j] &= in_class[c].w[j];
    if (A.search && S.get(0)) out.set(0);
}

std::string bits_key(const Bits &b) { return std::string(reinterpret_cast<const char *>(b.w.data()), b.w.size() * 8); }

}  // namespace

namespace sfa_impl {

// Regular expression -> position NFA -> subset construction (Alg. 1) ->
// minimal DFA (Moore's partition refinement).  delta: [nq*256], states
// numbered breadth first from the initial one.
int regex_to_dfa(const char *pattern, size_t len, uint32_t flags, int32_t cap, std::vector<int32_t> &delta,
                 std::vector<uint8_t> &accept, sfa_regex_info *info, size_t *err_pos) {
    PositionNfa A;
    int rc = build_nfa(pattern, len, flags, A, err_pos);
    if (rc) return rc;
    uint8_t cls[256];
    std::vector<uint8_t> rep;
    const int ncls = byte_classes(A, cls, rep);
    const int ns = A.P + 1;
    std::vector<Bits> in_class(ncls, Bits(ns));
    for (int c = 0; c < ncls; ++c)
        for (int q = 1; q <= A.P; ++q)
            if (A.sym[q][rep[c]]) in_class[c].set(q);
    // Alg. 1: FIFO worklist from {initial}, the empty set included as a state
    const size_t subset_cap = std::max<size_t>((size_t)cap * 16, 1u << 16);
    std::vector<Bits> sets;
    std::unordered_map<std::string, int32_t> id;
    std::vector<int32_t> sd;   // [nsets*ncls]
    Bits init(ns);
    init.set(0);
    sets.push_back(init);
    id.emplace(bits_key(init), 0);
    Bits nx;
    for (size_t h = 0; h < sets.size(); ++h) {
        for (int c = 0; c < ncls; ++c) {
            step_set(A, in_class, sets[h], c, nx);
            auto it = id.find(bits_key(nx));
            if (it == id.end()) {
                if (sets.size() >= subset_cap) return SFA_ERR_UNSUPPORTED;
                it = id.emplace(bits_key(nx), (int32_t)sets.size()).first;
                sets.push_back(nx);
            }
            sd.push_back(it->second);
        }
    }
    const int nsub = (int)sets.size();
    std::vector<uint8_t> fin(nsub);
    for (int s = 0; s < nsub; ++s) {
        bool f = false;
        for (size_t j = 0; j < sets[s].w.size() && !f; ++j) f = (sets[s].w[j] & A.last.w[j]) != 0;
        fin[s] = f;
    }
    // minimisation: refine (final?, classes of the successors) to a fixpoint
    std::vector<int32_t> part(nsub);
    int nparts = 0;
    if (flags & SFA_REGEX_NO_MINIMIZE) {
        for (int s = 0; s < nsub; ++s) part[s] = s;
        nparts = nsub;
    } else {
        for (int s = 0; s < nsub; ++s) part[s] = fin[s];
        nparts = -1;
        for (;;) {
            std::unordered_map<std::string, int32_t> key_id;
            std::vector<int32_t> next(nsub);
            std::string key((ncls + 1) * 4, '\0');
            for (int s = 0; s < nsub; ++s) {
                int32_t v = part[s];
                std::memcpy(&key[0], &v, 4);
                for (int c = 0; c < ncls; ++c) {
                    v = part[sd[(size_t)s * ncls + c]];
                    std::memcpy(&key[4 * (c + 1)], &v, 4);
                }
                auto it = key_id.find(key);
                if (it == key_id.end()) it = key_id.emplace(key, (int32_t)key_id.size()).first;
                next[s] = it->second;
            }
            const int k = (int)key_id.size();
            part.swap(next);
            if (k == nparts) break;
            nparts = k;
        }
    }
    // renumber the blocks breadth first from the initial state's block
    std::vector<int32_t> order_of(nparts, -1), rep_state;
    std::vector<int32_t> queue{part[0]};
    order_of[part[0]] = 0;
    std::vector<int32_t> any_state(nparts, -1);
    for (int s = 0; s < nsub; ++s)
        if (any_state[part[s]] < 0) any_state[part[s]] = s;
    for (size_t h = 0; h < queue.size(); ++h) {
        const int s = any_state[queue[h]];
        for (int c = 0; c < ncls; ++c) {
            const int t = part[sd[(size_t)s * ncls + c]];
            if (order_of[t] < 0) {
                order_of[t] = (int32_t)queue.size();
                queue.push_back(t);
            }
        }
    }
    const int nq = (int)queue.size();
    if (info) {
        info->nq = nq;
        info->q0 = 0;
        info->positions = A.P;
        info->subset_states = nsub;
        info->ncls = ncls;
    }
    if (nq > cap) return SFA_ERR_UNSUPPORTED;
    delta.assign((size_t)nq * 256, 0);
    accept.assign(nq, 0);
    for (int k = 0; k < nq; ++k) {
        const int s = any_state[queue[k]];
        accept[k] = fin[s];
        for (int b = 0; b < 256; ++b) delta[(size_t)k * 256 + b] = order_of[part[sd[(size_t)s * ncls + cls[b]]]];
    }
    return SFA_OK;
}

// Alg. 4 on the position NFA: correspondences f (f(q) a set of NFA states,
// f_I(q) = {q}), f_next(q) = the union of delta(q', sigma) over q' in f(q).
// Counts the states reachable from f_I, up to cap.
int regex_nsfa_states(const char *pattern, size_t len, uint32_t flags, uint64_t cap, uint64_t *n_states) {
    PositionNfa A;
    int rc = build_nfa(pattern, len, flags, A, nullptr);
    if (rc) return rc;
    uint8_t cls[256];
    std::vector<uint8_t> rep;
    const int ncls = byte_classes(A, cls, rep);
    const int ns = A.P + 1;
    std::vector<Bits> in_class(ncls, Bits(ns));
    for (int c = 0; c < ncls; ++c)
        for (int q = 1; q <= A.P; ++q)
            if (A.sym[q][rep[c]]) in_class[c].set(q);
    auto key_of = [&](const std::vector<Bits> &f) {
        std::string k;
        for (const Bits &b : f) k += bits_key(b);
        return k;
    };
    std::vector<std::vector<Bits>> states;
    std::unordered_map<std::string, uint64_t> seen;
    std::vector<Bits> fi(ns, Bits(ns));
    for (int q = 0; q < ns; ++q) fi[q].set(q);
    states.push_back(fi);
    seen.emplace(key_of(fi), 0);
    std::vector<Bits> g(ns);
    for (size_t h = 0; h < states.size(); ++h) {
        for (int c = 0; c < ncls; ++c) {
            for (int q = 0; q < ns; ++q) step_set(A, in_class, states[h][q], c, g[q]);
            const std::string k = key_of(g);
            if (!seen.count(k)) {
                if (states.size() >= cap) {
                    *n_states = states.size();
                    return SFA_ERR_UNSUPPORTED;
                }
                seen.emplace(k, states.size());
                states.push_back(g);
            }
        }
    }
    *n_states = states.size();
    return SFA_OK;
}

}  // namespace sfa_impl

using namespace sfa_impl;

extern "C" {

int sfa_regex_dfa(const char *pattern, size_t len, uint32_t flags, int32_t cap, int32_t *delta, uint8_t *accept,
                  sfa_regex_info *info, size_t *err_pos) {
    if (cap < 1 || (cap > 0 && (!!delta != !!accept))) return SFA_ERR_INVALID;
    std::vector<int32_t> d;
    std::vector<uint8_t> a;
    int rc;
    try {
        rc = regex_to_dfa(pattern, len, flags, delta ? cap : WIDE_MAX_STATES, d, a, info, err_pos);
    } catch (const std::bad_alloc &) {
        return SFA_ERR_OOM;
    }
    if (rc) return rc;
    if (delta) {
        std::memcpy(delta, d.data(), d.size() * 4);
        std::memcpy(accept, a.data(), a.size());
    }
    return SFA_OK;
}

int sfa_regex_nsfa_states(const char *pattern, size_t len, uint32_t flags, uint64_t cap, uint64_t *n_states) {
    if (!n_states || cap < 1) return SFA_ERR_INVALID;
    try {
        return regex_nsfa_states(pattern, len, flags, cap, n_states);
    } catch (const std::bad_alloc &) {
        return SFA_ERR_OOM;
    }
}

int sfa_regex_compile(const char *pattern, size_t len, uint32_t flags, const sfa_compile_opts *opts,
                      sfa_handle_t *out) {
    if (!out) return SFA_ERR_INVALID;
    *out = nullptr;
    std::vector<int32_t> d;
    std::vector<uint8_t> a;
    sfa_regex_info info{};
    int rc;
    try {
        rc = regex_to_dfa(pattern, len, flags, WIDE_MAX_STATES, d, a, &info, nullptr);
    } catch (const std::bad_alloc &) {
        return SFA_ERR_OOM;
    }
    if (rc) return rc;
    return sfa_compile(d.data(), info.nq, info.q0, a.data(), opts, out);
}

}  // extern "C"
