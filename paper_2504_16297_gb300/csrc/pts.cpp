// Pre-trajectory sampling on the host (Sec. 3.1, Algorithm 2).
//
// Every mode ends in the same bookkeeping: sets sorted into canonical order (lexicographic over
// the (site, k) list, a prefix before its extensions), duplicates merged (uniqueKraus of
// Algorithm 2, multiplicity = number of samples that produced the set), nominal probability
// q_alpha = Q0 * key(alpha) with Q0 = prod_s q_{s,0} and key = product of the set's ratios
// q_{s,k}/q_{s,0} taken in descending order, and shots allocated by largest remainders
// ("redistributing ... according to the relative populations", Sec. 3.1).
//
// Compiled without floating-point contraction so the FP64 decisions (categorical draws,
// keys, quotas) are reproducible on every host.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <thread>
#include <unordered_map>

#include "internal.h"
#include "philox.h"

namespace ptsbe {

namespace {

struct Entry {
    uint32_t site;
    uint8_t k;
    bool operator<(const Entry& o) const { return site != o.site ? site < o.site : k < o.k; }
    bool operator==(const Entry& o) const { return site == o.site && k == o.k; }
};
using List = std::vector<Entry>;

bool canon_less(const List& a, const List& b) {
    return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

// Smallest k with u < q_0 + ... + q_k, summed in listed order; the last index otherwise.
inline int categorical(double u, const double* q, int nk) {
    double acc = 0.0;
    for (int k = 0; k < nk; ++k) {
        acc += q[k];
        if (u < acc) return k;
    }
    return nk - 1;
}

double ratio(const Circuit& c, uint32_t site, int k) {
    const HostChannel& ch = c.ch[c.site_ch[site]];
    return ch.q[k] / ch.q[0];
}

// Sorts, merges duplicates, fills key/q and the CSR arrays of `out`.
void finish(const Circuit& c, std::vector<std::pair<List, uint64_t>>& sets, std::vector<uint64_t>* given_shots,
            KSet& out) {
    std::vector<size_t> idx(sets.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return canon_less(sets[a].first, sets[b].first); });
    out.off.assign(1, 0);
    out.site.clear(); out.k.clear(); out.mult.clear(); out.q.clear(); out.key.clear(); out.shots.clear();
    std::vector<uint64_t> gshots;
    const List* prev = nullptr;
    for (size_t t = 0; t < idx.size(); ++t) {
        auto& s = sets[idx[t]];
        if (prev && *prev == s.first) {
            out.mult.back() += s.second;
            if (given_shots) gshots.back() += (*given_shots)[idx[t]];
            continue;
        }
        for (const Entry& e : s.first) { out.site.push_back(e.site); out.k.push_back(e.k); }
        out.off.push_back((uint32_t)out.site.size());
        out.mult.push_back(s.second);
        if (given_shots) gshots.push_back((*given_shots)[idx[t]]);
        prev = &s.first;
    }
    const uint32_t n = (uint32_t)out.mult.size();
    out.key.resize(n); out.q.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        out.key[i] = set_key(c, out.site.data() + out.off[i], out.k.data() + out.off[i], out.off[i + 1] - out.off[i]);
        out.q[i] = c.Q0 * out.key[i];
    }
    if (given_shots) out.shots = gshots;
}

void allocate_shots(KSet& s, uint32_t alloc, uint64_t total, uint64_t per_set) {
    const uint32_t n = s.count();
    if (alloc == PTSBE_SHOTS_BY_COUNT) apportion_counts(s.mult, total, s.shots);
    else if (alloc == PTSBE_SHOTS_UNIFORM) s.shots.assign(n, per_set);
    else if (alloc == PTSBE_SHOTS_BY_PROB) apportion_weights(s.q, total, s.shots);
    else if (alloc == PTSBE_SHOTS_GIVEN) { /* already set */ }
    else fail(PTSBE_ERR_INVALID, "unknown shot allocation");
}

// ---- probabilistic modes -------------------------------------------------------------------------
template <class F>
void parallel_for(uint64_t n, F&& f) {
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    unsigned nt = (unsigned)std::min<uint64_t>(hw, std::max<uint64_t>(1, n / 64));
    if (nt <= 1) { f(0, n); return; }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        uint64_t b = n * t / nt, e = n * (t + 1) / nt;
        th.emplace_back([&f, b, e] { f(b, e); });
    }
    for (auto& x : th) x.join();
}

void pts_proportional(const Circuit& c, uint64_t ns, uint64_t seed, std::vector<std::pair<List, uint64_t>>& sets) {
    sets.assign(ns, {});
    const uint32_t S = (uint32_t)c.site_ch.size();
    parallel_for(ns, [&](uint64_t b, uint64_t e) {
        for (uint64_t i = b; i < e; ++i) {
            List& l = sets[i].first;
            sets[i].second = 1;
            for (uint32_t s = 0; s < S; ++s) {
                const HostChannel& ch = c.ch[c.site_ch[s]];
                const double u = uniform53(seed, s, (uint32_t)i, (uint32_t)(i >> 32), kDomPts);
                const int k = categorical(u, ch.q.data(), (int)ch.nk);
                if (k != 0) l.push_back({s, (uint8_t)k});
            }
        }
    });
}

void pts_literal(const Circuit& c, uint64_t ns, uint64_t seed, std::vector<std::pair<List, uint64_t>>& sets) {
    sets.assign(ns, {});
    const uint32_t S = (uint32_t)c.site_ch.size();
    parallel_for(ns, [&](uint64_t b, uint64_t e) {
        for (uint64_t i = b; i < e; ++i) {
            List& l = sets[i].first;
            sets[i].second = 1;
            for (uint32_t s = 0; s < S; ++s) {
                const HostChannel& ch = c.ch[c.site_ch[s]];
                bool taken = false;
                for (uint32_t k = 1; k < ch.nk; ++k) {
                    const double r = uniform53(seed, s, (uint32_t)i, (uint32_t)(i >> 32), kDomLiteral | (k << 8));
                    if (r <= ch.q[k] && !taken) { l.push_back({s, (uint8_t)k}); taken = true; }
                }
            }
        }
    });
}

// ---- most-likely modes: best-first enumeration ------------------------------------------------------
// Options (s, k != 0) with q_{s,k} > 0 sorted by ratio descending, then (s, k). A set is an
// increasing list of option indices with distinct sites. Children of a set S with last option j:
//   extend : S + {next option after j whose site is not in S}
//   replace: S - {j} + {next option after j whose site is not in S - {j}}
// Every set has exactly one parent, and a child never precedes its parent in the order
// (key descending, canonical ascending): extending multiplies by a ratio < 1; replacing with an
// equal ratio moves an entry to a larger (site, k). Best-first search on a max-heap in that order
// therefore pops sets exactly in sorted order.
struct Opt { uint32_t site; uint8_t k; double r; };

// Nodes live in flat arenas: options and site-sorted entries of node i are [off, off + len) of
// opt_ and ent_ (entries packed as site << 8 | k, so packed order is the canonical entry order).
// Heap entries carry the key, so comparisons only touch the arenas on ties.
struct Node {
    double key;          // product of the ratios of opts, in option order
    double prefix;       // product without the last option
    uint32_t off, len;
};

// Heap entries carry the key and the set's first two packed entries plus one (0: absent), which
// order two sets lexicographically at those positions (a shorter list first); the arenas are read
// only when the key and both words tie.
struct HeapItem {
    double key;
    uint64_t w0, w1;
    uint32_t node;
};

class BestFirst {
  public:
    explicit BestFirst(const Circuit& c) : c_(c) {
        const uint32_t S = (uint32_t)c.site_ch.size();
        for (uint32_t s = 0; s < S; ++s) {
            const HostChannel& ch = c.ch[c.site_ch[s]];
            for (uint32_t k = 1; k < ch.nk; ++k)
                if (ch.q[k] > 0) opts_.push_back({s, (uint8_t)k, ratio(c, s, (int)k)});
        }
        std::sort(opts_.begin(), opts_.end(), [](const Opt& a, const Opt& b) {
            if (a.r != b.r) return a.r > b.r;
            if (a.site != b.site) return a.site < b.site;
            return a.k < b.k;
        });
        nodes_.push_back({1.0, 1.0, 0, 0});
        push({1.0, 0, 0, 0});
    }

    // Pops the next set in order (its node: key and site-sorted packed entries stay readable);
    // false when exhausted.
    bool next_node(uint32_t& node) {
        if (heap_.empty()) return false;
        const HeapItem top = heap_.front();
        std::pop_heap(heap_.begin(), heap_.end(), after_);
        heap_.pop_back();
        node = top.node;
        expand(top.node);
        return true;
    }
    double key(uint32_t node) const { return nodes_[node].key; }
    uint32_t len(uint32_t node) const { return nodes_[node].len; }
    const uint64_t* entries(uint32_t node) const { return ent_.data() + nodes_[node].off; }
    // canonical order of two popped sets (entries packed site << 8 | k compare as (site, k))
    bool canon_before(uint32_t a, uint32_t b) const {
        const Node& na = nodes_[a];
        const Node& nb = nodes_[b];
        return std::lexicographical_compare(ent_.begin() + na.off, ent_.begin() + na.off + na.len,
                                            ent_.begin() + nb.off, ent_.begin() + nb.off + nb.len);
    }
    // packed entry i of node plus one, 0 past its end
    uint64_t word(uint32_t node, uint32_t i) const {
        const Node& nd = nodes_[node];
        return i < nd.len ? ent_[nd.off + i] + 1 : 0;
    }
    // Room for k pops (each pushes at most two children).
    void reserve(uint64_t k) {
        const size_t n = (size_t)std::min<uint64_t>(k, 1ull << 24);
        nodes_.reserve(2 * n + 1);
        heap_.reserve(2 * n + 1);
        opt_.reserve(8 * n + 8);
        ent_.reserve(8 * n + 8);
    }

  private:
    struct After {   // true if a comes after b (max-heap on key, then canonical ascending)
        const BestFirst* bf;
        bool operator()(const HeapItem& a, const HeapItem& b) const {
            if (a.key != b.key) return a.key < b.key;
            if (a.w0 != b.w0) return b.w0 < a.w0;
            if (a.w1 != b.w1) return b.w1 < a.w1;
            const Node& na = bf->nodes_[a.node];
            const Node& nb = bf->nodes_[b.node];
            return std::lexicographical_compare(bf->ent_.begin() + nb.off, bf->ent_.begin() + nb.off + nb.len,
                                                bf->ent_.begin() + na.off, bf->ent_.begin() + na.off + na.len);
        }
    };
    void push(HeapItem h) {
        heap_.push_back(h);
        std::push_heap(heap_.begin(), heap_.end(), after_);
    }
    bool site_used(uint32_t node, size_t upto, uint32_t site) const {
        const Node& nd = nodes_[node];
        for (size_t i = 0; i < upto; ++i) if (opts_[opt_[nd.off + i]].site == site) return true;
        return false;
    }
    // Smallest option index > after whose site is not among the first `upto` options of node.
    int64_t next_valid(uint32_t node, size_t upto, int64_t after) const {
        for (int64_t j = after + 1; j < (int64_t)opts_.size(); ++j)
            if (!site_used(node, upto, opts_[j].site)) return j;
        return -1;
    }
    void push_child(uint32_t base, size_t keep, double prefix, uint32_t j) {
        const uint32_t off = (uint32_t)opt_.size();
        const uint32_t boff = nodes_[base].off;
        for (size_t i = 0; i < keep; ++i) {
            const uint32_t o = opt_[boff + i];
            opt_.push_back(o);
        }
        opt_.push_back(j);
        ent_.resize(opt_.size());
        for (size_t i = 0; i <= keep; ++i) {
            const Opt& o = opts_[opt_[off + i]];
            ent_[off + i] = ((uint64_t)o.site << 8) | o.k;
        }
        std::sort(ent_.begin() + off, ent_.begin() + off + keep + 1);
        const uint32_t id = (uint32_t)nodes_.size();
        nodes_.push_back({prefix * opts_[j].r, prefix, off, (uint32_t)(keep + 1)});
        push({nodes_[id].key, word(id, 0), word(id, 1), id});
    }
    void expand(uint32_t node) {
        const uint32_t len = nodes_[node].len;
        const int64_t last = len == 0 ? -1 : (int64_t)opt_[nodes_[node].off + len - 1];
        const double key = nodes_[node].key, prefix = nodes_[node].prefix;
        int64_t j = next_valid(node, len, last);
        if (j >= 0) push_child(node, len, key, (uint32_t)j);
        if (len > 0) {
            j = next_valid(node, len - 1, last);
            if (j >= 0) push_child(node, len - 1, prefix, (uint32_t)j);
        }
    }

    const Circuit& c_;
    std::vector<Opt> opts_;
    std::vector<Node> nodes_;
    std::vector<uint32_t> opt_;
    std::vector<uint64_t> ent_;
    std::vector<HeapItem> heap_;
    After after_{this};
};

}  // namespace

double set_key(const Circuit& c, const uint32_t* sites, const uint8_t* ks, uint32_t len) {
    if (len == 0) return 1.0;
    double buf[16];
    std::vector<double> big;
    double* r = buf;
    if (len > 16) { big.resize(len); r = big.data(); }
    for (uint32_t i = 0; i < len; ++i) r[i] = ratio(c, sites[i], ks[i]);
    std::sort(r, r + len, [](double a, double b) { return a > b; });
    double key = 1.0;
    for (uint32_t i = 0; i < len; ++i) key *= r[i];
    return key;
}

void apportion_counts(const std::vector<uint64_t>& c, uint64_t M, std::vector<uint64_t>& out) {
    const size_t n = c.size();
    out.assign(n, 0);
    unsigned __int128 N = 0;
    for (uint64_t x : c) N += x;
    if (n == 0 || N == 0) return;
    std::vector<std::pair<uint64_t, uint32_t>> rem(n);
    uint64_t used = 0;
    uint64_t cmax = 0;
    for (uint64_t x : c) cmax = std::max(cmax, x);
    if (N <= UINT64_MAX && (cmax == 0 || M <= UINT64_MAX / cmax)) {   // the same quotients in 64 bits
        const uint64_t N64 = (uint64_t)N;
        for (size_t i = 0; i < n; ++i) {
            const uint64_t p = M * c[i];
            out[i] = p / N64;
            rem[i] = {p % N64, (uint32_t)i};
            used += out[i];
        }
    } else {
        for (size_t i = 0; i < n; ++i) {
            const unsigned __int128 p = (unsigned __int128)M * c[i];
            out[i] = (uint64_t)(p / N);
            rem[i] = {(uint64_t)(p % N), (uint32_t)i};
            used += out[i];
        }
    }
    // the M - used largest remainders (ties: lower index first) get one more shot; only the set
    // matters, and under this strict total order selection gives the same set as a full sort
    const uint64_t R = M - used;
    if (R == 0) return;
    auto first_r = [](const auto& a, const auto& b) { return a.first != b.first ? a.first > b.first : a.second < b.second; };
    if (R < n) std::nth_element(rem.begin(), rem.begin() + (ptrdiff_t)(R - 1), rem.end(), first_r);
    for (uint64_t j = 0; j < R; ++j) out[rem[j].second] += 1;
}

void apportion_weights(const std::vector<double>& w, uint64_t M, std::vector<uint64_t>& out) {
    const size_t n = w.size();
    out.assign(n, 0);
    if (n == 0) return;
    double W = 0.0;
    for (double x : w) W += x;
    std::vector<std::pair<double, uint32_t>> rem(n);
    uint64_t used = 0;
    for (size_t i = 0; i < n; ++i) {
        const double quota = W > 0 ? ((double)M * w[i]) / W : 0.0;
        const double fl = std::floor(quota);
        out[i] = (uint64_t)fl;
        rem[i] = {quota - fl, (uint32_t)i};
        used += out[i];
    }
    if (used <= M) {
        // as in apportion_counts: selection of the largest remainders, same set as a full sort
        const uint64_t R = std::min<uint64_t>(M - used, n);
        auto first_r = [](const auto& a, const auto& b) { return a.first != b.first ? a.first > b.first : a.second < b.second; };
        if (R > 0 && R < n) std::nth_element(rem.begin(), rem.begin() + (ptrdiff_t)(R - 1), rem.end(), first_r);
        for (uint64_t j = 0; j < R; ++j) out[rem[j].second] += 1;
    } else {
        std::sort(rem.begin(), rem.end(), [](const auto& a, const auto& b) {
            return a.first != b.first ? a.first < b.first : a.second > b.second;
        });
        uint64_t R = used - M;
        for (size_t j = 0; j < n && R > 0; ++j)
            if (out[rem[j].second] > 0) { out[rem[j].second] -= 1; --R; }
    }
}

namespace {

// Gate code of the last gate before op i that shares a qubit with it (UINT32_MAX if none).
uint32_t gate_before(const Circuit& c, size_t i) {
    const ptsbe_op& o = c.ops[i];
    for (size_t j = i; j-- > 0;) {
        const ptsbe_op& g = c.ops[j];
        if (g.kind != PTSBE_OP_GATE) continue;
        for (uint32_t a = 0; a < g.n_targets; ++a)
            for (uint32_t b = 0; b < o.n_targets; ++b)
                if (g.targets[a] == o.targets[b]) return g.id;
    }
    return UINT32_MAX;
}

// Targeted error sets by rule: the eligible (site, k) options, then every combination of 1 ..
// max_errors options at distinct sites (sites increasing), filtered by weight parity.
void pts_predicate(const Circuit& c, const ptsbe_pts_params& p, std::vector<std::pair<List, uint64_t>>& sets) {
    if (p.max_errors < 1 || p.max_errors > 8) fail(PTSBE_ERR_INVALID, "PREDICATE needs 1 <= max_errors <= 8");
    if (p.weight_parity > 2) fail(PTSBE_ERR_INVALID, "weight_parity must be 0, 1 or 2");
    const uint32_t S = (uint32_t)c.site_ch.size();
    const uint32_t lo = p.site_lo, hi = p.site_hi ? std::min<uint32_t>(p.site_hi, S) : S;
    std::vector<uint32_t> site_of;            // eligible sites, increasing
    std::vector<std::vector<uint8_t>> ks;     // their allowed Kraus indices
    for (uint32_t s = lo; s < hi; ++s) {
        const size_t op = c.site_op[s];
        const ptsbe_op& o = c.ops[op];
        bool ok = true;
        if (p.qubit_mask)
            for (uint32_t t = 0; t < o.n_targets; ++t) ok &= ((p.qubit_mask >> o.targets[t]) & 1ull) != 0;
        if (ok && p.gate_mask) {
            const uint32_t g = gate_before(c, op);
            ok = g < 32 && ((p.gate_mask >> g) & 1u);
        }
        if (!ok) continue;
        std::vector<uint8_t> kk;
        const HostChannel& ch = c.ch[c.site_ch[s]];
        for (uint32_t k = 1; k < ch.nk; ++k)
            if (!p.kraus_mask || ((p.kraus_mask >> k) & 1u)) kk.push_back((uint8_t)k);
        if (kk.empty()) continue;
        site_of.push_back(s);
        ks.push_back(std::move(kk));
    }
    // count before enumerating: e_w = number of w-error sets (elementary symmetric sums)
    const uint64_t cap = p.max_sets ? p.max_sets : 10000000ull;
    const uint32_t W = p.max_errors;
    std::vector<double> e(W + 1, 0.0);
    e[0] = 1.0;
    for (const auto& kk : ks)
        for (uint32_t w = W; w >= 1; --w) e[w] += e[w - 1] * (double)kk.size();
    double total = p.include_empty ? 1.0 : 0.0;
    for (uint32_t w = 1; w <= W; ++w)
        if (p.weight_parity == 0 || (p.weight_parity == 1) == (w % 2 == 1)) total += e[w];
    if (total > (double)cap) fail(PTSBE_ERR_UNSUPPORTED, "PREDICATE selects more than max_sets sets");
    if (p.include_empty) sets.push_back({List{}, 1});
    List cur;
    std::function<void(size_t)> rec = [&](size_t from) {
        const uint32_t w = (uint32_t)cur.size();
        if (w >= 1 && (p.weight_parity == 0 || (p.weight_parity == 1) == (w % 2 == 1))) sets.push_back({cur, 1});
        if (w == W) return;
        for (size_t i = from; i < site_of.size(); ++i)
            for (uint8_t k : ks[i]) {
                cur.push_back({site_of[i], k});
                rec(i + 1);
                cur.pop_back();
            }
    };
    rec(0);
}

}  // namespace

void pts_run(const Circuit& c, const ptsbe_pts_params& p, uint64_t seed, KSet& out) {
    std::vector<std::pair<List, uint64_t>> sets;
    std::vector<uint64_t> given;
    uint32_t alloc = p.shot_alloc;
    switch (p.mode) {
    case PTSBE_PTS_PROPORTIONAL:
        pts_proportional(c, p.nsamples, seed, sets);
        break;
    case PTSBE_PTS_LITERAL:
        pts_literal(c, p.nsamples, seed, sets);
        break;
    case PTSBE_PTS_TOPK:
    case PTSBE_PTS_BAND: {
        if (!c.k0_strict_mode)
            fail(PTSBE_ERR_UNSUPPORTED, "TOPK/BAND need q_{s,0} to be the strict maximum at every site");
        if (p.mode == PTSBE_PTS_BAND && !(p.p_min > 0) )
            fail(PTSBE_ERR_INVALID, "BAND needs p_min > 0");
        if (alloc == PTSBE_SHOTS_GIVEN) fail(PTSBE_ERR_INVALID, "SHOTS_GIVEN is for TARGETED");
        // The search yields distinct sets: they go to the output in canonical order straight from
        // the search's entry arena (no per-set lists, no merging of duplicates).
        BestFirst bf(c);
        std::vector<uint32_t> ids;
        uint32_t node;
        if (p.mode == PTSBE_PTS_TOPK) {
            bf.reserve(p.k);
            ids.reserve((size_t)std::min<uint64_t>(p.k, 1ull << 24));
            for (uint64_t i = 0; i < p.k && bf.next_node(node); ++i) ids.push_back(node);
        } else {
            while (bf.next_node(node)) {
                const double q = c.Q0 * bf.key(node);
                if (q < p.p_min) break;
                if (q <= p.p_max) ids.push_back(node);
                if (ids.size() > (1ull << 31)) fail(PTSBE_ERR_UNSUPPORTED, "band selects more than 2^31 sets");
            }
        }
        {   // canonical order, by the first two entry words and the arenas on their ties
            struct Keyed { uint64_t w0, w1; uint32_t id; };
            std::vector<Keyed> kv(ids.size());
            for (size_t i = 0; i < ids.size(); ++i) kv[i] = {bf.word(ids[i], 0), bf.word(ids[i], 1), ids[i]};
            std::sort(kv.begin(), kv.end(), [&](const Keyed& a, const Keyed& b) {
                if (a.w0 != b.w0) return a.w0 < b.w0;
                if (a.w1 != b.w1) return a.w1 < b.w1;
                return bf.canon_before(a.id, b.id);
            });
            for (size_t i = 0; i < ids.size(); ++i) ids[i] = kv[i].id;
        }
        out.off.assign(1, 0);
        out.site.clear(); out.k.clear(); out.mult.clear(); out.q.clear(); out.key.clear(); out.shots.clear();
        for (uint32_t id : ids) {
            const uint64_t* e = bf.entries(id);
            for (uint32_t i = 0; i < bf.len(id); ++i) { out.site.push_back((uint32_t)(e[i] >> 8)); out.k.push_back((uint8_t)(e[i] & 0xFF)); }
            out.off.push_back((uint32_t)out.site.size());
        }
        const uint32_t n = (uint32_t)ids.size();
        out.mult.assign(n, 1);
        out.key.resize(n); out.q.resize(n);
        for (uint32_t i = 0; i < n; ++i) {
            out.key[i] = set_key(c, out.site.data() + out.off[i], out.k.data() + out.off[i], out.off[i + 1] - out.off[i]);
            out.q[i] = c.Q0 * out.key[i];
        }
        allocate_shots(out, alloc, p.total_shots, p.shots_per_set);
        out.shot_off.assign(out.count() + 1, 0);
        for (uint32_t i = 0; i < out.count(); ++i) out.shot_off[i + 1] = out.shot_off[i] + out.shots[i];
        return;
    }
    case PTSBE_PTS_TARGETED: {
        if (p.t_count && (!p.t_offsets || !p.t_sites || !p.t_kidx)) fail(PTSBE_ERR_INVALID, "targeted set arrays missing");
        const uint32_t S = (uint32_t)c.site_ch.size();
        for (uint32_t i = 0; i < p.t_count; ++i) {
            const uint32_t b = p.t_offsets[i], e = p.t_offsets[i + 1];
            if (e < b) fail(PTSBE_ERR_INVALID, "targeted offsets decrease");
            List l;
            for (uint32_t j = b; j < e; ++j) {
                const uint32_t s = p.t_sites[j];
                if (s >= S) fail(PTSBE_ERR_INVALID, "targeted site out of range");
                if (p.t_kidx[j] == 0 || p.t_kidx[j] >= c.ch[c.site_ch[s]].nk) fail(PTSBE_ERR_INVALID, "targeted Kraus index out of range");
                if (j > b && s <= p.t_sites[j - 1]) fail(PTSBE_ERR_INVALID, "targeted sites must increase");
                l.push_back({s, p.t_kidx[j]});
            }
            sets.push_back({std::move(l), 1});
        }
        if (alloc == PTSBE_SHOTS_GIVEN) {
            if (!p.t_shots) fail(PTSBE_ERR_INVALID, "SHOTS_GIVEN needs t_shots");
            given.assign(p.t_shots, p.t_shots + p.t_count);
        }
        break;
    }
    case PTSBE_PTS_PREDICATE:
        pts_predicate(c, p, sets);
        break;
    default:
        fail(PTSBE_ERR_INVALID, "unknown PTS mode");
    }
    if (alloc == PTSBE_SHOTS_GIVEN && p.mode != PTSBE_PTS_TARGETED) fail(PTSBE_ERR_INVALID, "SHOTS_GIVEN is for TARGETED");
    finish(c, sets, alloc == PTSBE_SHOTS_GIVEN ? &given : nullptr, out);
    allocate_shots(out, alloc, p.total_shots, p.shots_per_set);
    out.shot_off.assign(out.count() + 1, 0);
    for (uint32_t i = 0; i < out.count(); ++i) out.shot_off[i + 1] = out.shot_off[i] + out.shots[i];
}

}  // namespace ptsbe
