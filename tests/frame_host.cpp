// Host run of the deferred-frame evolution (frame plan, program builder, tile steps) for tests.
// The step functions of the frame kernel take the thread index and count explicitly and touch
// disjoint amplitudes per thread, so running the threads of a CTA one after another, step by
// step, gives the kernel's result. Compiled with g++ from the library sources by the test.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "frame.cuh"
#include "internal.h"

namespace ptsbe {
void build_channel(const ptsbe_channel& in, HostChannel& c);
void register_ops(Circuit& c, const ptsbe_op* ops, uint64_t n_ops, const double* custom, uint32_t n_custom);
void build_device_ops(Circuit& c);
Plan make_frame_plan(const Circuit& c, int tile_bits);
}  // namespace ptsbe

using namespace ptsbe;
using namespace ptsbe::frame;

namespace {

Circuit g_circ;
Plan g_plan;

uint32_t threads_for(int tb) {
    uint32_t t = (1u << tb) / 16;
    return t < 64 ? 64 : (t > 512 ? 512 : t);
}

int g_guard_violations = 0;   // small-buffer stages: tile entries past 2^sbits that were touched
int g_order_checks = 0;       // sparse final stores whose support order (fused sampling) was checked
int g_order_violations = 0;   // ... whose order mask did not rank the support 0 .. N-1 increasingly

// The ranks the fused sampler gives the support entries (bits of the logical index at the order
// mask) must be a bijection onto 0 .. N-1 that increases with the logical index.
void check_support_order(const Step& sp, const DevFrameStage& fs, int n, int lb, const uint32_t* hi) {
    ++g_order_checks;
    const uint32_t H = sparse_order_mask(sp, fs, n, lb, hi);
    if (sp.ncomp == 0xFF || __builtin_popcount(H) != sp.ncomp) { ++g_order_violations; return; }
    const uint32_t N = 1u << sp.ncomp;
    std::vector<int64_t> at(N, -1);
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t l = sparse_logical(sp, fs, n, lb, hi, enum_base(sp, i, nullptr, 0));
        const uint32_t r = extract_bits(l, H);
        if (r >= N || at[r] != -1) { ++g_order_violations; return; }
        at[r] = l;
    }
    for (uint32_t r = 1; r < N; ++r)
        if (at[r] <= at[r - 1]) { ++g_order_violations; return; }
}

void run_cta(const EvolveArgs& a, int stage, bool last, uint32_t node, uint32_t tau, const float* scale_in) {
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    // the small-buffer kernel (sparse final stage with a support bound) runs 128 threads
    const bool small = a.fstages[stage].sparse_final && a.fstages[stage].sbits > 0;
    // the small-buffer kernel runs the program on warps 2-3 (64 threads) and the final store on 128
    const uint32_t nthr = small ? 64u : threads_for(tb);
    const uint32_t nthr_final = small ? 128u : nthr;
    const uint32_t tamps = small ? 1u << a.fstages[stage].sbits : 1u << tb;
    std::vector<float2> tile(1u << tb), tabs((size_t)kMaxTabs * kTabSize);
    // past the buffer the kernel would have: a sentinel that must survive the whole CTA, and that
    // turns any read into NaN in the result
    const uint32_t kSentinel = 0x7fc0a5a5u;
    float sent;
    std::memcpy(&sent, &kSentinel, 4);
    for (uint32_t v = tamps; v < (1u << tb); ++v) tile[v] = make_float2(sent, sent);
    // the small kernel's table buffer holds kMaxTabs << sbits entries: the same sentinel past it
    const size_t tabs_len = small ? ((size_t)kMaxTabs << a.fstages[stage].sbits) : tabs.size();
    for (size_t v = tabs_len; v < tabs.size(); ++v) tabs[v] = make_float2(sent, sent);
    static Builder B;
    static Step S[kProgSteps];
    static Factor pool[kProgPool];
    static Step S2[kMaxSteps];
    static Factor pool2[kMaxPool];
    uint32_t delta[kMaxTabs * kDeltaSlots];
    const DevStage& st = a.stages[stage];
    const DevFrameStage& fs = a.fstages[stage];
    const uint32_t* hi = a.hi + st.hi_off;
    const uint64_t outer = outer_offset(st, ob, tau);
    float2* g = a.states + ((size_t)node << n);
    const uint32_t src = stage == (int)a.node_sstage[node] ? a.node_src[node] : node;
    const float2* gin = a.states_in + ((size_t)src << n);
    builder_init(B, a, st, fs, node, a.node_fresh[node] && stage == 0);
    build_segment(B, S, pool, a, st, kProgSteps, kProgPool);
    const Step* Sp = S;
    const Factor* poolp = pool;
    const bool fresh = a.node_fresh[node] && stage == 0;
    const bool zero_tile = fresh && tau != 0;        // as in the kernel: only tile 0 is nonzero
    for (uint32_t v = 0; v < (tamps >> 1); ++v) {
        if (fresh) {
            tile[2 * v] = make_float2((v == 0 && tau == 0) ? 1.f : 0.f, 0.f);
            tile[2 * v + 1] = make_float2(0.f, 0.f);
        } else {
            const uint64_t gi = gaddr(2u * v, lb, hi, outer);
            tile[2 * v] = gin[gi];
            tile[2 * v + 1] = gin[gi + 1];
        }
    }
    while (true) {
        for (uint32_t si = 0; si < B.nsteps; ++si) {
            const Step& sp = Sp[si];
            if (zero_tile && sp.kind <= ST_DIAG) continue;
            if (sp.ntab && !zero_tile)
                for (uint32_t t = 0; t < nthr; ++t) prepare_tables(sp, fs, poolp, tabs.data(), delta, tb, tau, t, nthr);
            if (sp.kind == ST_MIX1) {
                for (uint32_t t = 0; t < nthr; ++t) run_mix1(sp, poolp, tile.data(), tabs.data(), delta, tb, tau, t, nthr);
            } else if (sp.kind == ST_MIX2) {
                for (uint32_t t = 0; t < nthr; ++t) run_mix2(sp, tile.data(), tabs.data(), delta, tb, tau, t, nthr);
            } else if (sp.kind == ST_DIAG) {
                for (uint32_t t = 0; t < nthr; ++t) run_diag(sp, tile.data(), tabs.data(), delta, tb, t, nthr);
            } else if (sp.kind == ST_FINAL && fs.sparse_final) {
                double part = 0;
                for (uint32_t t = 0; t < nthr_final; ++t)
                    part += run_sparse_final(sp, fs, tile.data(), tabs.data(), delta, n, lb, hi, nullptr, 1.f, 0, t, nthr_final);
                const double w = a.wmix[node] * part;
                const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
                const float scale = null ? 0.0f : (float)(1.0 / std::sqrt(part));
                for (size_t i = 0; i < (1ull << n); ++i) g[i] = make_float2(0.f, 0.f);
                if (!null) {
                    for (uint32_t t = 0; t < nthr_final; ++t)
                        run_sparse_final(sp, fs, tile.data(), tabs.data(), delta, n, lb, hi, g, scale, 1, t, nthr_final);
                    check_support_order(sp, fs, n, lb, hi);
                }
                a.weights[node] = w;
                a.status[node] = null ? 1 : 0;
            } else if (sp.kind == ST_STORE) {
                double part = 0;
                for (uint32_t t = 0; t < nthr; ++t)
                    part += run_store(sp, st, tile.data(), tabs.data(), delta, tb, lb, ob, hi, tau, g, t, nthr, zero_tile);
                if (a.store_norm) a.part[((size_t)node << ob) + tau] = part;
            } else if (!last) {
                for (uint32_t t = 0; t < nthr; ++t)
                    run_final(sp, fs, tile.data(), tabs.data(), delta, tb, ob, tau, g, 1.f, false, t, nthr, zero_tile);
            } else if (scale_in) {
                for (uint32_t t = 0; t < nthr; ++t)
                    run_final(sp, fs, tile.data(), tabs.data(), delta, tb, ob, tau, g, scale_in[node], false, t, nthr, zero_tile);
            } else if (ob == 0) {
                double part = 0;
                for (uint32_t t = 0; t < nthr; ++t)
                    part += run_final(sp, fs, tile.data(), tabs.data(), delta, tb, ob, tau, nullptr, 1.f, true, t, nthr);
                const double w = a.wmix[node] * part;
                const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
                const float scale = null ? 0.0f : (float)(1.0 / std::sqrt(part));
                for (uint32_t t = 0; t < nthr; ++t)
                    run_final(sp, fs, tile.data(), tabs.data(), delta, tb, ob, tau, g, scale, false, t, nthr);
                a.weights[node] = w;
                a.status[node] = null ? 1 : 0;
            } else {
                double part = 0;
                for (uint32_t t = 0; t < nthr; ++t)
                    part += run_final(sp, fs, tile.data(), tabs.data(), delta, tb, ob, tau, g, 1.f, true, t, nthr, zero_tile);
                a.part[((size_t)node << ob) + tau] = part;
            }
        }
        if (B.done) break;
        build_segment(B, S2, pool2, a, st, kMaxSteps, kMaxPool);
        Sp = S2;
        poolp = pool2;
    }
    for (uint32_t v = tamps; v < (1u << tb); ++v) {
        uint32_t bx, by;
        std::memcpy(&bx, &tile[v].x, 4);
        std::memcpy(&by, &tile[v].y, 4);
        if (bx != kSentinel || by != kSentinel) ++g_guard_violations;
    }
    for (size_t v = tabs_len; v < tabs.size(); ++v) {
        uint32_t bx, by;
        std::memcpy(&bx, &tabs[v].x, 4);
        std::memcpy(&by, &tabs[v].y, 4);
        if (bx != kSentinel || by != kSentinel) ++g_guard_violations;
    }
}

}  // namespace

extern "C" {

int fh_register(uint32_t n, const ptsbe_op* ops, uint64_t n_ops, const ptsbe_channel* chans, uint32_t n_ch,
                const double* custom, uint32_t n_custom, int tile_bits) {
    try {
        g_circ = Circuit();
        g_circ.n = n;
        g_circ.ch.resize(n_ch);
        for (uint32_t j = 0; j < n_ch; ++j) build_channel(chans[j], g_circ.ch[j]);
        register_ops(g_circ, ops, n_ops, custom, n_custom);
        build_device_ops(g_circ);
        g_plan = make_frame_plan(g_circ, tile_bits);
        return (int)g_plan.stages.size();
    } catch (const Error& e) {
        return -e.status;
    }
}

// Sets in CSR (off, site, k) with nominal probabilities q; the same schedule as ptsbe_evolve_batch
// (prefix reuse, alternating buffers, early norm when the last stage has no ops).
// Support bits of the plan's sparse final stage (0: none, or no support bound).
// Randomised check of the support order used by fused sampling: random supports (coset
// generators comp[j] of a 14-bit tile) under random invertible index maps (rowe) and offsets;
// the order mask must rank the 2^ncomp members 0 .. N-1 increasingly when the generators are
// independent, and show fewer than ncomp bits exactly when they are dependent.
int fh_order_selftest(uint64_t seed, int trials) {
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
    auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; };
    int bad = 0;
    static Step st;
    static DevFrameStage fs;
    const uint32_t hi0[1] = {0};
    for (int t = 0; t < trials; ++t) {
        const int n = 4 + (int)(rnd() % 17);                 // 4 .. 20 qubits
        const int tbits = n < 14 ? n : 14;
        std::memset(&fs, 0, sizeof(fs));
        std::memset(&st, 0, sizeof(st));
        for (int q = 0; q < n; ++q) fs.rowe[q] = 1u << q;
        for (int k = 0; k < 4 * n; ++k) {                     // random invertible rows: row additions
            const int a = (int)(rnd() % n), b = (int)(rnd() % n);
            if (a != b) fs.rowe[a] ^= fs.rowe[b];
        }
        st.ncomp = (uint8_t)(rnd() % 11);
        for (int j = 0; j < st.ncomp; ++j) {
            uint32_t v = 0;
            while (!v) v = (uint32_t)(rnd() & ((1u << tbits) - 1u));
            st.comp[j] = (uint16_t)v;
        }
        st.lb0 = (uint32_t)(rnd() & ((1u << n) - 1u));
        const uint32_t H = sparse_order_mask(st, fs, n, 14, hi0);
        const uint32_t N = 1u << st.ncomp;
        std::vector<int64_t> at(N, -1);
        std::vector<uint32_t> seen;
        bool distinct = true;
        for (uint32_t i = 0; i < N; ++i) seen.push_back(sparse_logical(st, fs, n, 14, hi0, enum_base(st, i, nullptr, 0)));
        std::vector<uint32_t> sorted = seen;
        std::sort(sorted.begin(), sorted.end());
        for (uint32_t i = 1; i < N; ++i) if (sorted[i] == sorted[i - 1]) distinct = false;
        if ((__builtin_popcount(H) == st.ncomp) != distinct) { ++bad; continue; }
        if (!distinct) continue;
        for (uint32_t i = 0; i < N; ++i) {
            const uint32_t r = extract_bits(seen[i], H);
            if (r >= N || at[r] != -1) { ++bad; break; }
            at[r] = seen[i];
        }
        for (uint32_t r = 0; r < N; ++r)
            if (at[r] != (int64_t)sorted[r]) { ++bad; break; }
    }
    return bad;
}

void fh_order_stats(int* checks, int* violations) {
    *checks = g_order_checks;
    *violations = g_order_violations;
}

int fh_sparse_bits() {
    for (const DevFrameStage& f : g_plan.fstages)
        if (f.sparse_final) return (int)f.sbits;
    return 0;
}

int fh_evolve(uint32_t count, const uint32_t* off, const uint32_t* site, const uint8_t* kk, const double* q, int reuse,
              float2* states, double* weights, uint8_t* status) {
    const Circuit& c = g_circ;
    const Plan& P = g_plan;
    const uint32_t S = (uint32_t)c.site_op.size(), J = (uint32_t)P.stages.size();
    std::vector<uint32_t> ebeg(count), eend(count), sstage(count), src(count);
    std::vector<uint8_t> fresh(count);
    std::vector<double> wmix(count), qa(count);
    std::unordered_map<std::string, uint32_t> index;
    auto key_of = [&](uint32_t a, uint32_t len) {
        std::string k(len * 5, '\0');
        for (uint32_t i = 0; i < len; ++i) {
            std::memcpy(&k[5 * i], &site[off[a] + i], 4);
            k[5 * i + 4] = (char)kk[off[a] + i];
        }
        return k;
    };
    for (uint32_t a = 0; a < count; ++a) {
        const uint32_t len = off[a + 1] - off[a];
        ebeg[a] = off[a]; eend[a] = off[a + 1]; qa[a] = q[a];
        uint32_t parent = UINT32_MAX;
        if (reuse) {
            for (int64_t p = (int64_t)len - 1; p >= 0; --p) {
                auto it = index.find(key_of(a, (uint32_t)p));
                if (it != index.end()) { parent = it->second; break; }
            }
            index.emplace(key_of(a, len), a);
        }
        sstage[a] = 0; src[a] = a; fresh[a] = 1;
        if (parent != UINT32_MAX) {
            const uint32_t plen = off[parent + 1] - off[parent];
            const uint32_t j = (uint32_t)P.op_stage[c.site_op[site[off[a] + plen]]];
            if (j > 0) { sstage[a] = j; src[a] = sstage[parent] == j ? src[parent] : parent; fresh[a] = 0; }
        }
        double w = 1.0;
        uint32_t e = off[a];
        for (uint32_t s = 0; s < S; ++s) {
            uint32_t k = 0;
            if (e < off[a + 1] && site[e] == s) k = kk[e++];
            const HostChannel& ch = c.ch[c.site_ch[s]];
            if (ch.mixture) w *= ch.q[k];
        }
        wmix[a] = w;
    }
    const int ob = (int)c.n - P.tb;
    std::vector<double> part(((size_t)count << ob) + 1);
    std::vector<float2> other(J > 1 ? ((size_t)count << c.n) : 1);
    std::vector<float> scale(count);
    EvolveArgs A{};
    A.ops = c.dops.data(); A.micro = c.dmicro.data(); A.mats = c.dmats.data(); A.chans = c.dchans.data();
    A.site_op = c.site_op.data(); A.stages = P.stages.data(); A.hi = P.hi.data(); A.fstages = P.fstages.data();
    A.n = (int)c.n; A.tb = P.tb; A.lb = P.lb;
    A.ent_site = site; A.ent_k = kk;
    A.node_ebeg = ebeg.data(); A.node_eend = eend.data(); A.node_sstage = sstage.data(); A.node_src = src.data();
    A.node_fresh = fresh.data(); A.wmix = wmix.data(); A.qalpha = qa.data();
    A.part = part.data(); A.weights = weights; A.status = status;
    float2* oth = J > 1 ? other.data() : states;
    auto out_buf = [&](uint32_t j) { return ((J - 1 - j) & 1u) ? oth : states; };
    const bool early = ob > 0 && J >= 2 && P.stages[J - 1].op_begin == P.stages[J - 1].op_end;
    int sparse_stage = -1;
    for (uint32_t j = 0; j < J; ++j)
        if (P.fstages[j].sparse_final) sparse_stage = (int)j;
    auto reduce = [&]() {
        for (uint32_t a = 0; a < count; ++a) {
            double T = 0;
            for (uint32_t t = 0; t < (1u << ob); ++t) T += part[((size_t)a << ob) + t];
            const double w = wmix[a] * T;
            const bool null = !(T > 0.0) || w < 1e-6 * qa[a];
            scale[a] = null ? 0.0f : (float)(1.0 / std::sqrt(T));
            weights[a] = w;
            status[a] = null ? 1 : 0;
        }
    };
    g_guard_violations = 0;
    for (uint32_t j = 0; j < J; ++j) {
        A.states = out_buf(j);
        A.states_in = j > 0 ? out_buf(j - 1) : out_buf(j);
        A.store_norm = early && j + 2 == J;
        const float* sin = early && j + 1 == J ? scale.data() : nullptr;
        for (uint32_t a = 0; a < count; ++a)
            if (sstage[a] <= j)
                for (uint32_t tau = 0; tau < ((int)j == sparse_stage ? 1u : (1u << ob)); ++tau)
                    run_cta(A, (int)j, j + 1 == J, a, tau, sin);
        if (A.store_norm) reduce();
    }
    if (ob > 0 && !early && sparse_stage < 0) {
        reduce();
        for (uint32_t a = 0; a < count; ++a)
            for (size_t i = 0; i < (1ull << c.n); ++i) {
                states[((size_t)a << c.n) + i].x *= scale[a];
                states[((size_t)a << c.n) + i].y *= scale[a];
            }
    }
    return g_guard_violations ? -100 : 0;
}

}  // extern "C"
