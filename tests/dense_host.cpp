// Host run of the dense tile passes (dense planner + the kernel's per-thread code) for tests.
// Within a register group every thread touches its own 16 amplitudes, and the tile load and store
// phases move disjoint amplitudes per thread, so running the threads of a CTA one after another,
// phase by phase, gives the kernel's result. Compiled with g++ from the library sources.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "internal.h"

namespace ptsbe {
void build_channel(const ptsbe_channel& in, HostChannel& c);
void register_ops(Circuit& c, const ptsbe_op* ops, uint64_t n_ops, const double* custom, uint32_t n_custom);
void build_device_ops(Circuit& c);
}  // namespace ptsbe

using namespace ptsbe;
using namespace ptsbe::dense;

namespace {

Circuit g_circ;
DensePlan g_plan;
int g_stage_errors = 0;     // staged passes whose size disagrees with the staging offsets
int g_pad_errors = 0;       // nonzero amplitudes on the padding qubits of a plan padded to kT qubits

// One pass of one state, in place (a tile is read whole before it is written).
void run_pass(uint32_t j, std::vector<float2>& psi, const std::vector<Override>& ovr, const std::vector<float2>& opool) {
    const DensePlan& P = g_plan;
    const Pass& ps = P.passes[j];
    const int ob = P.n - kT;
    std::vector<float2> tile(1u << kT);
    const uint32_t* hi = &P.hi[ps.hi_off];
    const uint16_t* omap = &P.omap[ps.omap_off];
    // the kernel's shared-memory staging of the pass (same offsets), or the plan's arrays
    std::vector<unsigned char> stage(ps.stage_bytes + 16);
    const Group* groups = &P.groups[ps.group_begin];
    const Block* blocks = &P.blocks[ps.blk_begin];
    const float2* mats = &P.mats[ps.mat_begin];
    if (ps.stage_bytes) {
        unsigned char* base = stage.data();
        while ((uintptr_t)base % 16) ++base;
        std::memcpy(base, groups, (ps.group_end - ps.group_begin) * sizeof(Group));
        std::memcpy(base + dense_stage_blocks_off(ps), blocks, (ps.blk_end - ps.blk_begin) * sizeof(Block));
        std::memcpy(base + dense_stage_mats_off(ps), mats, (ps.mat_end - ps.mat_begin) * sizeof(float2));
        if (dense_stage_mats_off(ps) + (ps.mat_end - ps.mat_begin) * sizeof(float2) != ps.stage_bytes) ++g_stage_errors;
        groups = reinterpret_cast<const Group*>(base);
        blocks = reinterpret_cast<const Block*>(base + dense_stage_blocks_off(ps));
        mats = reinterpret_cast<const float2*>(base + dense_stage_mats_off(ps));
    }
    for (uint64_t tau = 0; tau < (1ull << ob); ++tau) {
        const uint64_t outer = outer_offset(ps, tau);
        for (uint32_t tid = 0; tid < (uint32_t)kThreads; ++tid)
            for (int i = 0; i < (1 << (kT - 1)) / kThreads; ++i) {
                const uint32_t t = 2u * (i * kThreads + tid);
                const uint64_t g = outer + (t & 15u) + hi[t >> kC];
                const uint32_t s = swz(t);
                tile[s] = psi[g];
                tile[s ^ 1u] = psi[g + 1];
            }
        size_t ov = 0;
        while (ov < ovr.size() && ovr[ov].block < ps.blk_begin) ++ov;
        for (uint32_t gi = 0; gi < ps.group_end - ps.group_begin; ++gi) {
            const Group& G = groups[gi];
            // the override cursor is uniform over the CTA: every thread sees the same blocks
            const size_t ov0 = ov;
            for (uint32_t tid = 0; tid < (uint32_t)kThreads; ++tid) {
                ov = ov0;
                const uint32_t base = group_base(G, tid);
                alignas(16) float2 v[kAmps];
                for (int jj = 0; jj < kAmps; ++jj) v[jj] = tile[base ^ G.roff[jj]];
                for (uint32_t b = G.blk_begin - ps.blk_begin; b < G.blk_end - ps.blk_begin; ++b) {
                    const Block& B = blocks[b];
                    const float2* m = mats + (B.mat - ps.mat_begin);
                    int code = B.code;
                    if (ov < ovr.size() && ovr[ov].block == B.id) { m = &opool[ovr[ov].mat]; code = (int)ovr[ov].code; ++ov; }
                    apply_block(v, code, m);
                }
                for (int jj = 0; jj < kAmps; ++jj) tile[base ^ G.roff[jj]] = v[jj];
            }
        }
        for (uint32_t tid = 0; tid < (uint32_t)kThreads; ++tid)
            for (int i = 0; i < (1 << (kT - 1)) / kThreads; ++i) {
                const uint32_t L = 2u * (i * kThreads + tid);
                const uint32_t t0 = omap[L >> kC] ^ ps.olow[L & 15u];
                const uint64_t g = outer + (L & 15u) + hi[L >> kC];
                psi[g] = tile[swz(t0)];
                psi[g + 1] = tile[swz(t0 ^ ps.olow[1])];
            }
    }
}

}  // namespace

extern "C" {

// Registers the circuit and builds its dense plan; returns the number of passes (or -status).
int dh_register(uint32_t n, const ptsbe_op* ops, uint64_t n_ops, const ptsbe_channel* chans, uint32_t n_ch,
                const double* custom, uint32_t n_custom) {
    try {
        g_circ = Circuit();
        g_circ.n = n;
        g_circ.ch.resize(n_ch);
        for (uint32_t j = 0; j < n_ch; ++j) build_channel(chans[j], g_circ.ch[j]);
        register_ops(g_circ, ops, n_ops, custom, n_custom);
        build_device_ops(g_circ);
        make_dense_plan(g_circ, g_plan);
        return (int)g_plan.passes.size();
    } catch (const Error& e) {
        return -e.status;
    }
}

// Nonzero amplitudes found on padding qubits by dh_evolve so far (0 when the plan is not padded).
int dh_pad_errors() { return g_pad_errors; }

// out[0..10]: passes, fix-up passes, groups, blocks, operations placed, operations placed more than
// once or never, 2-qubit blocks, gates, passes staged in shared memory, staging size mismatches,
// blocks in diagonal-times-real form
void dh_stats(uint64_t* out) {
    const DensePlan& P = g_plan;
    std::vector<int> seen(g_circ.ops.size(), 0);
    for (uint32_t op : P.blk_ops) ++seen[op];
    uint64_t bad = 0;
    for (int x : seen) bad += x != 1;
    uint64_t two = 0;
    for (uint8_t q : P.blk_nq) two += q == 2;
    uint64_t gates = 0;
    for (uint32_t g : P.pass_gates) gates += g;
    out[0] = P.passes.size();
    out[1] = P.fixup_passes;
    out[2] = P.groups.size();
    out[3] = P.blocks.size();
    out[4] = P.blk_ops.size();
    out[5] = bad;
    out[6] = two;
    out[7] = gates;
    uint64_t staged = 0;
    for (const Pass& ps : P.passes) staged += ps.stage_bytes != 0;
    out[8] = staged;
    out[9] = (uint64_t)g_stage_errors;
    uint64_t dr = 0;
    for (const Block& B : P.blocks) dr += B.code >= kCodeDR;
    out[10] = dr;
}

// Prepares the state of one Kraus set (entries sorted by site) from |0...0> through every pass, as
// the kernel does; writes the unnormalised state (complex64) and returns its weight
// prod_{mixture sites} q_{s,k} * ||psi||^2.
double dh_evolve(const uint32_t* sites, const uint8_t* ks, uint32_t len, float* out) {
    const DensePlan& P = g_plan;
    const int n = P.n;
    std::vector<float2> psi((size_t)1 << n, make_float2(0.f, 0.f));
    psi[0] = make_float2(1.f, 0.f);
    // override blocks of the set (as the library builds them)
    std::vector<std::pair<uint32_t, uint32_t>> eb;
    for (uint32_t e = 0; e < len; ++e) eb.push_back({P.site_block[sites[e]], e});
    std::sort(eb.begin(), eb.end());
    std::vector<Override> ovr;
    std::vector<float2> opool;
    for (size_t i = 0; i < eb.size();) {
        const uint32_t blk = eb[i].first;
        std::vector<uint32_t> ss;
        std::vector<uint8_t> kk;
        for (; i < eb.size() && eb[i].first == blk; ++i) { ss.push_back(sites[eb[i].second]); kk.push_back(ks[eb[i].second]); }
        const uint32_t off = (uint32_t)opool.size();
        opool.resize(off + (P.blk_nq[blk] == 1 ? 4 : 16));
        uint32_t code = 0;
        dense_block_matrix(g_circ, P, blk, ss.data(), kk.data(), (uint32_t)ss.size(), &opool[off], &code);
        ovr.push_back({blk, off, code});
    }
    for (uint32_t j = 0; j < P.passes.size(); ++j) run_pass(j, psi, ovr, opool);
    // a plan padded to kT qubits: the circuit's state is the first 2^n amplitudes, the rest zero
    const size_t amps = (size_t)1 << g_circ.n;
    for (size_t i = amps; i < psi.size(); ++i)
        if (psi[i].x != 0.f || psi[i].y != 0.f) ++g_pad_errors;
    double nrm = 0;
    for (size_t i = 0; i < amps; ++i) {
        out[2 * i] = psi[i].x;
        out[2 * i + 1] = psi[i].y;
        nrm += (double)psi[i].x * psi[i].x + (double)psi[i].y * psi[i].y;
    }
    double w = 1.0;
    uint32_t e = 0;
    for (uint32_t s = 0; s < g_circ.site_op.size(); ++s) {
        uint32_t k = 0;
        if (e < len && sites[e] == s) k = ks[e++];
        const HostChannel& ch = g_circ.ch[g_circ.site_ch[s]];
        if (ch.mixture) w *= ch.q[k];
    }
    return w * nrm;
}

// Group statistics: for every group, the number of distinct float2 bank pairs hit by the first 16
// lanes of a warp (16 = conflict-free); returns the number of groups below 16 and writes the mean.
uint64_t dh_bank_stats(double* mean_pairs) {
    const DensePlan& P = g_plan;
    uint64_t bad = 0;
    double sum = 0;
    for (const Group& G : P.groups) {
        bool hit[16] = {false};
        int distinct = 0;
        for (uint32_t lane = 0; lane < 16; ++lane) {
            const uint32_t b = group_base(G, lane) & 15u;
            if (!hit[b]) { hit[b] = true; ++distinct; }
        }
        sum += distinct;
        bad += distinct < 16;
    }
    if (mean_pairs) *mean_pairs = P.groups.empty() ? 16.0 : sum / (double)P.groups.size();
    return bad;
}

}  // extern "C"
