// Deferred-frame tile pass of batched state preparation (the default evolve kernel).
//
// Most operators of a noisy, CX-heavy circuit are monomial inside a tile: a permutation of basis
// states times a diagonal (CX, CZ, SWAP, Pauli errors, amplitude-damping Kraus operators, and
// two-qubit gates fused with their no-error operators). Moving 2^tb amplitudes through shared
// memory for each of them is what bounds the per-operator sweep. Here the tile is kept in a frame
//
//     psi(l) = D(p) * s[p],      p = A l ^ b,
//
// l the logical tile index, s the tile in shared memory, A an invertible matrix over GF(2)
// (column j = col[j], the physical image of logical bit j), b a translation, and D a product of
// factors f(<r1,p>, <r2,p>) of parities of the physical address (<r,p> = popcount(r & p) mod 2).
// A permutation only updates A and b, a diagonal only adds a factor; operators that mix
// amplitudes (a general 2x2 or 4x4) run as tile passes, and stores write logical order. Before a
// mixing pass, the factors that are not constant along its pair directions are applied (they do
// not commute with it); the others stay deferred. At every pass, the factors it applies are
// grouped into at most kMaxTabs tables of 2^d entries, d <= kTabBits: a table is indexed by the
// parities of the address against d basis rows, so a lookup replaces a product of factors.
//
// One thread turns the op list of the stage into a short program (steps); the CTA runs it. The
// step functions take the thread index and count explicitly and touch disjoint amplitudes per
// thread, so the host can run them one thread at a time.
#pragma once
#include <cstdint>

#include "internal.h"

#ifdef __CUDACC__
#define PTSBE_HD __host__ __device__ __forceinline__
#define PTSBE_HD_CALL __host__ __device__ __noinline__
#else
#define PTSBE_HD inline
#define PTSBE_HD_CALL inline
#endif

namespace ptsbe {
namespace frame {

constexpr int kMaxSteps = 40;
constexpr int kMaxTabs = 3;
constexpr int kTabBits = 10;
constexpr int kTabSize = 1 << kTabBits;
constexpr int kMaxPending = 40;
constexpr int kMaxPool = 256;
constexpr int kStepsPerOp = 16;                      // worst case steps one op can emit
constexpr int kPoolPerOp = 4 * kMaxPending;          // worst case pool entries one op can take
constexpr int kDeltaSlots = 16;                      // per-table index deltas of a step

enum : uint8_t { ST_MIX1 = 0, ST_MIX2 = 1, ST_DIAG = 2, ST_STORE = 3 };

struct Factor {
    uint16_t r1, r2;   // value f[2 <r1,p> + <r2,p>]
    uint16_t c1, c2;   // r1, r2 in the coordinates of the table basis (set when grouped)
    float2 f[4];
};

struct Table {
    uint16_t fb, fe;                 // pool factors [fb, fe)
    uint8_t d, pad[3];
    uint16_t basis[kTabBits];        // index bit i = <basis[i], p>
};

struct Step {
    uint8_t kind, ntab, pa, pb;      // MIX1/MIX2: pivot bits of the pair enumeration
    uint16_t u, v;                   // MIX1: pair direction u; MIX2: directions of the two qubits
    uint16_t ra, rb;                 // MIX: rows giving the logical bits of the operand qubits
    uint8_t ca, cb, ident, pad;      // MIX: parities <ra,b>, <rb,b>; STORE: frame is the identity
    uint16_t col[kTileMax];          // STORE: frame columns
    uint16_t bv, pad2;               // STORE: frame translation
    Table tab[kMaxTabs];
    float2 m[16];                    // MIX1: 2x2, MIX2: 4x4 on 2 l_a + l_b
};

struct Builder {
    uint16_t col[kTileMax], row[kTileMax];   // A and A^-1 (rows)
    uint16_t bv, pad;
    uint32_t op, e, ee;                      // next op and entry cursor of the node
    uint32_t npend, nsteps, npool, done;
    uint16_t ech[kTabBits], comb[kTabBits];  // echelon rows of the table being filled
    uint8_t piv[kTabBits], pad2[2];
    Factor pend[kMaxPending];
};

// Program of one (state, stage): built once by a prepass kernel, shared by the state's tiles.
struct Program {
    Builder B;
    Step S[kMaxSteps];
    Factor pool[kMaxPool];
};

PTSBE_HD uint32_t par(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __popc(x) & 1u;
#else
    return __builtin_popcount(x) & 1u;
#endif
}
PTSBE_HD int low_bit(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __ffs((int)x) - 1;
#else
    return __builtin_ctz(x);
#endif
}
PTSBE_HD int high_bit(uint32_t x) {
#ifdef __CUDA_ARCH__
    return 31 - __clz((int)x);
#else
    return 31 - __builtin_clz(x);
#endif
}
PTSBE_HD float2 fmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
PTSBE_HD float2 fmul2(float2 a, float2 b, float2 c, float2 d) {   // a*b + c*d
    float2 r = fmul(c, d);
    r.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, r.x));
    r.y = fmaf(a.x, b.y, fmaf(a.y, b.x, r.y));
    return r;
}
PTSBE_HD uint32_t ins0(uint32_t i, int p) { return ((i >> p) << (p + 1)) | (i & ((1u << p) - 1u)); }
PTSBE_HD uint32_t ins00(uint32_t i, int pa, int pb) {
    const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
    return ins0(ins0(i, lo), hi);
}
PTSBE_HD bool is_one(float2 z) { return z.x == 1.0f && z.y == 0.0f; }

// ------------------------------------------------------------------------------------------
// Builder (one thread)
// ------------------------------------------------------------------------------------------

// Reduces r against the echelon rows of a table; returns its coordinates, adding r to the basis
// when it is new. d > kTabBits on return means the table is full.
PTSBE_HD uint32_t reduce_or_add(uint32_t r, Table& T, uint16_t* ech, uint16_t* comb, uint8_t* piv, int& d) {
    if (r == 0) return 0;
    uint32_t x = r, cm = 0;
    for (int i = 0; i < d; ++i)
        if ((x >> piv[i]) & 1u) { x ^= ech[i]; cm ^= comb[i]; }
    if (x == 0) return cm;
    if (d >= kTabBits) { d = kTabBits + 1; return 0; }
    T.basis[d] = (uint16_t)r;
    ech[d] = (uint16_t)x;
    comb[d] = (uint16_t)(cm ^ (1u << d));
    piv[d] = (uint8_t)high_bit(x);
    ++d;
    return 1u << (d - 1);
}

// Groups the pending factors of `mask` into tables of st; copies them into the pool. Returns the
// factors that found a table (all of them unless more than kMaxTabs tables would be needed).
PTSBE_HD uint64_t fill_tables(Builder& B, Step& st, Factor* pool, uint64_t mask) {
    st.ntab = 0;
    uint64_t used = 0, left = mask;
    while (left && st.ntab < kMaxTabs) {
        Table& T = st.tab[st.ntab];
        uint16_t* ech = B.ech;
        uint16_t* comb = B.comb;
        uint8_t* piv = B.piv;
        int d = 0;
        T.fb = (uint16_t)B.npool;
        uint64_t took = 0;
        for (uint32_t j = 0; j < B.npend; ++j) {
            if (!((left >> j) & 1u)) continue;
            const Factor& f = B.pend[j];
            const int d0 = d;
            const uint32_t c1 = reduce_or_add(f.r1, T, ech, comb, piv, d);
            uint32_t c2 = 0;
            if (d <= kTabBits) c2 = reduce_or_add(f.r2, T, ech, comb, piv, d);
            if (d > kTabBits) { d = d0; continue; }
            Factor& g = pool[B.npool++];
            g = f;
            g.c1 = (uint16_t)c1;
            g.c2 = (uint16_t)c2;
            took |= 1ull << j;
        }
        T.fe = (uint16_t)B.npool;
        T.d = (uint8_t)d;
        ++st.ntab;
        used |= took;
        left &= ~took;
    }
    return used;
}

// Drops the factors in rm from the pending list; returns keep remapped to the new indices.
PTSBE_HD uint64_t drop_pending(Builder& B, uint64_t rm, uint64_t keep) {
    uint32_t w = 0;
    uint64_t out = 0;
    for (uint32_t j = 0; j < B.npend; ++j) {
        if ((rm >> j) & 1u) continue;
        if ((keep >> j) & 1u) out |= 1ull << w;
        if (w != j) B.pend[w] = B.pend[j];
        ++w;
    }
    B.npend = w;
    return out;
}

// Returns the step S[B.nsteps] with tables for the factors of mask. If they need more than
// kMaxTabs tables, DIAG steps apply the overflow to the tile first (those factors leave the
// pending list). With remove, the factors of the returned step leave the pending list too.
PTSBE_HD Step& take_tables(Builder& B, Step* S, Factor* pool, uint64_t mask, bool remove) {
    while (true) {
        Step& st = S[B.nsteps];
        const uint64_t used = fill_tables(B, st, pool, mask);
        if (used == mask) {
            if (remove) drop_pending(B, used, 0);
            return st;
        }
        st.kind = ST_DIAG;
        ++B.nsteps;
        mask = drop_pending(B, used, mask & ~used);
    }
}

PTSBE_HD uint64_t all_pending(const Builder& B) { return B.npend >= 64 ? ~0ull : ((1ull << B.npend) - 1ull); }

// Adds the factor g[2 <r1,p> + <r2,p>], merging it with a pending factor on the same rows.
PTSBE_HD void push_factor(Builder& B, Step* S, Factor* pool, uint32_t r1, uint32_t r2, const float2* gin) {
    float2 g[4] = {gin[0], gin[1], gin[2], gin[3]};
    if (r1 == 0 && r2 != 0) { r1 = r2; r2 = 0; const float2 t = g[1]; g[1] = g[2]; g[2] = t; }
    if (r2 != 0 && r1 > r2) {
        const uint32_t t = r1; r1 = r2; r2 = t;
        const float2 h = g[1]; g[1] = g[2]; g[2] = h;
    }
    if (r2 == 0) { g[1] = g[0]; g[3] = g[2]; }
    if (r1 == 0) { g[1] = g[2] = g[3] = g[0]; }
    if (is_one(g[0]) && is_one(g[1]) && is_one(g[2]) && is_one(g[3])) return;
    for (uint32_t j = 0; j < B.npend; ++j) {
        Factor& f = B.pend[j];
        if (f.r1 == r1 && f.r2 == r2) {
            for (int x = 0; x < 4; ++x) f.f[x] = fmul(f.f[x], g[x]);
            return;
        }
    }
    if (B.npend == kMaxPending) {
        Step& st = take_tables(B, S, pool, all_pending(B), true);
        st.kind = ST_DIAG;
        ++B.nsteps;
    }
    Factor& f = B.pend[B.npend++];
    f.r1 = (uint16_t)r1; f.r2 = (uint16_t)r2; f.c1 = f.c2 = 0;
    for (int x = 0; x < 4; ++x) f.f[x] = g[x];
}

// diag(d0, d1) on logical bit q
PTSBE_HD void factor1(Builder& B, Step* S, Factor* pool, int q, float2 d0, float2 d1) {
    const uint32_t r = B.row[q], c = par(r & B.bv);
    const float2 g[4] = {c ? d1 : d0, c ? d1 : d0, c ? d0 : d1, c ? d0 : d1};
    push_factor(B, S, pool, r, 0, g);
}

// diagonal d[2 l_a + l_b] on logical bits (a, b)
PTSBE_HD void factor2(Builder& B, Step* S, Factor* pool, int a, int b, const float2* d) {
    const uint32_t ra = B.row[a], rb = B.row[b];
    const uint32_t x = 2u * par(ra & B.bv) + par(rb & B.bv);
    const float2 g[4] = {d[0 ^ x], d[1 ^ x], d[2 ^ x], d[3 ^ x]};
    push_factor(B, S, pool, ra, rb, g);
}

PTSBE_HD uint64_t varying(const Builder& B, uint32_t u, uint32_t v) {
    uint64_t m = 0;
    for (uint32_t j = 0; j < B.npend; ++j) {
        const Factor& f = B.pend[j];
        if (par(f.r1 & u) | par(f.r2 & u) | par(f.r1 & v) | par(f.r2 & v)) m |= 1ull << j;
    }
    return m;
}

PTSBE_HD void emit_mix1(Builder& B, Step* S, Factor* pool, int q, const float2* m) {
    const uint32_t u = B.col[q];
    Step& st = take_tables(B, S, pool, varying(B, u, 0), true);
    st.kind = ST_MIX1;
    st.u = (uint16_t)u;
    st.pa = (uint8_t)low_bit(u);
    st.ra = B.row[q];
    st.ca = (uint8_t)par(B.row[q] & B.bv);
    for (int i = 0; i < 4; ++i) st.m[i] = m[i];
    ++B.nsteps;
}

PTSBE_HD void emit_mix2(Builder& B, Step* S, Factor* pool, int a, int b, const float2* m) {
    const uint32_t u = B.col[a], v = B.col[b];
    Step& st = take_tables(B, S, pool, varying(B, u, v), true);
    st.kind = ST_MIX2;
    st.u = (uint16_t)u;
    st.v = (uint16_t)v;
    const int pa = low_bit(u);
    const uint32_t v2 = ((v >> pa) & 1u) ? (v ^ u) : v;
    st.pa = (uint8_t)pa;
    st.pb = (uint8_t)low_bit(v2);
    st.ra = B.row[a];
    st.rb = B.row[b];
    st.ca = (uint8_t)par(B.row[a] & B.bv);
    st.cb = (uint8_t)par(B.row[b] & B.bv);
    for (int i = 0; i < 16; ++i) st.m[i] = m[i];
    ++B.nsteps;
}

PTSBE_HD void emit_store(Builder& B, Step* S, Factor* pool, int tb) {
    Step& st = take_tables(B, S, pool, all_pending(B), false);
    st.kind = ST_STORE;
    bool ident = B.bv == 0;
    for (int j = 0; j < tb; ++j) {
        st.col[j] = B.col[j];
        ident = ident && B.col[j] == (1u << j);
    }
    st.bv = B.bv;
    st.ident = ident ? 1 : 0;
    ++B.nsteps;
}

// out[x] = d[x] * in[perm_x] on x = 2 l_a + l_b as a frame change (perm is a bijection).
PTSBE_HD void perm2(Builder& B, int a, int b, const uint32_t* pm) {
    const uint32_t t = pm[0], c1 = pm[1] ^ t, c2 = pm[2] ^ t;   // images of e_b and e_a
    const uint32_t ca = B.col[a], cb = B.col[b], ra = B.row[a], rb = B.row[b];
    B.bv ^= (uint16_t)(((t >> 1) ? ca : 0u) ^ ((t & 1u) ? cb : 0u));
    B.col[a] = (uint16_t)(((c2 >> 1) ? ca : 0u) ^ ((c2 & 1u) ? cb : 0u));
    B.col[b] = (uint16_t)(((c1 >> 1) ? ca : 0u) ^ ((c1 & 1u) ? cb : 0u));
    B.row[a] = (uint16_t)(((c1 & 1u) ? ra : 0u) ^ ((c1 >> 1) ? rb : 0u));
    B.row[b] = (uint16_t)(((c2 & 1u) ? ra : 0u) ^ ((c2 >> 1) ? rb : 0u));
}

// One operator on tile positions (a, b).
PTSBE_HD void process(Builder& B, Step* S, Factor* pool, uint8_t kind, int a, int b, const float2* m, uint32_t perm,
                      bool sep) {
    switch (kind) {
    case DOP_G1: emit_mix1(B, S, pool, a, m); break;
    case DOP_D1: factor1(B, S, pool, a, m[0], m[1]); break;
    case DOP_X1:   // [[0, m0], [m1, 0]]: psi'(l) = d[l_a] psi(l ^ e_a), d = (m0, m1)
        B.bv ^= B.col[a];
        factor1(B, S, pool, a, m[0], m[1]);
        break;
    case DOP_CX:
        B.col[a] ^= B.col[b];
        B.row[b] ^= B.row[a];
        break;
    case DOP_CZ: {
        const float2 d[4] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f), make_float2(1.f, 0.f), make_float2(-1.f, 0.f)};
        factor2(B, S, pool, a, b, d);
        break;
    }
    case DOP_SWAP: {
        uint16_t t = B.col[a]; B.col[a] = B.col[b]; B.col[b] = t;
        t = B.row[a]; B.row[a] = B.row[b]; B.row[b] = t;
        break;
    }
    case DOP_G2: emit_mix2(B, S, pool, a, b, m); break;
    case DOP_M2: {
        const uint32_t pm[4] = {perm & 3u, (perm >> 2) & 3u, (perm >> 4) & 3u, (perm >> 6) & 3u};
        if (((1u << pm[0]) | (1u << pm[1]) | (1u << pm[2]) | (1u << pm[3])) != 15u) {
            float2 g[16];
            for (int i = 0; i < 16; ++i) g[i] = make_float2(0.f, 0.f);
            for (int x = 0; x < 4; ++x) g[4 * x + pm[x]] = m[x];
            emit_mix2(B, S, pool, a, b, g);
            break;
        }
        perm2(B, a, b, pm);
        if (sep) {
            factor1(B, S, pool, a, m[4], m[5]);
            factor1(B, S, pool, b, m[6], m[7]);
        } else {
            factor2(B, S, pool, a, b, m);
        }
        break;
    }
    default: break;   // DOP_NOP
    }
}

PTSBE_HD_CALL void builder_init(Builder& B, const EvolveArgs& a, const DevStage& st, uint32_t node) {
    for (int j = 0; j < kTileMax; ++j) B.col[j] = B.row[j] = (uint16_t)(1u << j);
    B.bv = 0;
    B.op = st.op_begin;
    uint32_t e = a.node_ebeg[node];
    B.ee = a.node_eend[node];
    while (e < B.ee && a.site_op[a.ent_site[e]] < st.op_begin) ++e;
    B.e = e;
    B.npend = 0;
    B.done = 0;
}

// Emits steps until the stage ends (then the final store and done = 1) or the step list or the
// factor pool could overflow with one more op (the next segment continues from B.op).
PTSBE_HD_CALL void build_segment(Builder& B, Step* S, Factor* pool, const EvolveArgs& a, const DevStage& st) {
    B.nsteps = 0;
    B.npool = 0;
    while (true) {
        if (B.nsteps + kStepsPerOp > kMaxSteps || B.npool + kPoolPerOp > kMaxPool) return;
        if (B.op >= st.op_end) {
            emit_store(B, S, pool, a.tb);
            B.done = 1;
            return;
        }
        const uint32_t op = B.op;
        const DevOp o = a.ops[op];
        if (o.kind == DOP_NOISE) {
            uint32_t k = 0;
            if (B.e < B.ee && a.ent_site[B.e] == o.site) { k = a.ent_k[B.e]; ++B.e; }
            const DevChannel& ch = a.chans[o.ch];
            for (uint32_t u = ch.micro_off[k]; u < ch.micro_off[k + 1]; ++u) {
                const DevMicro mi = a.micro[u];
                process(B, S, pool, mi.kind, st.pos[mi.operand == 1 ? o.q1 : o.q0], st.pos[o.q1], a.mats + mi.mat, 0, false);
            }
            B.op = op + 1;
        } else if (o.fend != 0 && (B.e >= B.ee || a.ent_site[B.e] >= o.fsite1)) {
            // no error inside the fused block: gate and no-error operators at once
            process(B, S, pool, o.fkind, st.pos[o.q0], st.pos[o.q1], a.mats + o.fmat, o.fperm, o.fsep != 0);
            B.op = o.fend;
        } else {
            process(B, S, pool, o.kind, st.pos[o.q0], st.pos[o.q1], a.mats + o.mat, 0, false);
            B.op = op + 1;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Steps (every thread of the CTA; thread `tid` of `nthr`)
// ------------------------------------------------------------------------------------------

PTSBE_HD uint32_t lin_idx(const Table& T, uint32_t p) {
    uint32_t r = 0;
    for (int i = 0; i < T.d; ++i) r |= par(T.basis[i] & p) << i;
    return r;
}

// Physical address delta of bit j of the iteration counter (slots < 14), and of the pair
// directions (slots 14, 15), for a step.
PTSBE_HD uint32_t step_delta(const Step& st, int tb, uint32_t nthr, int j) {
    switch (st.kind) {
    case ST_MIX1:
        if (j == 15) return st.u;
        return j < 14 ? ins0(nthr << j, st.pa) & ((1u << tb) - 1u) : 0u;
    case ST_MIX2:
        if (j == 14) return st.v;
        if (j == 15) return st.u;
        return j < 14 ? ins00(nthr << j, st.pa, st.pb) & ((1u << tb) - 1u) : 0u;
    case ST_DIAG:
        return j < 14 ? (nthr << j) & ((1u << tb) - 1u) : 0u;
    default: {   // STORE: logical index l = 2 (tid + k nthr) + {0, 1}
        if (j == 15) return st.col[0];
        int lg = 0;
        while ((1u << lg) < nthr) ++lg;
        const int bit = 1 + lg + j;
        return (j < 14 && bit < tb) ? st.col[bit] : 0u;
    }
    }
}

// Table entries and index deltas of a step (before the pass; a barrier separates them).
PTSBE_HD void prepare_tables(const Step& st, const Factor* pool, float2* tabs, uint32_t* delta, int tb, uint32_t tid,
                             uint32_t nthr) {
    for (int t = 0; t < st.ntab; ++t) {
        const Table& T = st.tab[t];
        const uint32_t size = 1u << T.d;
        for (uint32_t idx = tid; idx < size; idx += nthr) {
            float2 v = make_float2(1.f, 0.f);
            for (uint32_t j = T.fb; j < T.fe; ++j) {
                const Factor& f = pool[j];
                v = fmul(v, f.f[2u * par(f.c1 & idx) + par(f.c2 & idx)]);
            }
            tabs[t * kTabSize + idx] = v;
        }
    }
    const uint32_t nd = (uint32_t)st.ntab * kDeltaSlots;
    for (uint32_t i = tid; i < nd; i += nthr)
        delta[i] = lin_idx(st.tab[i / kDeltaSlots], step_delta(st, tb, nthr, (int)(i % kDeltaSlots)));
}

struct Lookup {
    int ntab;
    uint32_t ix[kMaxTabs];
};

PTSBE_HD float2 apply_tabs(float2 x, const Lookup& L, const float2* tabs, const uint32_t* delta, int slot) {
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t)
        if (t < L.ntab) {
            const uint32_t i = slot < 0 ? L.ix[t] : (L.ix[t] ^ delta[t * kDeltaSlots + slot]);
            x = fmul(x, tabs[t * kTabSize + i]);
        }
    return x;
}

PTSBE_HD void lookup_init(Lookup& L, const Step& st, uint32_t p) {
    L.ntab = st.ntab;
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t) L.ix[t] = t < L.ntab ? lin_idx(st.tab[t], p) : 0u;
}
PTSBE_HD void lookup_step(Lookup& L, const uint32_t* delta, int j) {
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t)
        if (t < L.ntab) L.ix[t] ^= delta[t * kDeltaSlots + j];
}

// The iterations of a thread visit k = 0 .. K-1 in Gray-code order, so each step flips one bit
// of the address and of every table index.
PTSBE_HD void run_mix1(const Step& st, float2* s, const float2* tabs, const uint32_t* delta, int tb, uint32_t tid,
                       uint32_t nthr) {
    const uint32_t N = 1u << (tb - 1);
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    const float2 m00 = st.m[0], m01 = st.m[1], m10 = st.m[2], m11 = st.m[3];
    const uint32_t u = st.u, ra = st.ra, ca = st.ca;
    uint32_t p0 = ins0(tid, st.pa);
    Lookup L;
    lookup_init(L, st, p0);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            p0 ^= ins0(nthr << j, st.pa);
            lookup_step(L, delta, j);
        }
        const uint32_t p1 = p0 ^ u;
        float2 x0 = s[p0], x1 = s[p1];
        if (L.ntab) { x0 = apply_tabs(x0, L, tabs, delta, -1); x1 = apply_tabs(x1, L, tabs, delta, 15); }
        const bool fl = (par(ra & p0) ^ ca) != 0;
        const float2 a = fl ? x1 : x0, b = fl ? x0 : x1;
        const float2 y0 = fmul2(m00, a, m01, b), y1 = fmul2(m10, a, m11, b);
        s[p0] = fl ? y1 : y0;
        s[p1] = fl ? y0 : y1;
    }
}

PTSBE_HD void xswap(float2* z, uint32_t x0) {
    if (x0 & 1u) { float2 t = z[0]; z[0] = z[1]; z[1] = t; t = z[2]; z[2] = z[3]; z[3] = t; }
    if (x0 & 2u) { float2 t = z[0]; z[0] = z[2]; z[2] = t; t = z[1]; z[1] = z[3]; z[3] = t; }
}

PTSBE_HD void run_mix2(const Step& st, float2* s, const float2* tabs, const uint32_t* delta, int tb, uint32_t tid,
                       uint32_t nthr) {
    const uint32_t N = 1u << (tb - 2);
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    const uint32_t w[4] = {0u, st.v, st.u, (uint32_t)(st.u ^ st.v)};   // logical difference y -> offset
    uint32_t base = ins00(tid, st.pa, st.pb);
    Lookup L;
    lookup_init(L, st, base);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            base ^= ins00(nthr << j, st.pa, st.pb);
            lookup_step(L, delta, j);
        }
        float2 z[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) z[y] = s[base ^ w[y]];
        if (L.ntab) {
            z[0] = apply_tabs(z[0], L, tabs, delta, -1);
            z[1] = apply_tabs(z[1], L, tabs, delta, 14);
            z[2] = apply_tabs(z[2], L, tabs, delta, 15);
            Lookup L3 = L;
            lookup_step(L3, delta, 14);
            z[3] = apply_tabs(z[3], L3, tabs, delta, 15);
        }
        const uint32_t x0 = 2u * (par(st.ra & base) ^ st.ca) + (par(st.rb & base) ^ st.cb);
        xswap(z, x0);   // z[x] = amplitude of logical x
        float2 o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float2 acc = fmul(st.m[4 * r], z[0]);
#pragma unroll
            for (int l = 1; l < 4; ++l) {
                const float2 t = fmul(st.m[4 * r + l], z[l]);
                acc.x += t.x; acc.y += t.y;
            }
            o[r] = acc;
        }
        xswap(o, x0);
#pragma unroll
        for (int y = 0; y < 4; ++y) s[base ^ w[y]] = o[y];
    }
}

PTSBE_HD void run_diag(const Step& st, float2* s, const float2* tabs, const uint32_t* delta, int tb, uint32_t tid,
                       uint32_t nthr) {
    const uint32_t N = 1u << tb;
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    uint32_t p = tid;
    Lookup L;
    lookup_init(L, st, p);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            p ^= nthr << j;
            lookup_step(L, delta, j);
        }
        s[p] = apply_tabs(s[p], L, tabs, delta, -1);
    }
}

PTSBE_HD uint64_t gaddr(uint32_t l, int lb, const uint32_t* hi, uint64_t outer) {
    return (uint64_t)(l & ((1u << lb) - 1u)) | (uint64_t)hi[l >> lb] | outer;
}

// Writes the logical tile times `scale` to dst (when not null) and returns this thread's part of
// the squared norm of the logical amplitudes (when want_norm).
PTSBE_HD double run_store(const Step& st, const float2* s, const float2* tabs, const uint32_t* delta, int tb, int lb,
                          const uint32_t* hi, uint64_t outer, float2* dst, float scale, bool want_norm, uint32_t tid,
                          uint32_t nthr) {
    const uint32_t N = 1u << (tb - 1);
    double acc = 0.0;
    if (tid >= N) return acc;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    int lg = 0;
    while ((1u << lg) < nthr) ++lg;
    uint32_t v = tid;
    uint32_t p0 = st.bv;
    for (int b = 0; (1u << b) <= tid; ++b)
        if ((tid >> b) & 1u) p0 ^= st.col[b + 1];
    Lookup L;
    lookup_init(L, st, p0);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            v ^= nthr << j;
            p0 ^= st.col[1 + lg + j];
            lookup_step(L, delta, j);
        }
        float2 a0 = s[p0], a1 = s[p0 ^ st.col[0]];
        if (L.ntab) { a0 = apply_tabs(a0, L, tabs, delta, -1); a1 = apply_tabs(a1, L, tabs, delta, 15); }
        if (want_norm) acc += (double)fmaf(a0.x, a0.x, a0.y * a0.y) + (double)fmaf(a1.x, a1.x, a1.y * a1.y);
        if (dst)
            *reinterpret_cast<float4*>(dst + gaddr(2u * v, lb, hi, outer)) =
                make_float4(a0.x * scale, a0.y * scale, a1.x * scale, a1.y * scale);
    }
    return acc;
}

}  // namespace frame
}  // namespace ptsbe
