// Deferred-frame tile pass of batched state preparation (the default evolve kernel).
//
// Most operators of a noisy, CX-heavy circuit are monomial: a permutation of basis states times a
// diagonal (CX, CZ, SWAP, Pauli errors, amplitude-damping Kraus operators, and gates fused with
// their no-error operators). Moving amplitudes for each of them is what bounds a per-operator
// sweep. Here a state is kept in a frame
//
//     psi(l) = D(x) * s[x],      x = A l ^ b,
//
// l the logical index, x the global (physical) index, s the stored amplitudes, A an invertible
// matrix over GF(2) (column q = col[q], the physical image of logical bit q), b a translation and
// D a product of factors f(<r1,x>, <r2,x>) of parities of the physical index (<r,x> = popcount(r
// & x) mod 2). A permutation updates A and b, a diagonal adds a factor; only operators that mix
// amplitudes (a general 2x2 or 4x4) pass over the tile, along physical directions that the plan
// keeps inside the stage's tile (a set of global index bits). A changes only at gates, so it is
// the same for every Kraus set; b and D are per set. Between stages the state is stored with b
// and D applied (global index x holds psi(A^-1 x)); the last stage writes logical order.
//
// Before a mixing pass, the factors not constant along its directions are applied (they do not
// commute with it); the others stay deferred. The factors a pass applies are grouped into at most
// kMaxTabs tables of 2^d entries (d <= kTabBits), indexed by the parities of the tile-local
// address against d basis rows, so one lookup replaces a product of factors. A factor's parity
// against the outer bits of the index is constant on a tile and folds into its table.
//
// One thread turns the op list of a (set, stage) into a short program (steps); the CTAs of the
// set's tiles run it. The step functions take the thread index and count explicitly and touch
// disjoint amplitudes per thread, so the host can run them one thread at a time.
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

constexpr int kMaxSteps = 40;                        // program segment held in shared memory
constexpr int kMaxPool = 256;
constexpr int kProgSteps = 160;                      // program built by the prepass (global memory)
constexpr int kProgPool = 1024;
constexpr int kMaxTabs = 3;
constexpr int kTabBits = 10;
constexpr int kTabSize = 1 << kTabBits;
constexpr int kMaxPending = 40;
constexpr int kStepsPerOp = 16;                      // worst case steps one op can emit
constexpr int kPoolPerOp = 4 * kMaxPending;          // worst case pool entries one op can take
constexpr int kDeltaSlots = 16;                      // per-table index deltas of a step
constexpr int kMaxDirs = 4;                          // single-qubit mixes grouped into one pass

// MIX1: 1..kMaxDirs single-qubit mixes on independent directions (one pass, 2^ndir amplitudes per
// thread in registers); MIX2: one two-qubit mix; DIAG: factors only; STORE / FINAL: stage end.
enum : uint8_t { ST_MIX1 = 0, ST_MIX2 = 1, ST_DIAG = 2, ST_STORE = 3, ST_FINAL = 4 };

struct Factor {
    uint32_t r1, r2;   // value f[2 <r1,x> + <r2,x>] (global index masks)
    uint32_t r1o, r2o; // outer parts of r1, r2 in tile-index bits (set when grouped)
    uint16_t c1, c2;   // tile parts of r1, r2 in the coordinates of the table basis (set when grouped)
    uint32_t pad;
    float2 f[4];
};

struct Table {
    uint16_t fb, fe;                 // pool factors [fb, fe)
    uint8_t d, real, pad[2];         // real: every factor value is real (float entries, real products)
    uint16_t basis[kTabBits];        // index bit i = <basis[i], tile-local address>
};

struct Step {
    uint8_t kind, ntab, ndir, mreal;   // mreal bit i: the 2x2 of direction i and its folded factors are real
    uint8_t piv[kMaxDirs];           // MIX1: pivot bits of the coset enumeration (ascending); MIX2: pa, pb
    uint16_t dir[kMaxDirs];          // MIX: tile-local directions (MIX2: dir[0] first qubit, dir[1] second)
    uint16_t rin[kMaxDirs];          // MIX: tile parts of the rows of the operand qubits
    uint32_t rout[kMaxDirs];         // MIX: outer parts of those rows; STORE: rout[0] = outer part of b
    uint8_t cpar[kMaxDirs];          // MIX: <row, b>
    uint32_t lb0;                    // FINAL: R b (logical); STORE: tile part of b
    uint32_t npush, nframe;          // builder counters when emitted (grouping test)
    uint16_t fold_b[kMaxDirs], fold_e[kMaxDirs];   // MIX1: pool factors folded into direction i
    // Sparse passes (a stage started from |0...0>): the nonzero amplitudes lie in the span of the
    // directions mixed so far, so MIX / DIAG passes visit only the cosets base = sum_i bit_i comp[i]
    // of that span (complemented by the step's own directions); ncomp = 0xFF: the whole tile.
    uint8_t ncomp, tsb;              // tsb: table t starts at entry t << tsb of the table buffer
    uint16_t comp[kTileMax];
    Table tab[kMaxTabs];
    float2 m[16];                    // MIX1: 2x2 of direction i at m[4i..4i+3]; MIX2: 4x4 on 2 l_a + l_b
};

struct Builder {
    uint32_t col[kMaxQubits], row[kMaxQubits];   // A and the rows of A^-1
    uint32_t bv;
    uint32_t op, e, ee;                          // next op and entry cursor of the set
    uint32_t npend, nsteps, npool, done, last;
    uint32_t npush, nframe;                      // factor changes and frame changes so far
    uint32_t sparse, sdim;                       // support tracking (stage from |0...0>): basis size
    uint32_t sparse_final;                       // the stage ends with the sparse final store
    uint32_t tmask;                              // tile bits a table row keeps (the support's, small stages)
    uint16_t sech[kTileMax];                     // echelon basis of the support (tile-local)
    uint8_t spiv[kTileMax], tsb, pad3;          // tsb: log2 of the table stride of emitted steps
    uint16_t ech[kTabBits], comb[kTabBits];      // echelon rows of the table being filled
    uint32_t freal;                              // the factors folded by the last fold_factors are real
    uint8_t piv[kTabBits], pad2[2];
    Factor pend[kMaxPending];
};

// Program of one (set, stage): built once by a prepass kernel, shared by the set's tiles.
struct Program {
    Builder B;
    Step S[kProgSteps];
    Factor pool[kProgPool];
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
// Both lanes of a float2 times the same real factor, plus an addend: one packed FP32x2 FMA on the
// device (a + b*r per lane), two scalar FMAs on the host.
PTSBE_HD float2 fma2r(float2 b, float r, float2 a) {
#ifdef __CUDA_ARCH__
    unsigned long long d;
    const float2 rr = make_float2(r, r);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&b)), "l"(*reinterpret_cast<const unsigned long long*>(&rr)),
          "l"(*reinterpret_cast<const unsigned long long*>(&a)));
    return *reinterpret_cast<const float2*>(&d);
#else
    return make_float2(fmaf(b.x, r, a.x), fmaf(b.y, r, a.y));
#endif
}
PTSBE_HD float2 mul2r(float2 b, float r) { return fma2r(b, r, make_float2(-0.0f, -0.0f)); }

PTSBE_HD uint32_t ins0(uint32_t i, int p) { return ((i >> p) << (p + 1)) | (i & ((1u << p) - 1u)); }
PTSBE_HD uint32_t ins00(uint32_t i, int pa, int pb) {
    const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
    return ins0(ins0(i, lo), hi);
}
PTSBE_HD bool is_one(float2 z) { return z.x == 1.0f && z.y == 0.0f; }

// Tile-local and outer parts of a global index mask (DevStage::pos: tile bit, or 0x80 | outer bit).
PTSBE_HD uint32_t tile_part(const DevStage& st, uint32_t m) {
    uint32_t r = 0;
    while (m) {
        const int g = low_bit(m);
        m &= m - 1u;
        if (!(st.pos[g] & 0x80)) r |= 1u << st.pos[g];
    }
    return r;
}
PTSBE_HD uint32_t outer_part(const DevStage& st, uint32_t m) {
    uint32_t r = 0;
    while (m) {
        const int g = low_bit(m);
        m &= m - 1u;
        if (st.pos[g] & 0x80) r |= 1u << (st.pos[g] & 0x7F);
    }
    return r;
}

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

// Orders the index bits of a finished table by the lowest set bit of their basis rows. The lanes
// of a warp differ in the low tile-local bits, so their lookups then differ in the low index bits
// and spread over the shared-memory banks.
// The coordinates of pool factors [T.fb, T.fe) in the unordered basis are read from the pending
// factors they were copied from (pend entries of `took`, in order), so the pool entries, possibly
// in global memory, are only written.
PTSBE_HD void order_table(Table& T, Factor* pool, const Factor* pend, uint64_t took) {
    uint8_t ord[kTabBits], at[kTabBits];
    for (int i = 0; i < T.d; ++i) {
        int j = i;
        while (j > 0 && low_bit(T.basis[ord[j - 1]]) > low_bit(T.basis[i])) { ord[j] = ord[j - 1]; --j; }
        ord[j] = (uint8_t)i;
    }
    uint16_t nb[kTabBits];
    for (int i = 0; i < T.d; ++i) { nb[i] = T.basis[ord[i]]; at[ord[i]] = (uint8_t)i; }
    for (int i = 0; i < T.d; ++i) T.basis[i] = nb[i];
    for (uint32_t j = T.fb; j < T.fe; ++j) {
        uint32_t c1 = 0, c2 = 0;
        const int k = (uint32_t)took ? low_bit((uint32_t)took) : 32 + low_bit((uint32_t)(took >> 32));
        took &= took - 1ull;
        const uint32_t u1 = pend[k].c1, u2 = pend[k].c2;
        for (int i = 0; i < T.d; ++i) {
            if ((u1 >> i) & 1u) c1 |= 1u << at[i];
            if ((u2 >> i) & 1u) c2 |= 1u << at[i];
        }
        pool[j].c1 = (uint16_t)c1;
        pool[j].c2 = (uint16_t)c2;
    }
}

// Groups the pending factors of `mask` into tables of st; copies them into the pool. Returns the
// factors that found a table (all of them unless more than kMaxTabs tables would be needed).
PTSBE_HD uint64_t fill_tables(Builder& B, const DevStage& stg, Step& st, Factor* pool, uint64_t mask) {
    st.ntab = 0;
    st.tsb = B.tsb;
    uint64_t used = 0, left = mask;
    while (left && st.ntab < kMaxTabs) {
        Table& T = st.tab[st.ntab];
        int d = 0;
        T.fb = (uint16_t)B.npool;
        uint64_t took = 0;
        uint8_t real = 1;
        for (uint32_t j = 0; j < B.npend; ++j) {
            if (!((left >> j) & 1u)) continue;
            const Factor& f = B.pend[j];
            const int d0 = d;
            const uint32_t c1 = reduce_or_add(tile_part(stg, f.r1) & B.tmask, T, B.ech, B.comb, B.piv, d);
            uint32_t c2 = 0;
            if (d <= kTabBits) c2 = reduce_or_add(tile_part(stg, f.r2) & B.tmask, T, B.ech, B.comb, B.piv, d);
            if (d > kTabBits) { d = d0; continue; }
            B.pend[j].c1 = (uint16_t)c1;     // for order_table (a pending factor's c1, c2 are scratch)
            B.pend[j].c2 = (uint16_t)c2;
            for (int x = 0; x < 4; ++x) if (f.f[x].y != 0.0f) real = 0;
            Factor& g = pool[B.npool++];
            g = f;
            g.c1 = (uint16_t)c1;
            g.c2 = (uint16_t)c2;
            g.r1o = outer_part(stg, f.r1);
            g.r2o = outer_part(stg, f.r2);
            took |= 1ull << j;
        }
        T.fe = (uint16_t)B.npool;
        T.d = (uint8_t)d;
        T.real = real;
        order_table(T, pool, B.pend, took);
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
        if (w != j) {
            // a pending factor only carries its rows and values (r1o, r2o and pad stay zero; c1, c2
            // are scratch of fill_tables, overwritten in every pool copy)
            Factor& d = B.pend[w];
            const Factor& f = B.pend[j];
            d.r1 = f.r1; d.r2 = f.r2;
            for (int x = 0; x < 4; ++x) d.f[x] = f.f[x];
        }
        ++w;
    }
    B.npend = w;
    return out;
}

// Adds a tile-local direction to the support span (echelon with distinct lowest-bit pivots).
PTSBE_HD void support_add(Builder& B, uint32_t u) {
    for (uint32_t i = 0; i < B.sdim; ++i)
        if ((u >> B.spiv[i]) & 1u) u ^= B.sech[i];
    if (!u) return;
    B.sech[B.sdim] = (uint16_t)u;
    B.spiv[B.sdim] = (uint8_t)low_bit(u);
    ++B.sdim;
}

// Coset representatives of span(dirs) inside the support: the support basis reduced against the
// directions, keeping the independent remainders. The whole tile when the support is unknown.
PTSBE_HD void set_enumeration(const Builder& B, Step& st, const uint16_t* dirs, int nd) {
    if (!B.sparse) { st.ncomp = 0xFF; return; }
    uint32_t e[kTileMax + kMaxDirs];
    uint8_t pv[kTileMax + kMaxDirs];
    int ne = 0;
    auto reduce_add = [&](uint32_t x) {
        for (int i = 0; i < ne; ++i)
            if ((x >> pv[i]) & 1u) x ^= e[i];
        if (!x) return false;
        e[ne] = x; pv[ne] = (uint8_t)low_bit(x); ++ne;
        return true;
    };
    for (int i = 0; i < nd; ++i) reduce_add(dirs[i]);
    int nc = 0;
    for (uint32_t i = 0; i < B.sdim; ++i)
        if (reduce_add(B.sech[i])) st.comp[nc++] = (uint16_t)e[ne - 1];
    st.ncomp = (uint8_t)nc;
}

// Returns the step S[B.nsteps] with tables for the factors of mask. If they need more than
// kMaxTabs tables, DIAG steps apply the overflow to the tile first (those factors leave the
// pending list). With remove, the factors of the returned step leave the pending list too.
PTSBE_HD Step& take_tables(Builder& B, const DevStage& stg, Step* S, Factor* pool, uint64_t mask, bool remove) {
    while (true) {
        Step& st = S[B.nsteps];
        const uint64_t used = fill_tables(B, stg, st, pool, mask);
        if (used == mask) {
            if (remove) drop_pending(B, used, 0);
            return st;
        }
        st.kind = ST_DIAG;
        set_enumeration(B, st, nullptr, 0);
        ++B.nsteps;
        mask = drop_pending(B, used, mask & ~used);
    }
}

PTSBE_HD uint64_t all_pending(const Builder& B) { return B.npend >= 64 ? ~0ull : ((1ull << B.npend) - 1ull); }

// Adds the factor g[2 <r1,x> + <r2,x>], merging it with a pending factor on the same rows.
PTSBE_HD void push_factor(Builder& B, const DevStage& stg, Step* S, Factor* pool, uint32_t r1, uint32_t r2,
                          const float2* gin) {
    float2 g[4] = {gin[0], gin[1], gin[2], gin[3]};
    if (r1 == 0 && r2 != 0) { r1 = r2; r2 = 0; const float2 t = g[1]; g[1] = g[2]; g[2] = t; }
    if (r2 != 0 && r1 > r2) {
        const uint32_t t = r1; r1 = r2; r2 = t;
        const float2 h = g[1]; g[1] = g[2]; g[2] = h;
    }
    if (r2 == 0) { g[1] = g[0]; g[3] = g[2]; }
    if (r1 == 0) { g[1] = g[2] = g[3] = g[0]; }
    if (is_one(g[0]) && is_one(g[1]) && is_one(g[2]) && is_one(g[3])) return;
    ++B.npush;
    // at most one pending factor has these rows; four compared per iteration (independent loads)
    uint32_t hit = B.npend;
    uint32_t j = 0;
    for (; j + 4 <= B.npend && hit == B.npend; j += 4) {
        const bool h0 = B.pend[j].r1 == r1 && B.pend[j].r2 == r2;
        const bool h1 = B.pend[j + 1].r1 == r1 && B.pend[j + 1].r2 == r2;
        const bool h2 = B.pend[j + 2].r1 == r1 && B.pend[j + 2].r2 == r2;
        const bool h3 = B.pend[j + 3].r1 == r1 && B.pend[j + 3].r2 == r2;
        if (h0 | h1 | h2 | h3) hit = j + (h0 ? 0u : h1 ? 1u : h2 ? 2u : 3u);
    }
    for (; j < B.npend && hit == B.npend; ++j)
        if (B.pend[j].r1 == r1 && B.pend[j].r2 == r2) hit = j;
    if (hit < B.npend) {
        Factor& f = B.pend[hit];
        for (int x = 0; x < 4; ++x) f.f[x] = fmul(f.f[x], g[x]);
        return;
    }
    if (B.npend == kMaxPending) {
        Step& st = take_tables(B, stg, S, pool, all_pending(B), true);
        st.kind = ST_DIAG;
        set_enumeration(B, st, nullptr, 0);
        ++B.nsteps;
    }
    Factor& f = B.pend[B.npend++];
    f.r1 = r1; f.r2 = r2; f.r1o = f.r2o = 0; f.c1 = f.c2 = 0; f.pad = 0;
    for (int x = 0; x < 4; ++x) f.f[x] = g[x];
}

// diag(d0, d1) on logical bit q
PTSBE_HD void factor1(Builder& B, const DevStage& stg, Step* S, Factor* pool, int q, float2 d0, float2 d1) {
    const uint32_t r = B.row[q], c = par(r & B.bv);
    const float2 g[4] = {c ? d1 : d0, c ? d1 : d0, c ? d0 : d1, c ? d0 : d1};
    push_factor(B, stg, S, pool, r, 0, g);
}

// diagonal d[2 l_a + l_b] on logical bits (a, b)
PTSBE_HD void factor2(Builder& B, const DevStage& stg, Step* S, Factor* pool, int a, int b, const float2* d) {
    const uint32_t ra = B.row[a], rb = B.row[b];
    const uint32_t x = 2u * par(ra & B.bv) + par(rb & B.bv);
    const float2 g[4] = {d[0 ^ x], d[1 ^ x], d[2 ^ x], d[3 ^ x]};
    push_factor(B, stg, S, pool, ra, rb, g);
}

PTSBE_HD uint64_t varying(const Builder& B, uint32_t u, uint32_t v) {
    uint64_t m = 0;
    for (uint32_t j = 0; j < B.npend; ++j) {
        const Factor& f = B.pend[j];
        if (par(f.r1 & u) | par(f.r2 & u) | par(f.r1 & v) | par(f.r2 & v)) m |= 1ull << j;
    }
    return m;
}

// Pivot bits of the coset enumeration of independent directions (reduced echelon form: each
// direction contributes a distinct lowest bit; representatives have those bits clear).
PTSBE_HD void set_pivots(Step& st) {
    uint32_t ech[kMaxDirs];
    uint8_t pv[kMaxDirs];
    for (int i = 0; i < st.ndir; ++i) {
        uint32_t x = st.dir[i];
        for (int j = 0; j < i; ++j)
            if ((x >> pv[j]) & 1u) x ^= ech[j];
        ech[i] = x;
        pv[i] = (uint8_t)low_bit(x);
    }
    for (int i = 0; i < st.ndir; ++i) {   // ascending
        uint8_t b = pv[i];
        int j = i;
        while (j > 0 && st.piv[j - 1] > b) { st.piv[j] = st.piv[j - 1]; --j; }
        st.piv[j] = b;
    }
}

// Single-row factors that vary along u are folded into the mix of direction u: within a coset of
// the pass they only depend on the coordinate along u, so they scale the 2x2's columns by values
// computed once per coset. They go to the pool as [fb, fe) with c1 = tile part of the row.
PTSBE_HD uint64_t fold_factors(Builder& B, const DevStage& stg, Factor* pool, uint64_t var, uint16_t& fb, uint16_t& fe) {
    fb = (uint16_t)B.npool;
    uint64_t folded = 0;
    B.freal = 1;
    for (uint32_t j = 0; j < B.npend; ++j) {
        if (!((var >> j) & 1u) || B.pend[j].r2 != 0) continue;
        if (B.pend[j].f[0].y != 0.f || B.pend[j].f[2].y != 0.f) B.freal = 0;
        Factor& g = pool[B.npool++];
        g = B.pend[j];
        g.c1 = (uint16_t)tile_part(stg, g.r1);
        g.c2 = 0;
        g.r1o = outer_part(stg, g.r1);
        g.r2o = 0;
        folded |= 1ull << j;
    }
    fe = (uint16_t)B.npool;
    return folded;
}

// The 2x2 m and the factors folded into it (freal, from the builder) are real.
PTSBE_HD bool real_mix(const float2* m, uint32_t freal) {
    return m[0].y == 0.f && m[1].y == 0.f && m[2].y == 0.f && m[3].y == 0.f && freal;
}

PTSBE_HD void emit_mix1(Builder& B, const DevStage& stg, Step* S, Factor* pool, int q, const float2* m) {
    const uint32_t u = B.col[q];
    const uint32_t n0 = B.nsteps;
    uint64_t var = varying(B, u, 0);
    uint16_t fb, fe;
    const uint64_t folded = fold_factors(B, stg, pool, var, fb, fe);
    var = drop_pending(B, folded, var & ~folded);
    Step& st = take_tables(B, stg, S, pool, var, true);
    const uint32_t ut = tile_part(stg, u);
    // Join the previous single-qubit pass when nothing changed the factors or the frame since it
    // (its factors commute with the earlier mixes: they were pending and constant along them), and
    // no factor folded into its mixes varies along the new direction.
    if (B.nsteps == n0 && n0 > 0) {
        Step& pr = S[n0 - 1];
        bool ok = pr.kind == ST_MIX1 && pr.ndir < kMaxDirs && pr.npush == B.npush && pr.nframe == B.nframe &&
                  pr.ntab + st.ntab <= kMaxTabs;
        for (int i = 0; ok && i < pr.ndir; ++i) {
            ok = par(pr.rin[i] & ut) == 0;
            for (uint32_t j = pr.fold_b[i]; ok && j < pr.fold_e[i]; ++j) ok = par(pool[j].r1 & u) == 0;
        }
        if (ok) {
            for (int t = 0; t < st.ntab; ++t) pr.tab[pr.ntab + t] = st.tab[t];
            pr.ntab = (uint8_t)(pr.ntab + st.ntab);
            const int i = pr.ndir++;
            pr.fold_b[i] = fb;
            pr.fold_e[i] = fe;
            if (real_mix(m, B.freal)) pr.mreal |= (uint8_t)(1u << i);
            pr.dir[i] = (uint16_t)ut;
            pr.rin[i] = (uint16_t)tile_part(stg, B.row[q]);
            pr.rout[i] = outer_part(stg, B.row[q]);
            pr.cpar[i] = (uint8_t)par(B.row[q] & B.bv);
            for (int k = 0; k < 4; ++k) pr.m[4 * i + k] = m[k];
            set_pivots(pr);
            if (B.sparse) support_add(B, ut);
            set_enumeration(B, pr, pr.dir, pr.ndir);
            return;
        }
    }
    st.kind = ST_MIX1;
    st.ndir = 1;
    st.mreal = real_mix(m, B.freal) ? 1 : 0;
    st.fold_b[0] = fb;
    st.fold_e[0] = fe;
    st.dir[0] = (uint16_t)ut;
    st.rin[0] = (uint16_t)tile_part(stg, B.row[q]);
    st.rout[0] = outer_part(stg, B.row[q]);
    st.cpar[0] = (uint8_t)par(B.row[q] & B.bv);
    st.npush = B.npush;
    st.nframe = B.nframe;
    for (int k = 0; k < 4; ++k) st.m[k] = m[k];
    set_pivots(st);
    if (B.sparse) support_add(B, ut);
    set_enumeration(B, st, st.dir, 1);
    ++B.nsteps;
}

PTSBE_HD void emit_mix2(Builder& B, const DevStage& stg, Step* S, Factor* pool, int a, int b, const float2* m) {
    Step& st = take_tables(B, stg, S, pool, varying(B, B.col[a], B.col[b]), true);
    const uint32_t u = tile_part(stg, B.col[a]), v = tile_part(stg, B.col[b]);
    st.kind = ST_MIX2;
    st.ndir = 2;
    st.mreal = 0;
    for (int i = 0; i < kMaxDirs; ++i) st.fold_b[i] = st.fold_e[i] = 0;
    st.dir[0] = (uint16_t)u;
    st.dir[1] = (uint16_t)v;
    const int pa = low_bit(u);
    const uint32_t v2 = ((v >> pa) & 1u) ? (v ^ u) : v;
    st.piv[0] = (uint8_t)pa;
    st.piv[1] = (uint8_t)low_bit(v2);
    st.rin[0] = (uint16_t)tile_part(stg, B.row[a]);
    st.rin[1] = (uint16_t)tile_part(stg, B.row[b]);
    st.rout[0] = outer_part(stg, B.row[a]);
    st.rout[1] = outer_part(stg, B.row[b]);
    st.cpar[0] = (uint8_t)par(B.row[a] & B.bv);
    st.cpar[1] = (uint8_t)par(B.row[b] & B.bv);
    st.npush = B.npush;
    st.nframe = B.nframe;
    for (int i = 0; i < 16; ++i) st.m[i] = m[i];
    if (B.sparse) { support_add(B, u); support_add(B, v); }
    set_enumeration(B, st, st.dir, 2);
    ++B.nsteps;
}

// End of the stage: STORE writes D(x) s[x] to global index x ^ b; FINAL writes logical order.
PTSBE_HD void emit_end(Builder& B, const DevStage& stg, Step* S, Factor* pool, int n) {
    Step& st = take_tables(B, stg, S, pool, all_pending(B), false);
    if (B.sparse_final && B.sparse) set_enumeration(B, st, nullptr, 0);   // the support, for the scatter
    else st.ncomp = 0xFF;
    if (B.last) {
        st.kind = ST_FINAL;
        uint32_t l = 0;
        for (int q = 0; q < n; ++q) l |= par(B.row[q] & B.bv) << q;
        st.lb0 = l;
    } else {
        st.kind = ST_STORE;
        st.lb0 = tile_part(stg, B.bv);
        st.rout[0] = outer_part(stg, B.bv);
    }
    ++B.nsteps;
}

// out[x] = d[x] * in[perm_x] on x = 2 l_a + l_b as a frame change (perm is a bijection).
PTSBE_HD void perm2(Builder& B, int a, int b, const uint32_t* pm) {
    ++B.nframe;
    const uint32_t t = pm[0], c1 = pm[1] ^ t, c2 = pm[2] ^ t;   // images of e_b and e_a
    const uint32_t ca = B.col[a], cb = B.col[b], ra = B.row[a], rb = B.row[b];
    B.bv ^= ((t >> 1) ? ca : 0u) ^ ((t & 1u) ? cb : 0u);
    B.col[a] = ((c2 >> 1) ? ca : 0u) ^ ((c2 & 1u) ? cb : 0u);
    B.col[b] = ((c1 >> 1) ? ca : 0u) ^ ((c1 & 1u) ? cb : 0u);
    B.row[a] = ((c1 & 1u) ? ra : 0u) ^ ((c1 >> 1) ? rb : 0u);
    B.row[b] = ((c2 & 1u) ? ra : 0u) ^ ((c2 >> 1) ? rb : 0u);
}

// One operator on logical qubits (a, b).
PTSBE_HD void process(Builder& B, const DevStage& stg, Step* S, Factor* pool, uint8_t kind, int a, int b,
                      const float2* m, uint32_t perm, bool sep) {
    switch (kind) {
    case DOP_G1: emit_mix1(B, stg, S, pool, a, m); break;
    case DOP_D1: factor1(B, stg, S, pool, a, m[0], m[1]); break;
    case DOP_X1:   // [[0, m0], [m1, 0]]: psi'(l) = d[l_a] psi(l ^ e_a), d = (m0, m1)
        ++B.nframe;
        B.bv ^= B.col[a];
        factor1(B, stg, S, pool, a, m[0], m[1]);
        break;
    case DOP_CX:
        ++B.nframe;
        B.col[a] ^= B.col[b];
        B.row[b] ^= B.row[a];
        break;
    case DOP_CZ: {
        const float2 d[4] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f), make_float2(1.f, 0.f), make_float2(-1.f, 0.f)};
        factor2(B, stg, S, pool, a, b, d);
        break;
    }
    case DOP_SWAP: {
        ++B.nframe;
        uint32_t t = B.col[a]; B.col[a] = B.col[b]; B.col[b] = t;
        t = B.row[a]; B.row[a] = B.row[b]; B.row[b] = t;
        break;
    }
    case DOP_G2: emit_mix2(B, stg, S, pool, a, b, m); break;
    case DOP_M2: {
        const uint32_t pm[4] = {perm & 3u, (perm >> 2) & 3u, (perm >> 4) & 3u, (perm >> 6) & 3u};
        if (((1u << pm[0]) | (1u << pm[1]) | (1u << pm[2]) | (1u << pm[3])) != 15u) {
            float2 g[16];
            for (int i = 0; i < 16; ++i) g[i] = make_float2(0.f, 0.f);
            for (int x = 0; x < 4; ++x) g[4 * x + pm[x]] = m[x];
            emit_mix2(B, stg, S, pool, a, b, g);
            break;
        }
        perm2(B, a, b, pm);
        if (sep) {
            factor1(B, stg, S, pool, a, m[4], m[5]);
            factor1(B, stg, S, pool, b, m[6], m[7]);
        } else {
            factor2(B, stg, S, pool, a, b, m);
        }
        break;
    }
    default: break;   // DOP_NOP
    }
}

PTSBE_HD bool perm_is_bijection(uint32_t perm) {
    uint32_t seen = 0;
    for (int x = 0; x < 4; ++x) seen |= 1u << ((perm >> (2 * x)) & 3u);
    return seen == 15u;
}

// 4x4 matrix of a fused two-qubit block (general, or monomial d[x] at column perm_x).
PTSBE_HD void fused_matrix(const DevOp& o, const float2* m, float2* g) {
    if (o.fkind == DOP_G2) {
        for (int i = 0; i < 16; ++i) g[i] = m[i];
        return;
    }
    for (int i = 0; i < 16; ++i) g[i] = make_float2(0.f, 0.f);
    for (int x = 0; x < 4; ++x) g[4 * x + ((o.fperm >> (2 * x)) & 3u)] = m[x];
}

PTSBE_HD_CALL void builder_init(Builder& B, const EvolveArgs& a, const DevStage& st, const DevFrameStage& fs,
                                uint32_t node, bool from_zero) {
    for (int q = 0; q < kMaxQubits; ++q) { B.col[q] = fs.col[q]; B.row[q] = fs.row[q]; }
    B.bv = 0;
    B.op = st.op_begin;
    uint32_t e = a.node_ebeg[node];
    B.ee = a.node_eend[node];
    while (e < B.ee && a.site_op[a.ent_site[e]] < st.op_begin) ++e;
    B.e = e;
    B.npend = 0;
    B.done = 0;
    B.last = fs.last;
    B.npush = B.nframe = 0;
    B.sparse = from_zero ? 1u : 0u;      // the support starts as {0}
    B.sdim = 0;
    B.sparse_final = fs.sparse_final;
    // A sparse final stage with a support bound keeps every nonzero amplitude below tile address
    // 2^sbits: parities against the other tile bits never matter, so table rows drop them (at most
    // sbits index bits per table).
    const bool small = fs.sparse_final && fs.sbits > 0;
    B.tmask = small ? (1u << fs.sbits) - 1u : 0xFFFFFFFFu;
    B.tsb = (uint8_t)(small ? fs.sbits : kTabBits);
}

// Emits steps until the stage ends (then the end step and done = 1) or the step list or the
// factor pool could overflow with one more op (the next segment continues from B.op).
PTSBE_HD_CALL void build_segment(Builder& B, Step* S, Factor* pool, const EvolveArgs& a, const DevStage& st,
                                 uint32_t max_steps, uint32_t max_pool) {
    B.nsteps = 0;
    B.npool = 0;
    while (true) {
        if (B.nsteps + kStepsPerOp > max_steps || B.npool + kPoolPerOp > max_pool) return;
        if (B.op >= st.op_end) {
            emit_end(B, st, S, pool, a.n);
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
                process(B, st, S, pool, mi.kind, mi.operand == 1 ? o.q1 : o.q0, o.q1, a.mats + mi.mat, 0, false);
            }
            B.op = op + 1;
        } else if (o.fend != 0 && (B.e >= B.ee || a.ent_site[B.e] >= o.fsite1)) {
            // no error inside the fused block: gate and no-error operators at once
            const bool mixes = o.fkind == DOP_G2 || (o.fkind == DOP_M2 && !perm_is_bijection(o.fperm));
            if (mixes && (o.kind == DOP_CX || o.kind == DOP_SWAP)) {
                // The block M is not monomial, but the gate's permutation P must still move the
                // frame (the unfused path moves it too): P first, then M P^-1 mixes.
                const uint32_t pm[4] = {0u, o.kind == DOP_CX ? 1u : 2u, o.kind == DOP_CX ? 3u : 1u, o.kind == DOP_CX ? 2u : 3u};
                float2 g[16], h[16];
                fused_matrix(o, a.mats + o.fmat, g);
                for (int r = 0; r < 4; ++r)
                    for (int y = 0; y < 4; ++y) h[4 * r + y] = g[4 * r + pm[y]];
                perm2(B, o.q0, o.q1, pm);
                emit_mix2(B, st, S, pool, o.q0, o.q1, h);
            } else {
                process(B, st, S, pool, o.fkind, o.q0, o.q1, a.mats + o.fmat, o.fperm, o.fsep != 0);
            }
            B.op = o.fend;
        } else {
            process(B, st, S, pool, o.kind, o.q0, o.q1, a.mats + o.mat, 0, false);
            B.op = op + 1;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Steps (every thread of the CTA; thread `tid` of `nthr`, tile index `tau`)
// ------------------------------------------------------------------------------------------

PTSBE_HD uint32_t lin_idx(const Table& T, uint32_t p) {
    uint32_t r = 0;
    for (int i = 0; i < T.d; ++i) r |= par(T.basis[i] & p) << i;
    return r;
}

PTSBE_HD int log2u(uint32_t x) {
    int lg = 0;
    while ((1u << lg) < x) ++lg;
    return lg;
}

PTSBE_HD uint32_t ins_piv(uint32_t i, const uint8_t* piv, int k) {   // zeros at ascending pivots
    for (int j = 0; j < k; ++j) i = ins0(i, piv[j]);
    return i;
}

// Enumeration of a pass: coset index i -> representative. Whole tile: zeros inserted at the pivot
// bits of the step's directions; sparse: XOR of comp[j] over the set bits j of i.
PTSBE_HD uint32_t enum_count(const Step& st, int tb, int nd) { return st.ncomp == 0xFF ? 1u << (tb - nd) : 1u << st.ncomp; }
PTSBE_HD uint32_t enum_base(const Step& st, uint32_t i, const uint8_t* piv, int nd) {
    if (st.ncomp == 0xFF) return ins_piv(i, piv, nd);
    uint32_t b = 0;
    for (int j = 0; j < st.ncomp && (i >> j); ++j)
        if ((i >> j) & 1u) b ^= st.comp[j];
    return b;
}

// Tile-local address delta of bit j of the iteration counter (slots < 10), of the directions of
// a grouped mix (slots 10 + i), and of the fixed offsets of the other steps (slots 14, 15).
PTSBE_HD uint32_t step_delta(const Step& st, const DevFrameStage& fs, int tb, uint32_t nthr, int j) {
    const uint32_t mask = (1u << tb) - 1u;
    switch (st.kind) {
    case ST_MIX1:
        if (j >= 10) return j - 10 < st.ndir ? st.dir[j - 10] : 0u;
        if (st.ncomp != 0xFF) return enum_base(st, nthr << j, st.piv, st.ndir);
        return ins_piv(nthr << j, st.piv, st.ndir) & mask;
    case ST_MIX2:
        if (j == 14) return st.dir[1];
        if (j == 15) return st.dir[0];
        if (st.ncomp != 0xFF) return j < 14 ? enum_base(st, nthr << j, st.piv, 2) : 0u;
        return j < 14 ? ins00(nthr << j, st.piv[0], st.piv[1]) & mask : 0u;
    case ST_DIAG:
        if (st.ncomp != 0xFF) return j < 14 ? enum_base(st, nthr << j, st.piv, 0) : 0u;
        return j < 14 ? (nthr << j) & mask : 0u;
    case ST_STORE:   // destination d = 2 (tid + k nthr) + {0, 1}, source d ^ b
        if (j == 15) return 1u;
        return j < 14 ? ((2u * nthr) << j) & mask : 0u;
    default: {       // FINAL: tile-local address M t, t = 2 (tid + k nthr) + {0, 1}
        if (j == 15) return fs.m[0];
        const int bit = 1 + log2u(nthr) + j;
        return (j < 14 && bit < tb) ? fs.m[bit] : 0u;
    }
    }
}

// Table entries and index deltas of a step (before the pass; a barrier separates them).
PTSBE_HD void prepare_tables(const Step& st, const DevFrameStage& fs, const Factor* pool, float2* tabs, uint32_t* delta,
                             int tb, uint32_t tau, uint32_t tid, uint32_t nthr) {
    for (int t = 0; t < st.ntab; ++t) {
        const Table& T = st.tab[t];
        const uint32_t size = 1u << T.d;
        for (uint32_t idx = tid; idx < size; idx += nthr) {
            if (T.real) {
                float v = 1.f;
                for (uint32_t j = T.fb; j < T.fe; ++j) {
                    const Factor& f = pool[j];
                    v *= f.f[2u * (par(f.c1 & idx) ^ par(f.r1o & tau)) + (par(f.c2 & idx) ^ par(f.r2o & tau))].x;
                }
                tabs[((uint32_t)t << st.tsb) + idx] = make_float2(v, 0.f);
            } else {
                float2 v = make_float2(1.f, 0.f);
                for (uint32_t j = T.fb; j < T.fe; ++j) {
                    const Factor& f = pool[j];
                    v = fmul(v, f.f[2u * (par(f.c1 & idx) ^ par(f.r1o & tau)) + (par(f.c2 & idx) ^ par(f.r2o & tau))]);
                }
                tabs[((uint32_t)t << st.tsb) + idx] = v;
            }
        }
    }
    const uint32_t nd = (uint32_t)st.ntab * kDeltaSlots;
    for (uint32_t i = tid; i < nd; i += nthr)
        delta[i] = lin_idx(st.tab[i / kDeltaSlots], step_delta(st, fs, tb, nthr, (int)(i % kDeltaSlots)));
}

struct Lookup {
    int ntab, real;                  // real bit t: table t holds real values
    uint32_t ix[kMaxTabs];           // entry in the table buffer (table base t << tsb | index)
};

PTSBE_HD float2 apply_tabs(float2 x, const Lookup& L, const float2* tabs, const uint32_t* delta, int slot) {
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t)
        if (t < L.ntab) {
            const uint32_t i = slot < 0 ? L.ix[t] : (L.ix[t] ^ delta[t * kDeltaSlots + slot]);
            if ((L.real >> t) & 1) {
                x = mul2r(x, reinterpret_cast<const float*>(tabs + i)[0]);
            } else {
                x = fmul(x, tabs[i]);
            }
        }
    return x;
}

PTSBE_HD void lookup_init(Lookup& L, const Step& st, uint32_t p) {
    L.ntab = st.ntab;
    L.real = 0;
    for (int t = 0; t < st.ntab; ++t) L.real |= st.tab[t].real << t;
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t) L.ix[t] = t < L.ntab ? (((uint32_t)t << st.tsb) | lin_idx(st.tab[t], p)) : 0u;
}
PTSBE_HD void lookup_step(Lookup& L, const uint32_t* delta, int j) {
#pragma unroll
    for (int t = 0; t < kMaxTabs; ++t)
        if (t < L.ntab) L.ix[t] ^= delta[t * kDeltaSlots + j];
}

// The iterations of a thread visit k = 0 .. K-1 in Gray-code order, so each step flips one bit
// of the address and of every table index.
//
// Grouped single-qubit mixes: the thread holds the 2^ND amplitudes base ^ sum_i y_i dir[i] of one
// coset of the directions. The logical bit of operand i there is <rin[i], base> ^ cpar[i] ^ y_i
// (rows and columns of one frame), so each 2x2 acts on register pairs y, y | 1 << i with one
// orientation per coset.
template <int ND>
PTSBE_HD void run_mix1_n(const Step& st, const Factor* pool, float2* s, const float2* tabs, const uint32_t* delta, int tb,
                         uint32_t tau, uint32_t tid, uint32_t nthr) {
    constexpr int NA = 1 << ND;
    const uint32_t N = enum_count(st, tb, ND);
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    uint32_t dir[ND], rin[ND], c0[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) { dir[i] = st.dir[i]; rin[i] = st.rin[i]; c0[i] = st.cpar[i] ^ par(st.rout[i] & tau); }
    uint32_t base = enum_base(st, tid, st.piv, ND);
    Lookup L;
    lookup_init(L, st, base);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            base ^= enum_base(st, nthr << j, st.piv, ND);
            lookup_step(L, delta, j);
        }
        float2 v[NA];
#pragma unroll
        for (int y = 0; y < NA; ++y) {
            uint32_t off = 0;
#pragma unroll
            for (int i = 0; i < ND; ++i) if ((y >> i) & 1) off ^= dir[i];
            v[y] = s[base ^ off];
        }
        if (L.ntab) {
#pragma unroll
            for (int y = 0; y < NA; ++y) {
                Lookup Ly = L;
#pragma unroll
                for (int i = 0; i < ND; ++i) if ((y >> i) & 1) lookup_step(Ly, delta, 10 + i);
                v[y] = apply_tabs(v[y], Ly, tabs, delta, -1);
            }
        }
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            const bool fl = (par(rin[i] & base) ^ c0[i]) != 0;
            const float2 a00 = st.m[4 * i], a01 = st.m[4 * i + 1], a10 = st.m[4 * i + 2], a11 = st.m[4 * i + 3];
            float2 g00 = fl ? a11 : a00, g01 = fl ? a10 : a01, g10 = fl ? a01 : a10, g11 = fl ? a00 : a11;
            // folded factors: F0 on the half with y_i = 0, F1 on y_i = 1 (the matrix's columns)
            const uint32_t fb = st.fold_b[i], fe = st.fold_e[i];
            const bool real = (st.mreal >> i) & 1;
            if (fb < fe) {
                if (real) {
                    float F0 = 1.f, F1 = 1.f;
                    for (uint32_t j = fb; j < fe; ++j) {
                        const Factor& f = pool[j];
                        const uint32_t c = par(f.c1 & base) ^ par(f.r1o & tau);
                        F0 *= f.f[2u * c].x;
                        F1 *= f.f[2u * (c ^ 1u)].x;
                    }
                    g00.x *= F0; g10.x *= F0;
                    g01.x *= F1; g11.x *= F1;
                } else {
                    float2 F0 = make_float2(1.f, 0.f), F1 = make_float2(1.f, 0.f);
                    for (uint32_t j = fb; j < fe; ++j) {
                        const Factor& f = pool[j];
                        const uint32_t c = par(f.c1 & base) ^ par(f.r1o & tau);
                        F0 = fmul(F0, f.f[2u * c]);
                        F1 = fmul(F1, f.f[2u * (c ^ 1u)]);
                    }
                    g00 = fmul(g00, F0); g10 = fmul(g10, F0);
                    g01 = fmul(g01, F1); g11 = fmul(g11, F1);
                }
            }
            if (real) {
#pragma unroll
                for (int y = 0; y < NA; ++y) {
                    if ((y >> i) & 1) continue;
                    const float2 a = v[y], b = v[y | (1 << i)];
                    v[y] = fma2r(b, g01.x, mul2r(a, g00.x));
                    v[y | (1 << i)] = fma2r(b, g11.x, mul2r(a, g10.x));
                }
            } else {
#pragma unroll
                for (int y = 0; y < NA; ++y) {
                    if ((y >> i) & 1) continue;
                    const float2 a = v[y], b = v[y | (1 << i)];
                    v[y] = fmul2(g00, a, g01, b);
                    v[y | (1 << i)] = fmul2(g10, a, g11, b);
                }
            }
        }
#pragma unroll
        for (int y = 0; y < NA; ++y) {
            uint32_t off = 0;
#pragma unroll
            for (int i = 0; i < ND; ++i) if ((y >> i) & 1) off ^= dir[i];
            s[base ^ off] = v[y];
        }
    }
}

PTSBE_HD void run_mix1(const Step& st, const Factor* pool, float2* s, const float2* tabs, const uint32_t* delta, int tb,
                       uint32_t tau, uint32_t tid, uint32_t nthr) {
    static_assert(kMaxDirs == 4, "one instantiation per group size");
    switch (st.ndir) {
    case 1: run_mix1_n<1>(st, pool, s, tabs, delta, tb, tau, tid, nthr); break;
    case 2: run_mix1_n<2>(st, pool, s, tabs, delta, tb, tau, tid, nthr); break;
    case 3: run_mix1_n<3>(st, pool, s, tabs, delta, tb, tau, tid, nthr); break;
    default: run_mix1_n<4>(st, pool, s, tabs, delta, tb, tau, tid, nthr); break;
    }
}

PTSBE_HD void xswap(float2* z, uint32_t x0) {
    if (x0 & 1u) { float2 t = z[0]; z[0] = z[1]; z[1] = t; t = z[2]; z[2] = z[3]; z[3] = t; }
    if (x0 & 2u) { float2 t = z[0]; z[0] = z[2]; z[2] = t; t = z[1]; z[1] = z[3]; z[3] = t; }
}

PTSBE_HD void run_mix2(const Step& st, float2* s, const float2* tabs, const uint32_t* delta, int tb, uint32_t tau,
                       uint32_t tid, uint32_t nthr) {
    const uint32_t N = enum_count(st, tb, 2);
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    const uint32_t w[4] = {0u, st.dir[1], st.dir[0], (uint32_t)(st.dir[0] ^ st.dir[1])};   // logical difference y -> offset
    const uint32_t ca = st.cpar[0] ^ par(st.rout[0] & tau), cb = st.cpar[1] ^ par(st.rout[1] & tau);
    const uint8_t pv2[2] = {(uint8_t)(st.piv[0] < st.piv[1] ? st.piv[0] : st.piv[1]), (uint8_t)(st.piv[0] < st.piv[1] ? st.piv[1] : st.piv[0])};
    uint32_t base = enum_base(st, tid, pv2, 2);
    Lookup L;
    lookup_init(L, st, base);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            base ^= enum_base(st, nthr << j, pv2, 2);
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
        const uint32_t x0 = 2u * (par(st.rin[0] & base) ^ ca) + (par(st.rin[1] & base) ^ cb);
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
    const uint32_t N = enum_count(st, tb, 0);
    if (tid >= N) return;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    uint32_t p = enum_base(st, tid, nullptr, 0);
    Lookup L;
    lookup_init(L, st, p);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            p ^= enum_base(st, nthr << j, nullptr, 0);
            lookup_step(L, delta, j);
        }
        s[p] = apply_tabs(s[p], L, tabs, delta, -1);
    }
}

PTSBE_HD uint64_t gaddr(uint32_t l, int lb, const uint32_t* hi, uint64_t outer) {
    return (uint64_t)(l & ((1u << lb) - 1u)) | (uint64_t)hi[l >> lb] | outer;
}

PTSBE_HD uint64_t outer_offset(const DevStage& stg, int ob, uint32_t tau) {
    uint64_t o = 0;
    for (int b = 0; b < ob; ++b)
        if ((tau >> b) & 1u) o |= 1ull << stg.outer_q[b];
    return o;
}

// Intermediate store: tile-local d of tile tau ^ b_out receives D(x) s[d ^ b_in] (x the source).
// Returns this thread's part of the squared norm of what it wrote. zero: the tile is known to be
// zero (its amplitudes are not read).
PTSBE_HD double run_store(const Step& st, const DevStage& stg, const float2* s, const float2* tabs, const uint32_t* delta,
                          int tb, int lb, int ob, const uint32_t* hi, uint32_t tau, float2* dst, uint32_t tid, uint32_t nthr,
                          bool zero = false) {
    const uint32_t N = 1u << (tb - 1);
    if (tid >= N) return 0.0;
    float part = 0.f;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    const uint32_t bin = st.lb0;
    const uint64_t outer = outer_offset(stg, ob, tau ^ st.rout[0]);
    uint32_t d = 2u * tid;
    if (zero) {
        for (uint32_t k = 0; k < K; ++k, d += 2u * nthr)
            *reinterpret_cast<float4*>(dst + gaddr(d, lb, hi, outer)) = make_float4(0.f, 0.f, 0.f, 0.f);
        return 0.0;
    }
    Lookup L;
    lookup_init(L, st, d ^ bin);
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            d ^= (2u * nthr) << j;
            lookup_step(L, delta, j);
        }
        float2 a0 = s[d ^ bin], a1 = s[(d ^ bin) ^ 1u];
        if (L.ntab) { a0 = apply_tabs(a0, L, tabs, delta, -1); a1 = apply_tabs(a1, L, tabs, delta, 15); }
        part += fmaf(a0.x, a0.x, a0.y * a0.y) + fmaf(a1.x, a1.x, a1.y * a1.y);
        *reinterpret_cast<float4*>(dst + gaddr(d, lb, hi, outer)) = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
    return (double)part;
}

// Last stage: writes the logical amplitudes of this tile, times `scale`, to dst (when not null) and
// returns this thread's part of their squared norm (when want_norm).
PTSBE_HD double run_final(const Step& st, const DevFrameStage& fs, const float2* s, const float2* tabs,
                          const uint32_t* delta, int tb, int ob, uint32_t tau, float2* dst, float scale, bool want_norm,
                          uint32_t tid, uint32_t nthr, bool zero = false) {
    const uint32_t N = 1u << (tb - 1);
    if (tid >= N) return 0.0;
    const uint32_t K = N > nthr ? N / nthr : 1u;
    const int lg = log2u(nthr);
    uint32_t p = 0, l = st.lb0;
    for (int i = 0; i < ob; ++i)
        if ((tau >> i) & 1u) l ^= fs.ox[i];
    for (int b = 0; (1u << b) <= tid; ++b)
        if ((tid >> b) & 1u) { p ^= fs.m[b + 1]; l ^= fs.w[b + 1]; }
    Lookup L;
    lookup_init(L, st, p);
    float part = 0.f;
    for (uint32_t k = 0; k < K; ++k) {
        if (k) {
            const int j = low_bit(k);
            p ^= fs.m[1 + lg + j];
            l ^= fs.w[1 + lg + j];
            lookup_step(L, delta, j);
        }
        float2 a0 = make_float2(0.f, 0.f), a1 = a0;
        if (!zero) {
            a0 = s[p];
            a1 = s[p ^ fs.m[0]];
            if (L.ntab) { a0 = apply_tabs(a0, L, tabs, delta, -1); a1 = apply_tabs(a1, L, tabs, delta, 15); }
        }
        if (want_norm) part += fmaf(a0.x, a0.x, a0.y * a0.y) + fmaf(a1.x, a1.x, a1.y * a1.y);
        if (dst) {
            // w[0] = e_0: the pair is {l, l ^ 1}
            const float2 s0 = mul2r(a0, scale), s1 = mul2r(a1, scale);
            const float4 x = (l & 1u) ? make_float4(s1.x, s1.y, s0.x, s0.y) : make_float4(s0.x, s0.y, s1.x, s1.y);
            *reinterpret_cast<float4*>(dst + (l & ~1u)) = x;
        }
    }
    return (double)part;
}

// Sparse final store: the support of the state (span of comp, all in this tile) holds every
// nonzero amplitude. phase 0 returns this thread's part of the squared norm; phase 1 writes
// D(x) s[x] * scale to logical index R_end x ^ R_end b of dst (the caller zero-filled dst before).
// Support entry at tile position p of the sparse final store: its amplitude (deferred factors
// applied, before the normalisation scale) and its logical index.
PTSBE_HD float2 sparse_value(const Step& st, const float2* s, const float2* tabs, const uint32_t* delta, uint32_t p) {
    float2 a = s[p];
    if (st.ntab) {
        Lookup L;
        lookup_init(L, st, p);
        a = apply_tabs(a, L, tabs, delta, -1);
    }
    return a;
}
PTSBE_HD uint32_t sparse_logical(const Step& st, const DevFrameStage& fs, int n, int lb, const uint32_t* hi, uint32_t p) {
    const uint64_t x = gaddr(p, lb, hi, 0);
    uint32_t l = st.lb0;
    for (int q = 0; q < n; ++q) l ^= par(fs.rowe[q] & (uint32_t)x) << q;
    return l;
}

PTSBE_HD double run_sparse_final(const Step& st, const DevFrameStage& fs, const float2* s, const float2* tabs,
                                 const uint32_t* delta, int n, int lb, const uint32_t* hi, float2* dst, float scale,
                                 int phase, uint32_t tid, uint32_t nthr) {
    const uint32_t N = st.ncomp == 0xFF ? 0u : 1u << st.ncomp;
    double acc = 0.0;
    for (uint32_t i = tid; i < N; i += nthr) {
        const uint32_t p = enum_base(st, i, nullptr, 0);
        const float2 a = sparse_value(st, s, tabs, delta, p);
        if (phase == 0) acc += (double)fmaf(a.x, a.x, a.y * a.y);
        else dst[sparse_logical(st, fs, n, lb, hi, p)] = mul2r(a, scale);
    }
    return acc;
}

// Order of the support in logical index. The support's logical indices form an affine subspace
// c + span(v_0 .. v_{k-1}), v_j the image of the coset generator comp[j] (the map from tile
// position to logical index is affine over GF(2)). Reduce the v_j to an echelon basis with
// distinct leading bits h_j: two members differ by a nonzero combination whose highest bit is
// some h_j, so they agree above h_j and the one with bit h_j set is larger, and the bits of a
// member at the positions h_j, read as a k-bit integer, give its rank in increasing order.
// Returns the mask of the h_j (k bits set exactly when the images are independent).
PTSBE_HD uint32_t sparse_order_mask(const Step& st, const DevFrameStage& fs, int n, int lb, const uint32_t* hi) {
    if (st.ncomp == 0xFF) return 0u;
    uint32_t basis[32];
    uint32_t lead = 0;
    const uint32_t l0 = sparse_logical(st, fs, n, lb, hi, 0u);
    for (int j = 0; j < st.ncomp; ++j) {
        uint32_t v = sparse_logical(st, fs, n, lb, hi, st.comp[j]) ^ l0;
        while (v) {
            const int h = high_bit(v);
            if (!((lead >> h) & 1u)) { basis[h] = v; lead |= 1u << h; break; }
            v ^= basis[h];
        }
    }
    return lead;
}

// Bits of x at the set positions of mask, packed from bit 0 up.
PTSBE_HD uint32_t extract_bits(uint32_t x, uint32_t mask) {
    uint32_t r = 0;
    for (int k = 0; mask; ++k) {
        const int b = low_bit(mask);
        r |= ((x >> b) & 1u) << k;
        mask &= mask - 1u;
    }
    return r;
}

}  // namespace frame
}  // namespace ptsbe
