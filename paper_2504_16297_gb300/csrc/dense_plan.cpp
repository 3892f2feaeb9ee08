// Planner of the dense tile passes (dense.cuh).
//
// The circuit (gates and noise sites in order) is cut into passes. A pass holds kT logical qubits
// -- always the kC qubits currently at physical bits 0 .. kC-1, so tiles are made of contiguous
// runs -- and applies every not yet applied operation that acts only on those qubits and whose
// predecessors on its qubits are applied. The qubit set of a pass is the best of a few candidates
// (contiguous windows of qubit indices, the qubits of the next pending operations, a greedy
// one-qubit-at-a-time growth), scored by how many operations it applies. A pass then rewrites its
// tile bits in a new order that puts, at the low physical bits, qubits the next pass will want;
// trailing passes without operations restore logical order (qubit q = bit q) at the end.
//
// Within a pass, operations become blocks: consecutive operations on one qubit, or on one pair,
// multiplied together (a gate, then the Kraus operator of each noise site after it: operator 0 by
// default, the set's operator where the set has an entry -- an "override" block). Blocks are then
// packed into register groups of kR tile bits, taking later blocks forward past ones they commute
// with (disjoint qubits).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace ptsbe {

namespace {

using namespace dense;

struct OpQ {
    uint32_t q0, q1;
    uint8_t nq;
};

uint64_t qmask(const OpQ& o) { return (1ull << o.q0) | (o.nq == 2 ? (1ull << o.q1) : 0ull); }
int pop(uint64_t m) { return __builtin_popcountll(m); }

struct PassRec {
    uint64_t S;                          // logical qubits of the tile
    std::vector<uint32_t> ops;           // operations applied, circuit order
    std::vector<int> phys_in, phys_out;  // logical -> physical before / after the pass
};

struct Planner {
    int n = 0, T = 0;
    std::vector<OpQ> ops;
    std::vector<uint8_t> done;
    size_t first = 0;
    std::vector<int> phys, at;           // logical -> physical, physical -> logical

    // A pass holds at most kMaxPass2q two-qubit operations: its blocks (at most one 1-qubit block
    // per tile qubit, plus one per two-qubit operation), groups and matrices then always fit the
    // kernel's shared-memory staging (kStageMax).
    static constexpr uint32_t kMaxPass2q = 112;

    uint32_t exec(uint64_t S, std::vector<uint32_t>* out) const {
        uint64_t blocked = 0;
        uint32_t cnt = 0, cnt2 = 0;
        for (size_t i = first; i < ops.size(); ++i) {
            if (done[i]) continue;
            const uint64_t m = qmask(ops[i]);
            if ((m & ~S) || (m & blocked) || (ops[i].nq == 2 && cnt2 >= kMaxPass2q)) {
                blocked |= m;
                if ((blocked & S) == S) break;
                continue;
            }
            ++cnt;
            cnt2 += ops[i].nq == 2;
            if (out) out->push_back((uint32_t)i);
        }
        return cnt;
    }

    uint64_t low_set() const {
        uint64_t m = 0;
        for (int p = 0; p < kC; ++p) m |= 1ull << at[p];
        return m;
    }

    uint64_t choose(uint64_t must, uint32_t* best_cnt) const {
        uint64_t best = 0;
        uint32_t bc = 0;
        bool have = false;
        auto consider = [&](uint64_t S) {
            if (pop(S) != T) return;
            const uint32_t k = exec(S, nullptr);
            if (!have || k > bc) { best = S; bc = k; have = true; }
        };
        for (int a = 0; a < n; ++a) {
            uint64_t S = must;
            for (int q = a; q < n && pop(S) < T; ++q) S |= 1ull << q;
            for (int q = a - 1; q >= 0 && pop(S) < T; --q) S |= 1ull << q;
            consider(S);
        }
        {   // the qubits of the next pending operations, in order
            uint64_t S = must;
            for (size_t i = first; i < ops.size() && pop(S) < T; ++i) {
                if (done[i]) continue;
                const uint64_t m = qmask(ops[i]);
                if (pop(S | m) <= T) S |= m;
            }
            for (int q = 0; q < n && pop(S) < T; ++q) S |= 1ull << q;
            consider(S);
        }
        {   // greedy growth
            uint64_t S = must;
            while (pop(S) < T) {
                int bq = -1;
                uint32_t bk = 0;
                for (int q = 0; q < n; ++q) {
                    if ((S >> q) & 1u) continue;
                    const uint32_t k = exec(S | (1ull << q), nullptr);
                    if (bq < 0 || k > bk) { bq = q; bk = k; }
                }
                S |= 1ull << bq;
            }
            consider(S);
        }
        *best_cnt = bc;
        return best;
    }

    // first pending operation index of every qubit (ops.size() when none)
    std::vector<size_t> next_pending() const {
        std::vector<size_t> nx(n, ops.size());
        int left = n;
        for (size_t i = first; i < ops.size() && left > 0; ++i) {
            if (done[i]) continue;
            const OpQ& o = ops[i];
            if (nx[o.q0] == ops.size()) { nx[o.q0] = i; --left; }
            if (o.nq == 2 && nx[o.q1] == ops.size()) { nx[o.q1] = i; --left; }
        }
        return nx;
    }

    // Moves the qubits `low` (kC of them, all in S) to physical bits 0 .. kC-1; the qubits they
    // displace take the positions they leave.
    void set_low(const std::vector<int>& low) {
        std::vector<int> leaving;
        for (int p = 0; p < kC; ++p)
            if (std::find(low.begin(), low.end(), at[p]) == low.end()) leaving.push_back(at[p]);
        std::vector<int> arriving;
        for (int q : low)
            if (phys[q] >= kC) arriving.push_back(q);
        for (size_t i = 0; i < arriving.size(); ++i) {
            const int a = arriving[i], b = leaving[i];
            std::swap(phys[a], phys[b]);
            at[phys[a]] = a;
            at[phys[b]] = b;
        }
    }
};

// Tile bit of each logical qubit of S (rank of its physical position) and the positions.
void tile_positions(uint64_t S, const std::vector<int>& phys, std::vector<int>& P, std::vector<int>& tbit, int n) {
    P.clear();
    for (int q = 0; q < n; ++q)
        if ((S >> q) & 1u) P.push_back(phys[q]);
    std::sort(P.begin(), P.end());
    tbit.assign(n, -1);
    for (int q = 0; q < n; ++q)
        if ((S >> q) & 1u) tbit[q] = (int)(std::lower_bound(P.begin(), P.end(), phys[q]) - P.begin());
}

void op_matrix(const Circuit& c, uint32_t op, uint32_t k, cd* m, int& dim) {
    const ptsbe_op& o = c.ops[op];
    if (o.kind == PTSBE_OP_GATE) {
        const double* custom = nullptr;
        if (o.id == PTSBE_G_U1 || o.id == PTSBE_G_U2) custom = c.custom.data() + 32 * (size_t)o.params[0];
        gate_matrix_of(o.id, o.params, custom, m, dim);
        return;
    }
    const HostChannel& ch = c.ch[o.id];
    const uint32_t dd = ch.dim * ch.dim;
    const cd* src = ch.mixture ? &ch.U[(size_t)k * dd] : &ch.K[(size_t)k * dd];
    for (uint32_t i = 0; i < dd; ++i) m[i] = src[i];
    dim = (int)ch.dim;
}

// Number of the register pair (lo, hi), lo < hi < kR, in the order (0,1) (0,2) .. (0,kR-1) (1,2) ..
int pair_index(int lo, int hi) {
    int k = 0;
    for (int a = 0; a < kR; ++a)
        for (int b = a + 1; b < kR; ++b) {
            if (a == lo && b == hi) return k;
            ++k;
        }
    fail(PTSBE_ERR_INVALID, "bad register pair");
}

}  // namespace

namespace {

// Product of block b's operators in its logical basis (2 bit(qa) + bit(qb)), Kraus operator ks[i]
// at site sites[i] and operator 0 at the block's other sites.
void block_product(const Circuit& c, const DensePlan& P, uint32_t b, const uint32_t* sites, const uint8_t* ks,
                   uint32_t len, cd* M) {
    const int nq = P.blk_nq[b];
    const int d = nq == 1 ? 2 : 4;
    cd E[16], m[16], t[16];
    for (int i = 0; i < d * d; ++i) M[i] = (i % (d + 1) == 0) ? cd(1.0) : cd(0.0);
    uint32_t e = 0;
    const uint32_t qs2[2] = {P.blk_qa[b], P.blk_qb[b]};
    for (uint32_t i = P.blk_op_off[b]; i < P.blk_op_off[b + 1]; ++i) {
        const uint32_t op = P.blk_ops[i];
        const ptsbe_op& o = c.ops[op];
        uint32_t k = 0;
        if (o.kind == PTSBE_OP_NOISE) {
            // entries are sorted by site, and so are the block's sites
            while (e < len && c.site_op[sites[e]] < op) ++e;
            if (e < len && c.site_op[sites[e]] == op) k = ks[e];
        }
        int dim = 2;
        op_matrix(c, op, k, m, dim);
        const cd* A = m;
        if (nq == 2) {
            embed_pair(m, dim, o.targets, qs2[0], qs2[1], E);
            A = E;
        }
        for (int r = 0; r < d; ++r)
            for (int col = 0; col < d; ++col) {
                cd sum = 0;
                for (int x = 0; x < d; ++x) sum += A[r * d + x] * M[x * d + col];
                t[r * d + col] = sum;
            }
        for (int i2 = 0; i2 < d * d; ++i2) M[i2] = t[i2];
    }
}

// Entry l of a per-qubit diagonal pair product: 2 qubits l = 2 a + b -> x[a] y[b]; 1 qubit x[l].
cd diag_entry(const std::array<cd, 4>& D, int nq, int l) { return nq == 1 ? D[l] : D[l >> 1] * D[2 + (l & 1)]; }

// Logical -> kernel index of a block's local basis.
int kernel_index(const DensePlan& P, uint32_t b, int l) {
    return (P.blk_nq[b] == 2 && P.blk_swap[b]) ? (((l & 1) << 1) | (l >> 1)) : l;
}

// A = D_out R D_in with R real, D_in diagonal (entry 0 = 1) and D_out a product of one diagonal per
// qubit (x on qa, y on qb): phases phi_r + theta_c = arg A_rc (mod pi) over the nonzero entries,
// propagated from row 0, then checked on every entry. false when A has no such form.
bool factor_dr(const cd* A, int nq, cd* din, double* R, std::array<cd, 4>& dout) {
    const int d = nq == 1 ? 2 : 4;
    double amax = 0;
    for (int i = 0; i < d * d; ++i) amax = std::max(amax, std::abs(A[i]));
    if (!(amax > 0)) return false;
    const double eps = 1e-12 * amax;
    double phr[4], phc[4];
    bool kr[4] = {false, false, false, false}, kc[4] = {false, false, false, false};
    int r0 = -1;
    for (int r = 0; r < d && r0 < 0; ++r)
        for (int c2 = 0; c2 < d; ++c2)
            if (std::abs(A[r * d + c2]) > eps) { r0 = r; break; }
    phr[r0] = 0;
    kr[r0] = true;
    for (int it = 0; it < 2 * d; ++it)
        for (int r = 0; r < d; ++r)
            for (int c2 = 0; c2 < d; ++c2) {
                if (std::abs(A[r * d + c2]) <= eps) continue;
                const double ph = std::arg(A[r * d + c2]);
                if (kr[r] && !kc[c2]) { phc[c2] = ph - phr[r]; kc[c2] = true; }
                else if (kc[c2] && !kr[r]) { phr[r] = ph - phc[c2]; kr[r] = true; }
            }
    for (int i = 0; i < d; ++i) {
        if (!kr[i]) { if (nq == 2) return false; phr[i] = 0; }
        if (!kc[i]) { if (nq == 2) return false; phc[i] = 0; }
    }
    // every row and column is reached from row 0 (one component): the phases are fixed up to
    // multiples of pi per row (absorbed as signs of R); make the row phases separable over qubits
    if (nq == 2) {
        const double delta = phr[0] + phr[3] - phr[1] - phr[2];
        const double k = std::nearbyint(delta / M_PI);
        if (std::abs(delta - k * M_PI) > 1e-9) return false;
        if (((long long)k) & 1) phr[3] += M_PI;
    }
    // D_in entry 0 = 1: its phase moves to D_out (a common phase, separable)
    const double t0 = phc[0];
    for (int c2 = 0; c2 < d; ++c2) phc[c2] -= t0;
    for (int r = 0; r < d; ++r) phr[r] += t0;
    for (int r = 0; r < d; ++r)
        for (int c2 = 0; c2 < d; ++c2) {
            const cd x = A[r * d + c2] * std::polar(1.0, -(phr[r] + phc[c2]));
            if (std::abs(x.imag()) > 1e-10 * amax) return false;
            R[r * d + c2] = x.real();
        }
    for (int c2 = 0; c2 < d; ++c2) din[c2] = std::polar(1.0, phc[c2]);
    if (nq == 1) {
        dout = {std::polar(1.0, phr[0]), std::polar(1.0, phr[1]), cd(1.0), cd(1.0)};
    } else {
        // phr[2a + b] = alpha_a + beta_b with alpha_0 = 0
        dout = {cd(1.0), std::polar(1.0, phr[2] - phr[0]), std::polar(1.0, phr[0]), std::polar(1.0, phr[1])};
        for (int l = 0; l < 4; ++l)
            if (std::abs(diag_entry(dout, 2, l) - std::polar(1.0, phr[l])) > 1e-9) return false;
    }
    return true;
}

// Kernel-layout general matrix of K (logical basis) into out (complex64).
void store_general(const DensePlan& P, uint32_t b, const cd* K, float2* out) {
    const int d = P.blk_nq[b] == 1 ? 2 : 4;
    for (int r = 0; r < d; ++r)
        for (int c2 = 0; c2 < d; ++c2) {
            const cd x = K[r * d + c2];
            out[kernel_index(P, b, r) * d + kernel_index(P, b, c2)] = make_float2((float)x.real(), (float)x.imag());
        }
}

}  // namespace

void dense_block_matrix(const Circuit& c, const DensePlan& P, uint32_t b, const uint32_t* sites, const uint8_t* ks,
                        uint32_t len, float2* out, uint32_t* code) {
    const int nq = P.blk_nq[b];
    const int d = nq == 1 ? 2 : 4;
    cd M[16], K[16];
    block_product(c, P, b, sites, ks, len, M);
    // the kernel holds D_out^-1 (state) on the block's output and takes D_in-phased input
    for (int r = 0; r < d; ++r)
        for (int c2 = 0; c2 < d; ++c2)
            K[r * d + c2] = M[r * d + c2] * diag_entry(P.blk_pin[b], nq, c2) / diag_entry(P.blk_pout[b], nq, r);
    store_general(P, b, K, out);
    const int gcode = P.blocks[b].code >= kCodeDR ? P.blocks[b].code - kCodeDR : P.blocks[b].code;
    if (code) *code = (uint32_t)gcode;
}

void make_dense_plan(const Circuit& c, DensePlan& P) {
    // a state of fewer than kT qubits is planned as a kT-qubit one: the extra qubits carry no
    // operation and stay |0>, so the circuit's state is the first 2^n amplitudes of the plan's
    const int n = std::max((int)c.n, kT);
    if (c.n < 1 || n > kMaxQ) fail(PTSBE_ERR_UNSUPPORTED, "dense passes need 1 <= n <= 32");
    P = DensePlan{};
    P.n = n;
    Planner pl;
    pl.n = n;
    pl.T = kT;
    pl.ops.resize(c.ops.size());
    for (size_t i = 0; i < c.ops.size(); ++i) {
        const ptsbe_op& o = c.ops[i];
        pl.ops[i] = OpQ{o.targets[0], o.n_targets == 2 ? o.targets[1] : o.targets[0], (uint8_t)o.n_targets};
    }
    pl.done.assign(c.ops.size(), 0);
    pl.phys.resize(n);
    pl.at.resize(n);
    for (int q = 0; q < n; ++q) { pl.phys[q] = q; pl.at[q] = q; }

    std::vector<PassRec> recs;
    while (pl.first < pl.ops.size()) {
        uint32_t cnt = 0;
        const uint64_t S = pl.choose(pl.low_set(), &cnt);
        if (cnt == 0) fail(PTSBE_ERR_INVALID, "dense planner made no progress");
        PassRec r;
        r.S = S;
        r.phys_in = pl.phys;
        pl.exec(S, &r.ops);
        for (uint32_t i : r.ops) pl.done[i] = 1;
        while (pl.first < pl.ops.size() && pl.done[pl.first]) ++pl.first;
        if (pl.first < pl.ops.size()) {
            // qubits the next pass will likely hold go to the low bits
            uint32_t c2 = 0;
            const uint64_t S2 = pl.choose(0, &c2);
            const std::vector<size_t> nx = pl.next_pending();
            std::vector<int> cand;
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1u) cand.push_back(q);
            std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
                const bool ia = (S2 >> a) & 1u, ib = (S2 >> b) & 1u;
                if (ia != ib) return ia;
                return nx[a] < nx[b];
            });
            std::vector<int> low(cand.begin(), cand.begin() + kC);
            pl.set_low(low);
        }
        r.phys_out = pl.phys;
        recs.push_back(std::move(r));
    }
    // restore logical order: passes without operations, each fixing the qubits whose home lies
    // in its tile (tiles grown along permutation cycles, so every pass makes progress)
    for (int guard = 0; guard < 4 * n; ++guard) {
        std::vector<int> disp;
        for (int p = 0; p < n; ++p)
            if (pl.at[p] != p) disp.push_back(p);
        if (disp.empty()) break;
        std::vector<int> Pp;
        for (int p = 0; p < kC; ++p) Pp.push_back(p);
        auto has = [&](int p) { return std::find(Pp.begin(), Pp.end(), p) != Pp.end(); };
        for (int p0 : disp) {
            int p = p0;
            while ((int)Pp.size() < kT && !has(p)) {
                Pp.push_back(p);
                p = pl.at[p];   // the home of the qubit at p is position at[p]
            }
            if ((int)Pp.size() >= kT) break;
        }
        for (int p = 0; p < n && (int)Pp.size() < kT; ++p)
            if (!has(p)) Pp.push_back(p);
        PassRec r;
        r.S = 0;
        for (int p : Pp) r.S |= 1ull << pl.at[p];
        r.phys_in = pl.phys;
        // qubits whose home is in the tile go home; the others take the free tile positions
        std::vector<int> qs;
        for (int p : Pp) qs.push_back(pl.at[p]);
        std::vector<int> freep;
        std::vector<uint8_t> taken(n, 0);
        for (int q : qs)
            if (has(q)) taken[q] = 1;
        for (int p : Pp)
            if (!taken[p]) freep.push_back(p);
        size_t fi = 0;
        for (int q : qs) pl.phys[q] = has(q) ? q : freep[fi++];
        for (int q : qs) pl.at[pl.phys[q]] = q;
        r.phys_out = pl.phys;
        recs.push_back(std::move(r));
        ++P.fixup_passes;
    }
    for (int p = 0; p < n; ++p)
        if (pl.at[p] != p) fail(PTSBE_ERR_INVALID, "dense planner could not restore logical order");

    // --- blocks, groups and tables of every pass ---
    std::vector<uint32_t> op_site(c.ops.size(), UINT32_MAX);
    for (uint32_t s = 0; s < c.site_op.size(); ++s) op_site[c.site_op[s]] = s;
    P.site_block.assign(c.site_op.size(), UINT32_MAX);
    P.blk_op_off.push_back(0);
    for (size_t j = 0; j < recs.size(); ++j) {
        const PassRec& r = recs[j];
        std::vector<int> pos, tbit;
        tile_positions(r.S, r.phys_in, pos, tbit, n);
        // fuse
        struct TB {
            int nq;
            uint32_t qa, qb;
            std::vector<uint32_t> ops;
            bool alive;
        };
        std::vector<TB> bl;
        std::vector<int> open(n, -1);
        for (uint32_t i : r.ops) {
            const OpQ& o = pl.ops[i];
            if (o.nq == 1) {
                const int b = open[o.q0];
                if (b >= 0) bl[b].ops.push_back(i);
                else { bl.push_back(TB{1, o.q0, o.q0, {i}, true}); open[o.q0] = (int)bl.size() - 1; }
                continue;
            }
            const int bx = open[o.q0], by = open[o.q1];
            if (bx >= 0 && bx == by) { bl[bx].ops.push_back(i); continue; }
            TB nb{2, o.q0, o.q1, {}, true};
            if (bx >= 0 && bl[bx].nq == 1) { nb.ops = bl[bx].ops; bl[bx].alive = false; }
            if (by >= 0 && bl[by].nq == 1) {
                nb.ops.insert(nb.ops.end(), bl[by].ops.begin(), bl[by].ops.end());
                bl[by].alive = false;
            }
            nb.ops.push_back(i);
            bl.push_back(std::move(nb));
            open[o.q0] = open[o.q1] = (int)bl.size() - 1;
        }
        std::vector<int> order;
        for (size_t b = 0; b < bl.size(); ++b)
            if (bl[b].alive) {
                // an absorbed block's operations were appended out of circuit order; circuit order
                // restricted to a block's operations is a valid order for its product
                std::sort(bl[b].ops.begin(), bl[b].ops.end());
                order.push_back((int)b);
            }
        auto tmask = [&](const TB& b) {
            uint32_t m = 1u << tbit[b.qa];
            if (b.nq == 2) m |= 1u << tbit[b.qb];
            return m;
        };
        Pass ps{};
        ps.group_begin = (uint32_t)P.groups.size();
        ps.blk_begin = (uint32_t)P.blocks.size();
        ps.nops = (uint32_t)r.ops.size();
        std::vector<uint8_t> used(order.size(), 0);
        size_t left = order.size();
        while (left > 0) {
            uint32_t G = 0, blocked = 0;
            std::vector<int> chosen;
            for (size_t x = 0; x < order.size(); ++x) {
                if (used[x]) continue;
                const uint32_t m = tmask(bl[order[x]]);
                if (m & blocked) { blocked |= m; continue; }
                if (pop(G | m) <= kR) { G |= m; chosen.push_back((int)x); }
                else blocked |= m;
            }
            for (int x : chosen) used[x] = 1;
            left -= chosen.size();
            // register bits: G, padded with the tile bits of the most common residue mod 4
            std::vector<int> R;
            for (int t = 0; t < kT; ++t)
                if ((G >> t) & 1u) R.push_back(t);
            while ((int)R.size() < kR) {
                int cntres[4] = {0, 0, 0, 0};
                for (int t = 0; t < kT; ++t)
                    if (std::find(R.begin(), R.end(), t) == R.end()) ++cntres[t & 3];
                int pick = -1;
                for (int t = kT - 1; t >= 0; --t) {
                    if (std::find(R.begin(), R.end(), t) != R.end()) continue;
                    if (pick < 0 || cntres[t & 3] > cntres[pick & 3]) pick = t;
                }
                R.push_back(pick);
            }
            std::sort(R.begin(), R.end());
            // thread bits: lanes 0..3 on tile bits of distinct residues mod 4 (distinct banks)
            std::vector<int> rest;
            for (int t = 0; t < kT; ++t)
                if (std::find(R.begin(), R.end(), t) == R.end()) rest.push_back(t);
            std::vector<int> tb;
            bool res_used[4] = {false, false, false, false};
            for (int t : rest)
                if ((int)tb.size() < 4 && !res_used[t & 3]) { tb.push_back(t); res_used[t & 3] = true; }
            for (int t : rest)
                if (std::find(tb.begin(), tb.end(), t) == tb.end()) tb.push_back(t);
            Group g{};
            for (int k = 0; k < kTB; ++k) g.toff[k] = (uint16_t)swz(1u << tb[k]);
            for (int jj = 0; jj < kAmps; ++jj) {
                uint32_t t = 0;
                for (int mbit = 0; mbit < kR; ++mbit)
                    if ((jj >> mbit) & 1) t |= 1u << R[mbit];
                g.roff[jj] = (uint16_t)swz(t);
            }
            g.blk_begin = (uint32_t)P.blocks.size();
            for (int x : chosen) {
                const TB& b = bl[order[x]];
                const uint32_t id = (uint32_t)P.blocks.size();
                Block B{};
                B.id = id;
                const int ia = (int)(std::find(R.begin(), R.end(), tbit[b.qa]) - R.begin());
                uint8_t swap = 0;
                if (b.nq == 1) {
                    B.code = (uint8_t)ia;
                } else {
                    const int ib = (int)(std::find(R.begin(), R.end(), tbit[b.qb]) - R.begin());
                    B.code = (uint8_t)(kCodes1 + pair_index(std::min(ia, ib), std::max(ia, ib)));
                    swap = ia < ib ? 1 : 0;
                }
                P.blocks.push_back(B);
                P.blk_nq.push_back((uint8_t)b.nq);
                P.blk_qa.push_back(b.qa);
                P.blk_qb.push_back(b.qb);
                P.blk_swap.push_back(swap);
                P.blk_pass.push_back((uint32_t)j);
                for (uint32_t op : b.ops) {
                    P.blk_ops.push_back(op);
                    if (op_site[op] != UINT32_MAX) P.site_block[op_site[op]] = id;
                }
                P.blk_op_off.push_back((uint32_t)P.blk_ops.size());
            }
            g.blk_end = (uint32_t)P.blocks.size();
            P.groups.push_back(g);
        }
        ps.group_end = (uint32_t)P.groups.size();
        ps.blk_end = (uint32_t)P.blocks.size();
        // tables: input offsets of tile bits [kC, kT); output order
        ps.hi_off = (uint32_t)P.hi.size();
        for (int h = 0; h < kHi; ++h) {
            uint32_t o = 0;
            for (int b = 0; b < kT - kC; ++b)
                if ((h >> b) & 1) o |= 1u << pos[kC + b];
            P.hi.push_back(o);
        }
        std::vector<int> rho(kT);   // output rank -> tile bit
        for (int q = 0; q < n; ++q) {
            if (!((r.S >> q) & 1u)) continue;
            const int rank = (int)(std::lower_bound(pos.begin(), pos.end(), r.phys_out[q]) - pos.begin());
            if (rank >= kT || pos[rank] != r.phys_out[q]) fail(PTSBE_ERR_INVALID, "dense planner moved a qubit out of its tile");
            rho[rank] = tbit[q];
        }
        ps.omap_off = (uint32_t)P.omap.size();
        for (int h = 0; h < kHi; ++h) {
            uint32_t t = 0;
            for (int b = 0; b < kT - kC; ++b)
                if ((h >> b) & 1) t |= 1u << rho[kC + b];
            P.omap.push_back((uint16_t)t);
        }
        for (int x = 0; x < (1 << kC); ++x) {
            uint32_t t = 0;
            for (int b = 0; b < kC; ++b)
                if ((x >> b) & 1) t |= 1u << rho[b];
            ps.olow[x] = (uint16_t)t;
        }
        ps.nouter = 0;
        for (int p = 0; p < n; ++p)
            if (!std::binary_search(pos.begin(), pos.end(), p)) ps.opos[ps.nouter++] = (uint8_t)p;
        P.passes.push_back(ps);
    }
    // default matrices, in block order (each pass's matrices one contiguous range). A block whose
    // qubits all have a later block takes the diagonal-times-real form: with the phases P_in it
    // inherits, M P_in = D_out R D_in; it applies D_in then R, and D_out (one diagonal per qubit)
    // passes on to the next blocks of those qubits. A qubit's last block is general and absorbs
    // what is left, so the final state carries no pending phase.
    const uint32_t NB = (uint32_t)P.blocks.size();
    std::vector<uint32_t> last_blk(n, UINT32_MAX);
    for (uint32_t b = 0; b < NB; ++b) {
        last_blk[P.blk_qa[b]] = b;
        if (P.blk_nq[b] == 2) last_blk[P.blk_qb[b]] = b;
    }
    std::vector<std::array<cd, 2>> pend(n, {cd(1.0), cd(1.0)});
    P.blk_pin.resize(NB);
    P.blk_pout.resize(NB);
    for (uint32_t b = 0; b < NB; ++b) {
        const int nq = P.blk_nq[b];
        const int d = nq == 1 ? 2 : 4;
        const uint32_t qa = P.blk_qa[b], qb = P.blk_qb[b];
        P.blk_pin[b] = {pend[qa][0], pend[qa][1], nq == 2 ? pend[qb][0] : cd(1.0), nq == 2 ? pend[qb][1] : cd(1.0)};
        cd M[16], A[16], din[4];
        double R[16];
        block_product(c, P, b, nullptr, nullptr, 0, M);
        for (int r = 0; r < d; ++r)
            for (int c2 = 0; c2 < d; ++c2) A[r * d + c2] = M[r * d + c2] * diag_entry(P.blk_pin[b], nq, c2);
        std::array<cd, 4> dout{};
        const bool later = last_blk[qa] != b && (nq == 1 || last_blk[qb] != b);
        P.blocks[b].mat = (uint32_t)P.mats.size();
        if (later && factor_dr(A, nq, din, R, dout)) {
            P.blk_pout[b] = dout;
            pend[qa] = {dout[0], dout[1]};
            if (nq == 2) pend[qb] = {dout[2], dout[3]};
            P.blocks[b].code = (uint8_t)(P.blocks[b].code + kCodeDR);
            const uint32_t cnt = code_mat_count(P.blocks[b].code);
            P.mats.resize(P.mats.size() + cnt, make_float2(0.f, 0.f));
            float2* m = &P.mats[P.blocks[b].mat];
            float dk[4][2], Rk[16];
            for (int c2 = 0; c2 < d; ++c2) {
                const int kc = kernel_index(P, b, c2);
                dk[kc][0] = (float)din[c2].real();
                dk[kc][1] = (float)din[c2].imag();
                for (int r = 0; r < d; ++r) Rk[kernel_index(P, b, r) * d + kc] = (float)R[r * d + c2];
            }
            for (int i = 1; i < d; ++i) m[i - 1] = make_float2(dk[i][0], dk[i][1]);
            float* rf = reinterpret_cast<float*>(m + (nq == 1 ? 2 : 4));
            for (int i = 0; i < d * d; ++i) rf[i] = Rk[i];
        } else {
            P.blk_pout[b] = {cd(1.0), cd(1.0), cd(1.0), cd(1.0)};
            pend[qa] = {cd(1.0), cd(1.0)};
            if (nq == 2) pend[qb] = {cd(1.0), cd(1.0)};
            const uint32_t cnt = code_mat_count(P.blocks[b].code);
            P.mats.resize(P.mats.size() + cnt);
            store_general(P, b, A, &P.mats[P.blocks[b].mat]);
        }
    }
    for (Pass& ps : P.passes) {
        ps.mat_begin = ps.blk_begin < ps.blk_end ? P.blocks[ps.blk_begin].mat : 0;
        ps.mat_end = ps.blk_begin < ps.blk_end ? P.blocks[ps.blk_end - 1].mat + code_mat_count(P.blocks[ps.blk_end - 1].code) : 0;
        const size_t bytes = dense_stage_bytes(ps);
        if (bytes > (size_t)kStageMax) fail(PTSBE_ERR_INVALID, "dense planner: a pass's tables exceed the shared-memory stage");
        ps.stage_bytes = (uint32_t)bytes;
    }
    // gates applied per pass (prefix-reuse accounting)
    P.pass_fma.assign(P.passes.size(), 0);
    for (uint32_t b = 0; b < P.blocks.size(); ++b) {
        const int code = P.blocks[b].code;
        // per amplitude: general 2x2 8, 4x4 16; diagonal-times-real 2x2 6 (2 + 4), 4x4 11 (3 + 8)
        P.pass_fma[P.blk_pass[b]] += code < kCodes1 ? 8 : code < kCodeDR ? 16 : code < kCodeDR + kCodes1 ? 6 : 11;
    }
    P.pass_gates.assign(P.passes.size(), 0);
    for (size_t j = 0; j < recs.size(); ++j)
        for (uint32_t i : recs[j].ops)
            if (c.ops[i].kind == PTSBE_OP_GATE) ++P.pass_gates[j];
    for (uint32_t s = 0; s < c.site_op.size(); ++s)
        if (P.site_block[s] == UINT32_MAX) fail(PTSBE_ERR_INVALID, "dense planner left a noise site out");
    P.built = true;
}

}  // namespace ptsbe
