// Host plan of the adjoint backward: fused blocks ("items"), qubit-position swaps between the
// CTAs of a cluster, and the matrix tables the kernels read.
//
// Items. Consecutive operators (gates and noise sites) that act inside one or two qubits are
// multiplied into one block. A qubit keeps one open item; an operator on qubits already covered by
// an open item joins it; a two-qubit operator merges the open one-qubit items of its qubits (they
// commute with everything issued since they opened) and closes open two-qubit items it cannot
// join. Items are issued in the order they close, which respects every dependence.
//
// Layout. A state of n qubits is spread over 2^(n - nl) CTAs: physical bit positions [0, nl) are
// the local index, [nl, n) the CTA rank. Logical qubit q sits at position pos[q]; an item whose
// qubit is at a rank position first swaps it with the local position whose next use lies farthest
// in the future.
//
// Matrices. For every member: its variants (one for a gate, one per Kraus operator for a noise
// site) embedded in the item's 2 or 4 dimensional space, their inverses (FP32), the same variants
// in FP64 and the derivative matrices of the parameters the loss is differentiated by (FP64).
// Unitary-mixture channels of the Pauli kinds are applied as U_k = K_k / sqrt(q_k) with the scale
// tracked on the host; every other channel applies K_k.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace ptsbe {

namespace {

using Mat = std::array<cd, 16>;

bool param_gate(uint32_t g, int& nangles) {
    switch (g) {
    case PTSBE_G_RX: case PTSBE_G_RY: case PTSBE_G_RZ: nangles = 1; return true;
    case PTSBE_G_U3: nangles = 3; return true;
    default: nangles = 0; return false;
    }
}

// d/d params[j] of the gate matrix (RX, RY, RZ: theta = exp(-i theta P / 2); U3 in the OpenQASM
// convention), 2x2 row-major.
void gate_derivative(uint32_t g, const double* p, int j, cd* m) {
    const cd I(0, 1);
    for (int i = 0; i < 4; ++i) m[i] = 0;
    const double t = p[0] / 2, c = std::cos(t), s = std::sin(t);
    switch (g) {
    case PTSBE_G_RX: m[0] = -0.5 * s; m[3] = m[0]; m[1] = -0.5 * I * c; m[2] = m[1]; break;
    case PTSBE_G_RY: m[0] = -0.5 * s; m[1] = -0.5 * c; m[2] = 0.5 * c; m[3] = -0.5 * s; break;
    case PTSBE_G_RZ: m[0] = -0.5 * I * std::polar(1.0, -t); m[3] = 0.5 * I * std::polar(1.0, t); break;
    case PTSBE_G_U3: {
        const double ph = p[1], la = p[2];
        if (j == 0) {
            m[0] = -0.5 * s; m[1] = -0.5 * std::polar(1.0, la) * c;
            m[2] = 0.5 * std::polar(1.0, ph) * c; m[3] = -0.5 * std::polar(1.0, ph + la) * s;
        } else if (j == 1) {
            m[2] = I * std::polar(1.0, ph) * s; m[3] = I * std::polar(1.0, ph + la) * c;
        } else {
            m[1] = -I * std::polar(1.0, la) * s; m[3] = I * std::polar(1.0, ph + la) * c;
        }
        break;
    }
    default: break;
    }
}

// Gauss-Jordan inverse with partial pivoting (d <= 4). Returns false when a pivot is negligible
// or the inverse amplifies by more than 1e4 (the input then comes from a checkpoint instead).
bool invert(const cd* a, int d, cd* out) {
    cd m[4][8];
    double scale = 0;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) { m[r][c] = a[r * d + c]; m[r][d + c] = r == c ? 1.0 : 0.0; scale = std::max(scale, std::abs(m[r][c])); }
    if (!(scale > 0)) return false;
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (std::abs(m[r][c]) > std::abs(m[piv][c])) piv = r;
        if (!(std::abs(m[piv][c]) > 1e-9 * scale)) return false;
        if (piv != c) for (int k = 0; k < 2 * d; ++k) std::swap(m[piv][k], m[c][k]);
        const cd inv = 1.0 / m[c][c];
        for (int k = 0; k < 2 * d; ++k) m[c][k] *= inv;
        for (int r = 0; r < d; ++r)
            if (r != c) {
                const cd f = m[r][c];
                if (f != 0.0) for (int k = 0; k < 2 * d; ++k) m[r][k] -= f * m[c][k];
            }
    }
    double big = 0;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) { out[r * d + c] = m[r][d + c]; big = std::max(big, std::abs(out[r * d + c])); }
    return big <= 1e4;
}

// Largest eigenvalue of A^dag A, the squared spectral norm of the d x d matrix A (power iteration;
// d <= 4, a bound for a planning threshold, not a result).
double norm2_sq(const cd* A, int d) {
    cd v[4];
    for (int i = 0; i < d; ++i) v[i] = cd(1.0 + 0.17 * i, 0.05 * i);
    double lam = 0.0;
    for (int it = 0; it < 200; ++it) {
        double nv = 0.0;
        for (int i = 0; i < d; ++i) nv += std::norm(v[i]);
        nv = std::sqrt(nv);
        if (!(nv > 0.0)) return 0.0;
        for (int i = 0; i < d; ++i) v[i] /= nv;
        cd t[4], w[4];
        for (int r = 0; r < d; ++r) {
            t[r] = 0.0;
            for (int c = 0; c < d; ++c) t[r] += A[r * d + c] * v[c];
        }
        for (int c = 0; c < d; ++c) {
            w[c] = 0.0;
            for (int r = 0; r < d; ++r) w[c] += std::conj(A[r * d + c]) * t[r];
        }
        double nw = 0.0;
        for (int i = 0; i < d; ++i) { nw += std::norm(w[i]); v[i] = w[i]; }
        lam = std::sqrt(nw);
    }
    return lam;
}

void mul(const cd* A, const cd* B, cd* out, int d) {   // out = A B
    cd t[16];
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            cd s = 0;
            for (int k = 0; k < d; ++k) s += A[r * d + k] * B[k * d + c];
            t[r * d + c] = s;
        }
    std::copy(t, t + d * d, out);
}

struct Work {   // item under construction
    uint32_t q[2];
    int nq;
    std::vector<uint32_t> ops;
};

}  // namespace

void make_backward_plan(const Circuit& c, BwPlan& P) {
    P = BwPlan{};
    const int n = (int)c.n;
    if (n > kBwMaxQubits) fail(PTSBE_ERR_UNSUPPORTED, "backward handles at most 16 qubits");
    P.nl = std::min(n, kBwLocalBits);
    const size_t nops = c.ops.size();

    // ---- items ---------------------------------------------------------------------------------
    std::vector<Work> done;
    std::vector<int> open(n, -1);        // qubit -> index into `live`
    std::vector<Work> live;
    std::vector<bool> alive;
    auto close = [&](int w) {
        Work& it = live[w];
        for (int i = 0; i < it.nq; ++i) open[it.q[i]] = -1;
        done.push_back(it);
        alive[w] = false;
    };
    auto fresh = [&](uint32_t a, uint32_t b, int nq) {
        live.push_back(Work{{a, b}, nq, {}});
        alive.push_back(true);
        const int w = (int)live.size() - 1;
        open[a] = w;
        if (nq == 2) open[b] = w;
        return w;
    };
    for (size_t i = 0; i < nops; ++i) {
        const ptsbe_op& o = c.ops[i];
        const uint32_t a = o.targets[0], b = o.n_targets == 2 ? o.targets[1] : a;
        if (o.n_targets == 1) {
            int w = open[a];
            if (w >= 0 && live[w].ops.size() >= (size_t)kBwMaxMembers) { close(w); w = -1; }
            if (w < 0) w = fresh(a, a, 1);
            live[w].ops.push_back((uint32_t)i);
            continue;
        }
        int wa = open[a], wb = open[b];
        if (wa >= 0 && wa == wb && live[wa].ops.size() < (size_t)kBwMaxMembers) {
            live[wa].ops.push_back((uint32_t)i);
            continue;
        }
        if (wa >= 0 && (live[wa].nq == 2 || live[wa].ops.size() >= (size_t)kBwMaxMembers / 2)) { close(wa); wa = -1; }
        wb = open[b];
        if (wb >= 0 && (live[wb].nq == 2 || live[wb].ops.size() >= (size_t)kBwMaxMembers / 2)) { close(wb); wb = -1; }
        std::vector<uint32_t> merged;
        if (wa >= 0) { merged = live[wa].ops; alive[wa] = false; open[a] = -1; }
        if (wb >= 0) { merged.insert(merged.end(), live[wb].ops.begin(), live[wb].ops.end()); alive[wb] = false; open[b] = -1; }
        const int w = fresh(a, b, 2);
        live[w].ops = std::move(merged);
        live[w].ops.push_back((uint32_t)i);
    }
    for (size_t w = 0; w < live.size(); ++w)
        if (alive[w]) close((int)w);

    // ---- positions and swaps ---------------------------------------------------------------------
    std::vector<int> pos(n), at(n);
    for (int q = 0; q < n; ++q) { pos[q] = q; at[q] = q; }
    const int nl = P.nl;
    // next use of each qubit after item t, for the farthest-future choice
    auto next_use = [&](uint32_t q, size_t from) {
        for (size_t t = from; t < done.size(); ++t)
            for (int i = 0; i < done[t].nq; ++i)
                if (done[t].q[i] == q) return t;
        return done.size() + 1;
    };
    std::vector<uint32_t> item_of_step;
    for (size_t t = 0; t < done.size(); ++t) {
        const Work& it = done[t];
        for (int i = 0; i < it.nq; ++i) {
            const uint32_t q = it.q[i];
            if (pos[q] < nl) continue;
            int best = -1;
            size_t best_use = 0;
            for (int l = 0; l < nl; ++l) {
                const uint32_t ql = (uint32_t)at[l];
                if (it.nq == 2 && ql == it.q[1 - i]) continue;
                const size_t u = next_use(ql, t);
                if (best < 0 || u > best_use) { best = l; best_use = u; }
            }
            const int g = pos[q];
            P.steps.push_back(BwStep{1u, (uint32_t)best, (uint32_t)g, 0u});
            const uint32_t qb = (uint32_t)at[best];
            std::swap(at[best], at[g]);
            pos[q] = best; pos[qb] = g;
        }
        P.steps.push_back(BwStep{0u, 0u, 0u, (uint32_t)t});
        BwItem bi{};
        bi.nq = (uint8_t)it.nq;
        bi.p0 = (uint8_t)pos[it.q[0]];
        bi.p1 = (uint8_t)(it.nq == 2 ? pos[it.q[1]] : 0);
        P.items.push_back(bi);
    }
    for (const BwItem& it : P.items)
        if (it.p0 >= nl || (it.nq == 2 && (it.p1 >= nl || it.p1 == it.p0)))
            fail(PTSBE_ERR_INVALID, "backward plan placed a block outside the local bits");
    P.pos_final.resize(n);
    for (int q = 0; q < n; ++q) P.pos_final[q] = (uint8_t)pos[q];

    // ---- members and matrices -------------------------------------------------------------------
    auto push32 = [&](const cd* m, int d) {
        const uint32_t blk = (uint32_t)(P.pool.size() / 16);
        P.pool.resize(P.pool.size() + 16, float2{0.f, 0.f});
        for (int i = 0; i < d * d; ++i) P.pool[blk * 16 + i] = float2{(float)m[i].real(), (float)m[i].imag()};
        return blk;
    };
    auto push64 = [&](const cd* m, int d) {
        const uint32_t blk = (uint32_t)(P.pool64.size() / 32);
        P.pool64.resize(P.pool64.size() + 32, 0.0);
        for (int i = 0; i < d * d; ++i) { P.pool64[blk * 32 + 2 * i] = m[i].real(); P.pool64[blk * 32 + 2 * i + 1] = m[i].imag(); }
        return blk;
    };
    const uint32_t S = (uint32_t)c.site_op.size();
    P.site_item.assign(S, kBwNone);
    P.site_mem.assign(S, kBwNone);
    std::vector<uint32_t> op_site(nops, kBwNone);
    for (uint32_t s = 0; s < S; ++s) op_site[c.site_op[s]] = s;
    P.P0mix = 1.0;
    for (uint32_t s = 0; s < S; ++s) {
        const HostChannel& ch = c.ch[c.site_ch[s]];
        if (bw_unit_channel(ch)) P.P0mix *= ch.q[0];
    }
    double cond_run = 0.0;   // log2 of the product of kappa since the last stored copy
    P.cond_ckpts = 0;
    P.logc.clear();
    P.logc_off.clear();
    P.logc_default = 0.0;
    for (size_t t = 0; t < done.size(); ++t) {
        const Work& it = done[t];
        BwItem& bi = P.items[t];
        const int d = it.nq == 2 ? 4 : 2;
        bi.mbeg = (uint32_t)P.members.size();
        Mat B{}, Bi{};
        for (int i = 0; i < d; ++i) { B[i * d + i] = 1; Bi[i * d + i] = 1; }
        bool dsing = false, diff = false;
        for (uint32_t opi : it.ops) {
            const ptsbe_op& o = c.ops[opi];
            BwMember m{};
            m.dslot = kBwNone;
            auto embed = [&](const cd* src, int sd, cd* out) {
                if (it.nq == 1) { std::copy(src, src + 4, out); return; }
                embed_pair(src, sd, o.targets, it.q[0], it.q[1], out);
            };
            std::vector<Mat> var, der;
            if (o.kind == PTSBE_OP_GATE) {
                cd g[16]; int gd;
                const double* custom = nullptr;
                if (o.id == PTSBE_G_U1 || o.id == PTSBE_G_U2) custom = c.custom.data() + 32 * (size_t)o.params[0];
                gate_matrix_of(o.id, o.params, custom, g, gd);
                Mat e{}; embed(g, gd, e.data()); var.push_back(e);
                int na = 0;
                if (param_gate(o.id, na)) {
                    for (int j = 0; j < na; ++j) {
                        cd dm[4]; gate_derivative(o.id, o.params, j, dm);
                        Mat de{}; embed(dm, 2, de.data()); der.push_back(de);
                        P.dslot_out.push_back(3 * (uint32_t)opi + (uint32_t)j);
                    }
                    m.dslot = P.ndslots; P.ndslots += (uint32_t)na;
                    m.nd = (uint8_t)na;
                    diff = true;
                }
                m.noise = 0; m.nk = 1;
            } else {
                const uint32_t s = op_site[opi];
                const HostChannel& ch = c.ch[o.id];
                const bool unit = bw_unit_channel(ch);
                const uint32_t dd = ch.dim * ch.dim;
                for (uint32_t k = 0; k < ch.nk; ++k) {
                    const cd* src = unit ? &ch.U[k * dd] : &ch.K[k * dd];
                    Mat e{}; embed(src, (int)ch.dim, e.data()); var.push_back(e);
                }
                if (ch.kind == PTSBE_CH_AMPDAMP) {
                    const double gm = ch.param;
                    cd d0[4] = {0, 0, 0, gm < 1 ? -0.5 / std::sqrt(1 - gm) : 0.0};
                    cd d1[4] = {0, gm > 0 ? 0.5 / std::sqrt(gm) : 0.0, 0, 0};
                    Mat e0{}, e1{}; embed(d0, 2, e0.data()); embed(d1, 2, e1.data());
                    der.push_back(e0); der.push_back(e1);
                    m.dslot = P.ndslots++;
                    P.dslot_out.push_back(0x80000000u | o.id);
                    m.nd = 1;
                    diff = true;
                }
                if (!unit) {
                    // variants (and their derivatives, same constant) scaled to spectral norm 1
                    P.logc_off.resize(P.members.size() + 1, kBwNone);
                    P.logc_off[P.members.size()] = (uint32_t)P.logc.size();
                    for (uint32_t k = 0; k < ch.nk; ++k) {
                        const double n2 = norm2_sq(&ch.K[k * dd], (int)ch.dim);
                        const double c = n2 > 0.0 ? 1.0 / std::sqrt(n2) : 1.0;
                        for (cd& x : var[k]) x *= c;
                        if (k < der.size()) for (cd& x : der[k]) x *= c;
                        P.logc.push_back(2.0 * std::log(c));
                    }
                    P.logc_default += P.logc[P.logc_off[P.members.size()]];
                }
                m.noise = 1; m.nk = (uint8_t)ch.nk;
                P.site_item[s] = (uint32_t)t;
                P.site_mem[s] = (uint32_t)P.members.size();
            }
            m.mat = (uint32_t)(P.pool.size() / 16);
            for (const Mat& e : var) push32(e.data(), d);
            m.inv = (uint32_t)(P.pool.size() / 16);
            m.sing = 0;
            for (size_t k = 0; k < var.size(); ++k) {
                Mat inv{};
                if (!invert(var[k].data(), d, inv.data())) { m.sing |= 1u << k; inv.fill(0.0); }
                push32(inv.data(), d);
            }
            m.m64 = (uint32_t)(P.pool64.size() / 32);
            for (const Mat& e : var) push64(e.data(), d);
            m.d64 = (uint32_t)(P.pool64.size() / 32);
            for (const Mat& e : der) push64(e.data(), d);
            // default product: variant 0
            mul(var[0].data(), B.data(), B.data(), d);
            if (m.sing & 1u) dsing = true;
            else {
                Mat inv{};
                invert(var[0].data(), d, inv.data());
                mul(Bi.data(), inv.data(), Bi.data(), d);
            }
            P.members.push_back(m);
        }
        bi.mend = (uint32_t)P.members.size();
        P.logc_off.resize(P.members.size(), kBwNone);
        bi.def = push32(B.data(), d);
        if (dsing) Bi.fill(0.0);
        bi.definv = push32(Bi.data(), d);
        bi.defsing = dsing ? 1u : 0u;
        bi.diff = diff ? 1 : 0;
        bi.gslot = diff ? P.ngs++ : kBwNone;
        if (dsing) P.defsing_items.push_back((uint32_t)t);
        // items are in forward order: a stored copy before block t ends the run of un-computed
        // blocks at t (a block whose default cannot be inverted is stored anyway)
        if (dsing) {
            cond_run = 0.0;
        } else {
            const double l2k = 0.5 * std::log2(std::max(1.0, norm2_sq(B.data(), d) * norm2_sq(Bi.data(), d)));
            if (cond_run + l2k > kBwCondLog2) {
                bi.ckpt = 1;
                ++P.cond_ckpts;
                cond_run = 0.0;
            } else {
                cond_run += l2k;
            }
        }
    }
    P.first_diff_step = (uint32_t)P.steps.size();
    for (size_t j = 0; j < P.steps.size(); ++j)
        if (P.steps[j].kind == 0 && P.items[P.steps[j].item].diff) { P.first_diff_step = (uint32_t)j; break; }
    P.built = true;
}

}  // namespace ptsbe
