// Circuit registration (Fig. 1) and evolution planning.
//
// Channels are CPTP Kraus sets (Sec. 2.2). A channel whose every operator satisfies
// K_k^dag K_k = q_k I is a unitary mixture (Sec. 2.2, item 2): its branch probabilities do not
// depend on the state, it is applied as U_k = K_k / sqrt(q_k) and needs no norm.
//
// Evolution plan: a state of n qubits is processed in tiles of 2^tb amplitudes held in shared
// memory. When n <= tb one tile is the whole state and the whole circuit runs in one pass.
// Otherwise the op sequence is cut greedily into stages whose ops all act inside one set of tb
// qubits; the set always contains the lb lowest qubits so each tile is made of contiguous
// 2^lb-amplitude segments (coalesced loads).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace ptsbe {

namespace {

const double kSqrtHalf = 0.70710678118654752440;

void gate_matrix(uint32_t g, const double* p, const double* custom, cd* m, int& dim) {
    const cd I(0, 1);
    for (int i = 0; i < 16; ++i) m[i] = 0;
    const double th = p[0], ph = p[1], la = p[2];
    dim = 2;
    switch (g) {
    case PTSBE_G_I: m[0] = 1; m[3] = 1; break;
    case PTSBE_G_X: m[1] = 1; m[2] = 1; break;
    case PTSBE_G_Y: m[1] = -I; m[2] = I; break;
    case PTSBE_G_Z: m[0] = 1; m[3] = -1; break;
    case PTSBE_G_H: m[0] = kSqrtHalf; m[1] = kSqrtHalf; m[2] = kSqrtHalf; m[3] = -kSqrtHalf; break;
    case PTSBE_G_S: m[0] = 1; m[3] = I; break;
    case PTSBE_G_SDG: m[0] = 1; m[3] = -I; break;
    case PTSBE_G_T: m[0] = 1; m[3] = std::polar(1.0, M_PI / 4); break;
    case PTSBE_G_TDG: m[0] = 1; m[3] = std::polar(1.0, -M_PI / 4); break;
    case PTSBE_G_RX: m[0] = std::cos(th / 2); m[1] = -I * std::sin(th / 2); m[2] = m[1]; m[3] = m[0]; break;
    case PTSBE_G_RY: m[0] = std::cos(th / 2); m[1] = -std::sin(th / 2); m[2] = std::sin(th / 2); m[3] = m[0]; break;
    case PTSBE_G_RZ: m[0] = std::polar(1.0, -th / 2); m[3] = std::polar(1.0, th / 2); break;
    case PTSBE_G_U3:
        m[0] = std::cos(th / 2);
        m[1] = -std::polar(1.0, la) * std::sin(th / 2);
        m[2] = std::polar(1.0, ph) * std::sin(th / 2);
        m[3] = std::polar(1.0, ph + la) * std::cos(th / 2);
        break;
    case PTSBE_G_U1:
        m[0] = cd(custom[0], custom[1]); m[1] = cd(custom[2], custom[3]);
        m[2] = cd(custom[8], custom[9]); m[3] = cd(custom[10], custom[11]);
        break;
    case PTSBE_G_CX: dim = 4; m[0] = 1; m[5] = 1; m[11] = 1; m[14] = 1; break;
    case PTSBE_G_CZ: dim = 4; m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
    case PTSBE_G_SWAP: dim = 4; m[0] = 1; m[6] = 1; m[9] = 1; m[15] = 1; break;
    case PTSBE_G_U2: dim = 4; for (int i = 0; i < 16; ++i) m[i] = cd(custom[2 * i], custom[2 * i + 1]); break;
    default: fail(PTSBE_ERR_INVALID, "unknown gate code " + std::to_string(g));
    }
}

uint32_t gate_arity(uint32_t g) {
    return (g == PTSBE_G_CX || g == PTSBE_G_CZ || g == PTSBE_G_SWAP || g == PTSBE_G_U2) ? 2 : 1;
}

void pauli(int a, cd* m) {
    const cd I(0, 1);
    m[0] = m[1] = m[2] = m[3] = 0;
    if (a == 0) { m[0] = 1; m[3] = 1; }
    if (a == 1) { m[1] = 1; m[2] = 1; }
    if (a == 2) { m[1] = -I; m[2] = I; }
    if (a == 3) { m[0] = 1; m[3] = -1; }
}

}  // namespace

// Builds the Kraus operators, nominal probabilities and unitary-mixture data of one channel.
void gate_matrix_of(uint32_t g, const double* params, const double* custom, cd* m, int& dim) {
    gate_matrix(g, params, custom, m, dim);
}

void build_channel(const ptsbe_channel& in, HostChannel& c) {
    c.kind = in.kind; c.arity = in.arity; c.nk = in.n_kraus; c.param = in.param;
    if (in.arity < 1 || in.arity > 2) fail(PTSBE_ERR_INVALID, "channel arity must be 1 or 2");
    if (in.n_kraus < 1 || in.n_kraus > (uint32_t)kMaxKraus) fail(PTSBE_ERR_INVALID, "channel needs 1..16 Kraus operators");
    c.dim = 1u << in.arity;
    const uint32_t d = c.dim, dd = d * d;
    const double p = in.param;
    c.K.assign((size_t)c.nk * dd, 0.0);
    c.q.assign(c.nk, 0.0);
    c.U.clear();
    auto need = [&](uint32_t ar, uint32_t nk) {
        if (in.arity != ar || in.n_kraus != nk) fail(PTSBE_ERR_INVALID, "channel arity/n_kraus mismatch for its kind");
        if (!(p >= 0 && p <= 1)) fail(PTSBE_ERR_INVALID, "channel strength must lie in [0, 1]");
    };
    cd P[4][4];
    for (int a = 0; a < 4; ++a) pauli(a, P[a]);
    bool pauli_mixture = false;
    switch (in.kind) {
    case PTSBE_CH_DEPOL1:
        need(1, 4);
        for (int a = 0; a < 4; ++a) {
            const double s = a == 0 ? std::sqrt(1 - p) : std::sqrt(p / 3);
            for (int i = 0; i < 4; ++i) c.K[a * 4 + i] = s * P[a][i];
            c.q[a] = a == 0 ? 1 - p : p / 3;
        }
        pauli_mixture = true;
        break;
    case PTSBE_CH_DEPOL2:
        need(2, 16);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const int k = 4 * a + b;
                const double s = k == 0 ? std::sqrt(1 - p) : std::sqrt(p / 15);
                for (int r = 0; r < 4; ++r)
                    for (int col = 0; col < 4; ++col)
                        c.K[k * 16 + r * 4 + col] = s * P[a][(r >> 1) * 2 + (col >> 1)] * P[b][(r & 1) * 2 + (col & 1)];
                c.q[k] = k == 0 ? 1 - p : p / 15;
            }
        pauli_mixture = true;
        break;
    case PTSBE_CH_AMPDAMP:
        need(1, 2);
        c.K[0] = 1; c.K[3] = std::sqrt(1 - p);
        c.K[5] = std::sqrt(p);
        c.q[0] = 1 - p / 2; c.q[1] = p / 2;
        break;
    case PTSBE_CH_BITFLIP:
    case PTSBE_CH_PHASEFLIP: {
        need(1, 2);
        const int e = in.kind == PTSBE_CH_BITFLIP ? 1 : 3;
        for (int i = 0; i < 4; ++i) { c.K[i] = std::sqrt(1 - p) * P[0][i]; c.K[4 + i] = std::sqrt(p) * P[e][i]; }
        c.q[0] = 1 - p; c.q[1] = p;
        pauli_mixture = true;
        break;
    }
    case PTSBE_CH_CUSTOM:
        if (!in.kraus) fail(PTSBE_ERR_INVALID, "CUSTOM channel needs Kraus matrices");
        for (uint32_t k = 0; k < c.nk; ++k) {
            double s = 0;
            for (uint32_t i = 0; i < dd; ++i) {
                const double re = in.kraus[2 * (k * dd + i)], im = in.kraus[2 * (k * dd + i) + 1];
                if (!std::isfinite(re) || !std::isfinite(im)) fail(PTSBE_ERR_INVALID, "non-finite Kraus entry");
                c.K[k * dd + i] = cd(re, im);
                s += re * re + im * im;
            }
            c.q[k] = s / d;
        }
        break;
    default:
        fail(PTSBE_ERR_INVALID, "unknown channel kind");
    }
    // CPTP: sum_k K_k^dag K_k = I
    double worst = 0;
    for (uint32_t r = 0; r < d; ++r)
        for (uint32_t col = 0; col < d; ++col) {
            cd s = 0;
            for (uint32_t k = 0; k < c.nk; ++k)
                for (uint32_t i = 0; i < d; ++i) s += std::conj(c.K[k * dd + i * d + r]) * c.K[k * dd + i * d + col];
            worst = std::max(worst, std::abs(s - (r == col ? 1.0 : 0.0)));
        }
    if (worst > 1e-10) fail(PTSBE_ERR_NOT_CPTP, "channel is not trace preserving (|sum K^dag K - I| = " + std::to_string(worst) + ")");
    // unitary mixture: K_k^dag K_k = q_k I
    c.mixture = true;
    for (uint32_t k = 0; k < c.nk && c.mixture; ++k)
        for (uint32_t r = 0; r < d; ++r)
            for (uint32_t col = 0; col < d; ++col) {
                cd s = 0;
                for (uint32_t i = 0; i < d; ++i) s += std::conj(c.K[k * dd + i * d + r]) * c.K[k * dd + i * d + col];
                if (std::abs(s - (r == col ? c.q[k] : 0.0)) > 1e-12) c.mixture = false;
            }
    if (c.mixture) {
        c.U.assign((size_t)c.nk * dd, 0.0);
        for (uint32_t k = 0; k < c.nk; ++k) {
            if (pauli_mixture) {
                // exact Pauli products
                if (c.arity == 1) {
                    int a = in.kind == PTSBE_CH_DEPOL1 ? (int)k : (k == 0 ? 0 : (in.kind == PTSBE_CH_BITFLIP ? 1 : 3));
                    for (int i = 0; i < 4; ++i) c.U[k * 4 + i] = P[a][i];
                } else {
                    const int a = (int)k / 4, b = (int)k % 4;
                    for (int r = 0; r < 4; ++r)
                        for (int col = 0; col < 4; ++col)
                            c.U[k * 16 + r * 4 + col] = P[a][(r >> 1) * 2 + (col >> 1)] * P[b][(r & 1) * 2 + (col & 1)];
                }
            } else if (c.q[k] > 0) {
                const double s = 1.0 / std::sqrt(c.q[k]);
                for (uint32_t i = 0; i < dd; ++i) c.U[k * dd + i] = c.K[k * dd + i] * s;
            }
        }
    }
}

void register_ops(Circuit& c, const ptsbe_op* ops, uint64_t n_ops, const double* custom, uint32_t n_custom) {
    const uint32_t n = c.n;
    c.ops.assign(ops, ops + n_ops);
    c.custom.assign(custom ? custom : nullptr, custom ? custom + 32 * (size_t)n_custom : nullptr);
    c.site_op.clear(); c.site_ch.clear();
    c.n_gates = 0;
    for (uint64_t i = 0; i < n_ops; ++i) {
        const ptsbe_op& o = ops[i];
        if (o.n_targets < 1 || o.n_targets > 2) fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": n_targets must be 1 or 2");
        if (o.targets[0] >= n || (o.n_targets == 2 && (o.targets[1] >= n || o.targets[1] == o.targets[0])))
            fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": bad target qubits");
        if (o.kind == PTSBE_OP_GATE) {
            if (o.id > PTSBE_G_U2 || gate_arity(o.id) != o.n_targets) fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": bad gate");
            if (o.id == PTSBE_G_U1 || o.id == PTSBE_G_U2) {
                const double r = o.params[0];
                if (!(r >= 0 && r < n_custom) || r != std::floor(r) || !custom) fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": bad custom gate row");
            }
            ++c.n_gates;
        } else if (o.kind == PTSBE_OP_NOISE) {
            if (o.id >= c.ch.size() || c.ch[o.id].arity != o.n_targets) fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": bad channel");
            c.site_op.push_back((uint32_t)i);
            c.site_ch.push_back(o.id);
        } else {
            fail(PTSBE_ERR_INVALID, "op " + std::to_string(i) + ": kind must be GATE or NOISE");
        }
    }
    if (c.site_op.size() >= (1ull << 32) || n_ops >= (1ull << 32)) fail(PTSBE_ERR_UNSUPPORTED, "too many ops");
    c.Q0 = 1.0;
    c.k0_strict_mode = true;
    for (uint32_t s : c.site_ch) {
        const HostChannel& ch = c.ch[s];
        c.Q0 *= ch.q[0];
        if (!(ch.q[0] > 0)) c.k0_strict_mode = false;
        for (uint32_t k = 1; k < ch.nk; ++k) if (!(ch.q[k] < ch.q[0])) c.k0_strict_mode = false;
    }
}

namespace {

uint32_t push_mat(Circuit& c, const cd* m, int count) {
    const uint32_t off = (uint32_t)c.dmats.size();
    for (int i = 0; i < count; ++i) c.dmats.push_back(make_float2((float)m[i].real(), (float)m[i].imag()));
    return off;
}

// Classifies a 2x2 operator (after rounding to complex64) into a micro-op.
DevMicro micro1(Circuit& c, const cd* m, uint8_t operand) {
    DevMicro u{};
    u.operand = operand;
    auto f0 = [](cd z) { return (float)z.real() == 0.0f && (float)z.imag() == 0.0f; };
    auto f1 = [](cd z) { return (float)z.real() == 1.0f && (float)z.imag() == 0.0f; };
    if (f0(m[1]) && f0(m[2])) {
        if (f1(m[0]) && f1(m[3])) { u.kind = DOP_NOP; return u; }
        cd d[2] = {m[0], m[3]};
        u.kind = DOP_D1; u.mat = push_mat(c, d, 2);
    } else if (f0(m[0]) && f0(m[3])) {
        cd d[2] = {m[1], m[2]};
        u.kind = DOP_X1; u.mat = push_mat(c, d, 2);
    } else {
        u.kind = DOP_G1; u.mat = push_mat(c, m, 4);
    }
    return u;
}

// Splits a 4x4 operator into a product of single-qubit factors when it is a Kronecker product
// A (x) B (true for the Pauli products of two-qubit depolarising noise); otherwise keeps G2.
bool kron_split(const cd* m, cd* A, cd* B) {
    // find the largest entry to anchor the factorisation
    int br = 0, bc = 0;
    double best = -1;
    for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 4; ++col)
            if (std::abs(m[r * 4 + col]) > best) { best = std::abs(m[r * 4 + col]); br = r; bc = col; }
    if (best <= 0) return false;
    const int ar = br >> 1, ac = bc >> 1, b_r = br & 1, b_c = bc & 1;
    // B = m[block (ar, ac)] / m[br][bc] * scale, A[i][j] = m[(i, b_r), (j, b_c)]
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            A[i * 2 + j] = m[(i * 2 + b_r) * 4 + (j * 2 + b_c)];
            B[i * 2 + j] = m[(ar * 2 + i) * 4 + (ac * 2 + j)] / m[br * 4 + bc];
        }
    for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 4; ++col) {
            const cd want = A[(r >> 1) * 2 + (col >> 1)] * B[(r & 1) * 2 + (col & 1)];
            if (std::abs(want - m[r * 4 + col]) > 1e-14) return false;
        }
    return true;
}

}  // namespace

void fuse_gates_with_noise(Circuit& c);

void build_device_ops(Circuit& c) {
    c.dops.clear(); c.dmicro.clear(); c.dmats.clear(); c.dchans.clear();
    // channels: micro ops of every Kraus operator
    for (const HostChannel& ch : c.ch) {
        DevChannel dc{};
        dc.nk = (uint8_t)ch.nk; dc.arity = (uint8_t)ch.arity; dc.mixture = ch.mixture ? 1 : 0;
        const uint32_t dd = ch.dim * ch.dim;
        for (uint32_t k = 0; k < ch.nk; ++k) {
            dc.micro_off[k] = (uint32_t)c.dmicro.size();
            dc.q[k] = ch.q[k];
            const cd* m = ch.mixture ? &ch.U[k * dd] : &ch.K[k * dd];
            if (ch.arity == 1) {
                DevMicro u = micro1(c, m, 0);
                if (u.kind != DOP_NOP) c.dmicro.push_back(u);
            } else {
                cd A[4], B[4];
                if (kron_split(m, A, B)) {
                    DevMicro ua = micro1(c, A, 0), ub = micro1(c, B, 1);
                    if (ua.kind != DOP_NOP) c.dmicro.push_back(ua);
                    if (ub.kind != DOP_NOP) c.dmicro.push_back(ub);
                } else {
                    DevMicro u{};
                    u.kind = DOP_G2; u.operand = 2; u.mat = push_mat(c, m, 16);
                    c.dmicro.push_back(u);
                }
            }
            // K_k^dag K_k for Algorithm 1 probabilities
            std::vector<cd> h(dd, 0.0);
            for (uint32_t r = 0; r < ch.dim; ++r)
                for (uint32_t col = 0; col < ch.dim; ++col)
                    for (uint32_t i = 0; i < ch.dim; ++i)
                        h[r * ch.dim + col] += std::conj(ch.K[k * dd + i * ch.dim + r]) * ch.K[k * dd + i * ch.dim + col];
            dc.herm_mat[k] = push_mat(c, h.data(), (int)dd);
        }
        dc.micro_off[ch.nk] = (uint32_t)c.dmicro.size();
        c.dchans.push_back(dc);
    }
    // ops
    for (size_t i = 0; i < c.ops.size(); ++i) {
        const ptsbe_op& o = c.ops[i];
        DevOp d{};
        d.fkind = DOP_NOP;
        d.q0 = (uint8_t)o.targets[0];
        d.q1 = (uint8_t)(o.n_targets == 2 ? o.targets[1] : o.targets[0]);
        d.nt = (uint8_t)o.n_targets;
        if (o.kind == PTSBE_OP_NOISE) {
            d.kind = DOP_NOISE; d.ch = o.id;
            d.site = (uint32_t)(std::lower_bound(c.site_op.begin(), c.site_op.end(), (uint32_t)i) - c.site_op.begin());
        } else if (o.id == PTSBE_G_CX) {
            d.kind = DOP_CX;
        } else if (o.id == PTSBE_G_CZ) {
            d.kind = DOP_CZ;
        } else if (o.id == PTSBE_G_SWAP) {
            d.kind = DOP_SWAP;
        } else {
            cd m[16];
            int dim;
            const double* custom = nullptr;
            if (o.id == PTSBE_G_U1 || o.id == PTSBE_G_U2) custom = c.custom.data() + 32 * (size_t)o.params[0];
            gate_matrix(o.id, o.params, custom, m, dim);
            if (dim == 2) {
                DevMicro u = micro1(c, m, 0);
                d.kind = u.kind; d.mat = u.mat;
            } else {
                d.kind = DOP_G2; d.mat = push_mat(c, m, 16);
            }
        }
        c.dops.push_back(d);
    }
    fuse_gates_with_noise(c);
}

// ---------------------------------------------------------------------------------------------
// Gate fusion: gate G followed by noise sites on (a subset of) its own qubits. For the "no error"
// branch every such site applies its Kraus operator 0 (U_0 for a unitary mixture), so the whole
// block is the single operator K0_m ... K0_1 G. Sets with an error among those sites fall back to
// applying the ops one by one, so the result is the same operator product either way.
// ---------------------------------------------------------------------------------------------
namespace {

// 4x4 operator of `m` (dim x dim on qubits qs) within the two-qubit space (q0, q1), local index
// 2*bit(q0) + bit(q1).
void embed2(const cd* m, int dim, const uint32_t* qs, uint32_t q0, uint32_t q1, cd* out) {
    for (int i = 0; i < 16; ++i) out[i] = 0;
    for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 4; ++col) {
            const int r0 = r >> 1, r1 = r & 1, c0 = col >> 1, c1 = col & 1;
            auto bit = [&](int b0, int b1, uint32_t q) { return q == q0 ? b0 : b1; };
            if (dim == 2) {
                const uint32_t q = qs[0];
                // identity on the other qubit
                const int other_same = (q == q0) ? (r1 == c1) : (r0 == c0);
                if (!other_same) continue;
                out[r * 4 + col] = m[bit(r0, r1, q) * 2 + bit(c0, c1, q)];
            } else {
                const int lr = bit(r0, r1, qs[0]) * 2 + bit(r0, r1, qs[1]);
                const int lc = bit(c0, c1, qs[0]) * 2 + bit(c0, c1, qs[1]);
                out[r * 4 + col] = m[lr * 4 + lc];
            }
        }
}

void matmul(const cd* A, const cd* B, cd* out, int d) {  // out = A B
    cd t[16];
    for (int r = 0; r < d; ++r)
        for (int col = 0; col < d; ++col) {
            cd s = 0;
            for (int k = 0; k < d; ++k) s += A[r * d + k] * B[k * d + col];
            t[r * d + col] = s;
        }
    for (int i = 0; i < d * d; ++i) out[i] = t[i];
}

bool is_identity(const cd* m, int d) {
    for (int r = 0; r < d; ++r)
        for (int col = 0; col < d; ++col)
            if (m[r * d + col] != (r == col ? cd(1.0) : cd(0.0))) return false;
    return true;
}

}  // namespace

void embed_pair(const cd* m, int dim, const uint32_t* qs, uint32_t q0, uint32_t q1, cd* out) {
    embed2(m, dim, qs, q0, q1, out);
}

// Linear part over GF(2) of a two-qubit permutation on x = 2 l_a + l_b, as the images of e_b and
// e_a packed in 4 bits; CX (control a) and SWAP have their own, every other gate the identity's.
uint32_t perm_linear(const int* perm) { return (uint32_t)((perm[1] ^ perm[0]) | ((perm[2] ^ perm[0]) << 2)); }
uint32_t gate_linear(uint8_t kind) {
    if (kind == DOP_CX) return 1u | (3u << 2);
    if (kind == DOP_SWAP) return 2u | (1u << 2);
    return 1u | (2u << 2);
}

void fuse_gates_with_noise(Circuit& c) {
    const size_t nops = c.ops.size();
    for (size_t i = 0; i < nops; ++i) {
        const ptsbe_op& g = c.ops[i];
        if (g.kind != PTSBE_OP_GATE) continue;
        size_t j = i + 1;
        while (j < nops && c.ops[j].kind == PTSBE_OP_NOISE) {
            const ptsbe_op& nz = c.ops[j];
            bool inside = true;
            for (uint32_t t = 0; t < nz.n_targets; ++t) {
                const uint32_t q = nz.targets[t];
                if (!(q == g.targets[0] || (g.n_targets == 2 && q == g.targets[1]))) inside = false;
            }
            if (!inside) break;
            ++j;
        }
        if (j == i + 1) continue;
        const int dim = g.n_targets == 2 ? 4 : 2;
        cd M[16];
        int gd;
        const double* custom = nullptr;
        if (g.id == PTSBE_G_U1 || g.id == PTSBE_G_U2) custom = c.custom.data() + 32 * (size_t)g.params[0];
        gate_matrix(g.id, g.params, custom, M, gd);
        bool any = false;
        for (size_t t = i + 1; t < j; ++t) {
            const ptsbe_op& nz = c.ops[t];
            const HostChannel& ch = c.ch[nz.id];
            const cd* K0 = ch.mixture ? &ch.U[0] : &ch.K[0];
            if (is_identity(K0, (int)ch.dim)) continue;
            any = true;
            if (dim == 2) {
                matmul(K0, M, M, 2);
            } else {
                cd E[16];
                embed2(K0, (int)ch.dim, nz.targets, g.targets[0], g.targets[1], E);
                matmul(E, M, M, 4);
            }
        }
        DevOp& d = c.dops[i];
        d.fend = (uint32_t)j;
        d.fsite1 = c.dops[j - 1].site + 1;
        if (!any) {              // only identity no-error operators: skip them in one step
            d.fkind = d.kind; d.fmat = d.mat; d.fperm = 0;
            continue;
        }
        if (dim == 2) {
            DevMicro u = micro1(c, M, 0);
            d.fkind = u.kind; d.fmat = u.mat;
        } else {
            // monomial? one nonzero per row and column
            int perm[4];
            bool mono = true;
            for (int r = 0; r < 4 && mono; ++r) {
                int nz = -1;
                for (int col = 0; col < 4; ++col)
                    if ((float)M[r * 4 + col].real() != 0.0f || (float)M[r * 4 + col].imag() != 0.0f) {
                        if (nz >= 0) mono = false;
                        nz = col;
                    }
                if (nz < 0) mono = false;
                perm[r] = nz;
            }
            if (mono && perm_linear(perm) != gate_linear(c.dops[i].kind)) mono = false;   // keeps the frame set-independent
            if (mono) {
                cd dv[8];
                uint8_t packed = 0;
                for (int r = 0; r < 4; ++r) { dv[r] = M[r * 4 + perm[r]]; packed |= (uint8_t)(perm[r] << (2 * r)); }
                // separable diagonal d[2 l_a + l_b] = alpha[l_a] beta[l_b] (damping on both qubits)
                d.fsep = 0;
                if (std::abs(dv[0]) > 0) {
                    dv[4] = dv[0]; dv[5] = dv[2]; dv[6] = 1.0; dv[7] = dv[1] / dv[0];
                    if (std::abs(dv[5] * dv[7] - dv[3]) <= 1e-12 * std::abs(dv[0])) d.fsep = 1;
                }
                d.fkind = DOP_M2; d.fmat = push_mat(c, dv, d.fsep ? 8 : 4); d.fperm = packed;
            } else {
                d.fkind = DOP_G2; d.fmat = push_mat(c, M, 16);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------------------------
namespace {

uint64_t op_mask(const Circuit& c, size_t i) {
    const ptsbe_op& o = c.ops[i];
    uint64_t m = 1ull << o.targets[0];
    if (o.n_targets == 2) m |= 1ull << o.targets[1];
    return m;
}

bool general_noise(const Circuit& c, size_t i) {
    const ptsbe_op& o = c.ops[i];
    return o.kind == PTSBE_OP_NOISE && !c.ch[o.id].mixture;
}

uint32_t tile_mask(const Circuit& c, const DevStage& st, size_t i) {
    const ptsbe_op& o = c.ops[i];
    uint32_t m = 1u << st.pos[o.targets[0]];
    if (o.n_targets == 2) m |= 1u << st.pos[o.targets[1]];
    return m;
}

void emit_group(Plan& P, uint32_t b, uint32_t e, const std::vector<int>& used) {
    DevGroup g{};
    g.op_begin = b; g.op_end = e;
    std::memset(g.rbit, 0xFF, sizeof(g.rbit));
    std::memset(g.lane_pos, 0xFF, sizeof(g.lane_pos));
    int nb = 0;
    uint32_t taken = 0;
    for (int p : used) { g.reg_pos[nb] = (uint8_t)p; g.rbit[p] = (uint8_t)nb; taken |= 1u << p; ++nb; }
    // fill with the highest free positions so the lanes keep the low (contiguous) ones
    for (int p = P.tb - 1; p >= 0 && nb < kRegBits; --p)
        if (!(taken & (1u << p))) { g.reg_pos[nb] = (uint8_t)p; g.rbit[p] = (uint8_t)nb; taken |= 1u << p; ++nb; }
    // Lane positions: the first five (the lane id bits of a warp) get distinct residues mod 5, so
    // the kernel's XOR swizzle of shared memory (bits 5..9 and 10..14 folded onto bits 0..4) puts a
    // warp's 32 slots on 32 distinct banks; the rest follow in ascending order.
    int nl = 0;
    uint32_t lanes = 0, residues = 0;
    for (int p = 0; p < P.tb && nl < 5; ++p)
        if (!(taken & (1u << p)) && !(residues & (1u << (p % 5)))) {
            g.lane_pos[nl++] = (uint8_t)p; lanes |= 1u << p; residues |= 1u << (p % 5);
        }
    for (int p = 0; p < P.tb; ++p)
        if (!(taken & (1u << p)) && !(lanes & (1u << p))) g.lane_pos[nl++] = (uint8_t)p;
    P.groups.push_back(g);
}

// Splits the ops of a stage into register groups of at most kRegBits tile positions each.
void plan_groups(Plan& P, const Circuit& c, DevStage& st) {
    st.group_begin = st.group_end = (uint32_t)P.groups.size();
    if (P.tb < kRegBits || st.op_end == st.op_begin) return;
    uint32_t cur = 0, gb = st.op_begin;
    std::vector<int> used;
    for (uint32_t i = st.op_begin; i < st.op_end; ++i) {
        const uint32_t m = tile_mask(c, st, i);
        if (__builtin_popcount(cur | m) > kRegBits) {
            emit_group(P, gb, i, used);
            cur = 0; used.clear(); gb = i;
        }
        for (int p = 0; p < P.tb; ++p)
            if ((m & (1u << p)) && !(cur & (1u << p))) used.push_back(p);
        cur |= m;
    }
    emit_group(P, gb, st.op_end, used);
    st.group_end = (uint32_t)P.groups.size();
}

void close_stage(Plan& P, const Circuit& c, uint64_t Q, uint32_t b, uint32_t e, bool probe, uint32_t probe_op,
                 bool groups = true) {
    const int n = (int)c.n, tb = P.tb, lb = P.lb;
    // fill the qubit set up to tb with the lowest unused qubits
    for (int q = 0; q < n && __builtin_popcountll(Q) < tb; ++q) Q |= 1ull << q;
    DevStage st{};
    st.op_begin = b; st.op_end = e;
    st.flags = probe ? 1u : 0u;
    st.probe_op = probe_op;
    std::memset(st.pos, 0xFF, sizeof(st.pos));
    std::memset(st.outer_q, 0xFF, sizeof(st.outer_q));
    int tq[kMaxQubits];
    int t = 0;
    for (int q = 0; q < lb; ++q) tq[t++] = q;
    for (int q = lb; q < n; ++q) if (Q & (1ull << q)) tq[t++] = q;
    int ob = 0;
    for (int q = 0; q < n; ++q)
        if (!(Q & (1ull << q))) { st.pos[q] = (uint8_t)(0x80 | ob); st.outer_q[ob++] = (uint8_t)q; }
    for (int i = 0; i < tb; ++i) st.pos[tq[i]] = (uint8_t)i;
    st.hi_off = (uint32_t)P.hi.size();
    for (uint32_t h = 0; h < (1u << (tb - lb)); ++h) {
        uint32_t g = 0;
        for (int bit = 0; bit < tb - lb; ++bit) if (h & (1u << bit)) g |= 1u << tq[lb + bit];
        P.hi.push_back(g);
    }
    for (uint32_t i = b; i < e; ++i) P.op_stage[i] = (int32_t)P.stages.size();
    if (groups) plan_groups(P, c, st);
    else st.group_begin = st.group_end = (uint32_t)P.groups.size();
    P.stages.push_back(st);
}

}  // namespace

Plan make_plan(const Circuit& c, int tile_bits, bool pershot) {
    Plan P;
    const int n = (int)c.n;
    P.tb = std::min(n, tile_bits);
    P.lb = std::min(P.tb, kLowBits);
    const size_t nops = c.ops.size();
    P.op_stage.assign(nops, 0);
    const uint64_t low = (P.lb >= 64) ? ~0ull : ((1ull << P.lb) - 1);
    if (n <= tile_bits) {
        close_stage(P, c, (n >= 64 ? ~0ull : ((1ull << n) - 1)), 0, (uint32_t)nops, false, 0);
        return P;
    }
    if (P.tb < P.lb + 4) fail(PTSBE_ERR_UNSUPPORTED, "tile too small for the planner");
    uint64_t Q = low;
    uint32_t begin = 0;
    for (size_t i = 0; i < nops; ++i) {
        if (pershot && general_noise(c, i)) {
            // Algorithm 1: the branch probabilities of this site are accumulated by the epilogue
            // of the stage that ends here, so the site's qubits belong to that stage.
            const uint64_t need = Q | op_mask(c, i);
            if (__builtin_popcountll(need) > P.tb) fail(PTSBE_ERR_UNSUPPORTED, "planner invariant violated");
            close_stage(P, c, need, begin, (uint32_t)i, true, (uint32_t)i);
            begin = (uint32_t)i;
            Q = low | op_mask(c, i);
            if (i + 1 < nops && general_noise(c, i + 1)) Q |= op_mask(c, i + 1);
            continue;
        }
        uint64_t need = Q | op_mask(c, i);
        if (pershot && i + 1 < nops && general_noise(c, i + 1)) need |= op_mask(c, i + 1);
        if (__builtin_popcountll(need) > P.tb) {
            close_stage(P, c, Q, begin, (uint32_t)i, false, 0);
            begin = (uint32_t)i;
            need = low | op_mask(c, i);
            if (pershot && i + 1 < nops && general_noise(c, i + 1)) need |= op_mask(c, i + 1);
        }
        Q = need;
    }
    close_stage(P, c, Q, begin, (uint32_t)nops, false, 0);
    return P;
}

// ---------------------------------------------------------------------------------------------
// Deferred-frame plan. The permutation part of the frame (columns A) changes only at CX and SWAP
// gates (fused blocks keep the gate's permutation part, see fuse_gates_with_noise), so it is the
// same for every Kraus set and the host can follow it. A stage needs the global directions of
// the operators that may mix amplitudes inside its tile; everything else is bookkeeping.
// ---------------------------------------------------------------------------------------------
namespace {

bool mixing_kind(uint8_t k) { return k == DOP_G1 || k == DOP_G2; }

bool perm_bijective(uint32_t perm) {
    uint32_t seen = 0;
    for (int x = 0; x < 4; ++x) seen |= 1u << ((perm >> (2 * x)) & 3u);
    return seen == 15u;
}

// Global directions op i may mix along (0 if it never mixes), for the current columns.
uint32_t frame_dirs(const Circuit& c, size_t i, const uint32_t* col) {
    const DevOp& o = c.dops[i];
    uint32_t d = 0;
    if (o.kind == DOP_NOISE) {
        const DevChannel& ch = c.dchans[o.ch];
        for (uint32_t u = ch.micro_off[0]; u < ch.micro_off[ch.nk]; ++u) {
            const DevMicro& mi = c.dmicro[u];
            if (!mixing_kind(mi.kind)) continue;
            if (mi.operand != 1) d |= col[o.q0];
            if (mi.operand != 0) d |= col[o.q1];
        }
        return d;
    }
    bool mix = mixing_kind(o.kind);
    if (o.fend != 0 && (mixing_kind(o.fkind) || (o.fkind == DOP_M2 && !perm_bijective(o.fperm)))) mix = true;
    if (!mix) return 0;
    d = col[o.q0];
    if (o.nt == 2) d |= col[o.q1];
    return d;
}

// The individual global directions op i may mix along (one per mixing target), for the current
// columns; the span of these vectors bounds the support of a state that starts from |0...0>.
int frame_dir_vectors(const Circuit& c, size_t i, const uint32_t* col, uint32_t* out) {
    const DevOp& o = c.dops[i];
    int k = 0;
    if (o.kind == DOP_NOISE) {
        const DevChannel& ch = c.dchans[o.ch];
        bool m0 = false, m1 = false;
        for (uint32_t u = ch.micro_off[0]; u < ch.micro_off[ch.nk]; ++u) {
            const DevMicro& mi = c.dmicro[u];
            if (!mixing_kind(mi.kind)) continue;
            if (mi.operand != 1) m0 = true;
            if (mi.operand != 0) m1 = true;
        }
        if (m0) out[k++] = col[o.q0];
        if (m1) out[k++] = col[o.q1];
        return k;
    }
    if (!frame_dirs(c, i, col)) return 0;
    out[k++] = col[o.q0];
    if (o.nt == 2) out[k++] = col[o.q1];
    return k;
}

void frame_linear(const Circuit& c, size_t i, uint32_t* col) {
    const DevOp& o = c.dops[i];
    if (o.kind == DOP_CX) col[o.q0] ^= col[o.q1];
    else if (o.kind == DOP_SWAP) std::swap(col[o.q0], col[o.q1]);
}

// Rows of A^-1 for the columns of A (n x n over GF(2), Gauss-Jordan).
void invert_cols(int n, const uint32_t* col, uint32_t* row) {
    uint32_t M[kMaxQubits], I[kMaxQubits];     // row x of A (bit q = bit x of col[q]), identity
    for (int x = 0; x < n; ++x) {
        M[x] = 0;
        for (int q = 0; q < n; ++q) if ((col[q] >> x) & 1u) M[x] |= 1u << q;
        I[x] = 1u << x;
    }
    for (int q = 0; q < n; ++q) {
        int piv = -1;
        for (int x = q; x < n; ++x) if ((M[x] >> q) & 1u) { piv = x; break; }
        if (piv < 0) fail(PTSBE_ERR_INVALID, "frame plan: singular permutation");
        std::swap(M[q], M[piv]); std::swap(I[q], I[piv]);
        for (int x = 0; x < n; ++x)
            if (x != q && ((M[x] >> q) & 1u)) { M[x] ^= M[q]; I[x] ^= I[q]; }
    }
    for (int q = 0; q < n; ++q) row[q] = I[q];   // row q of A^-1 as a mask over global bits
}

void close_frame_stage(Plan& P, const Circuit& c, uint32_t T, uint32_t b, uint32_t e, const uint32_t* entry,
                       bool last, int lbf) {
    const int n = (int)c.n;
    close_stage(P, c, T, b, e, false, 0, false);
    const DevStage& st = P.stages.back();
    DevFrameStage f{};
    for (int q = 0; q < n; ++q) f.col[q] = entry[q];
    invert_cols(n, f.col, f.row);
    f.last = last ? 1u : 0u;
    f.lbf = (uint32_t)lbf;
    if (last) {
        uint32_t col[kMaxQubits], row[kMaxQubits];
        for (int q = 0; q < n; ++q) col[q] = entry[q];
        for (uint32_t i = b; i < e; ++i) frame_linear(c, i, col);
        invert_cols(n, col, row);
        auto logical_of = [&](int x) {          // R e_x
            uint32_t v = 0;
            for (int q = 0; q < n; ++q) if ((row[q] >> x) & 1u) v |= 1u << q;
            return v;
        };
        // basis of R(span T): e_0 .. e_{lbf-1} first, then R e_x for tile bits x
        uint32_t ech[kMaxQubits];
        int piv[kMaxQubits], d = 0;
        auto try_add = [&](uint32_t v) {
            uint32_t x = v;
            for (int i = 0; i < d; ++i) if ((x >> piv[i]) & 1u) x ^= ech[i];
            if (!x) return false;
            ech[d] = x; piv[d] = 31 - __builtin_clz(x); f.w[d] = v; ++d;
            return true;
        };
        for (int k = 0; k < lbf; ++k)
            if (!try_add(1u << k)) fail(PTSBE_ERR_INVALID, "frame plan: output bits outside the last tile");
        if (lbf == 0) { P.fstages.push_back(f); return; }   // sparse final: no dense output map
        for (int t = 0; t < P.tb && d < P.tb; ++t) {
            int x = -1;
            for (int g = 0; g < n; ++g) if (st.pos[g] == t) x = g;
            try_add(logical_of(x));
        }
        if (d != P.tb) fail(PTSBE_ERR_INVALID, "frame plan: incomplete output basis");
        for (int k = 0; k < P.tb; ++k) {
            uint32_t g = 0;   // A w_k (global), then its tile-local address
            for (int q = 0; q < n; ++q) if ((f.w[k] >> q) & 1u) g ^= col[q];
            uint32_t m = 0;
            for (int x = 0; x < n; ++x)
                if ((g >> x) & 1u) {
                    if (st.pos[x] & 0x80) fail(PTSBE_ERR_INVALID, "frame plan: output basis leaves the tile");
                    m |= 1u << st.pos[x];
                }
            f.m[k] = (uint16_t)m;
        }
        for (int i = 0; i < n - P.tb; ++i) f.ox[i] = logical_of(st.outer_q[i]);
    }
    P.fstages.push_back(f);
}

}  // namespace

namespace {

// The frame plan with the first stage entered in layout entry0 (columns: global image of each
// logical bit); later stages after a logical-order store restart at the identity.
Plan frame_plan_from(const Circuit& c, int tile_bits, const uint32_t* entry0) {
    Plan P;
    const int n = (int)c.n;
    if (n > 32) fail(PTSBE_ERR_UNSUPPORTED, "more than 32 qubits");
    P.tb = std::min(n, tile_bits);
    P.lb = std::min(P.tb, kLowBits);
    const size_t nops = c.ops.size();
    P.op_stage.assign(nops, 0);
    uint32_t col[kMaxQubits], entry[kMaxQubits];
    for (int q = 0; q < n; ++q) col[q] = entry[q] = entry0[q];
    const uint32_t all = n == 32 ? ~0u : ((1u << n) - 1u);
    if (n <= tile_bits) {
        close_frame_stage(P, c, all, 0, (uint32_t)nops, entry, true, P.lb);
        return P;
    }
    const uint32_t low = (1u << P.lb) - 1u;
    uint32_t U = low, begin = 0;
    // Ends the stage [begin, e) with a store in logical order (the tile then also holds the images
    // of the low logical bits, else one more op-free stage does that store); the frame restarts
    // at the identity.
    auto close_logical = [&](uint32_t e) {
        uint32_t F = 0;
        for (int k = 0; k < P.lb; ++k) F |= col[k];
        if (e == nops && begin == 0 && P.stages.empty()) {
            // the whole circuit in one stage from |0...0>: the final store scatters from the one
            // nonzero tile (no tile constraint on the output bits)
            close_frame_stage(P, c, U, begin, e, entry, true, 0);
            DevFrameStage& f = P.fstages.back();
            f.sparse_final = 1;
            invert_cols(n, col, f.rowe);
            for (int q = 0; q < n; ++q) col[q] = entry[q] = 1u << q;
            return;
        }
        if (__builtin_popcount(U | F) <= P.tb) {
            close_frame_stage(P, c, U | F, begin, e, entry, true, P.lb);
        } else {
            close_frame_stage(P, c, U, begin, e, entry, false, 0);
            int lbf = P.lb;
            while (lbf > 1) {
                uint32_t G = 0;
                for (int k = 0; k < lbf; ++k) G |= col[k];
                if (__builtin_popcount(low | G) <= P.tb) break;
                --lbf;
            }
            uint32_t G = 0;
            for (int k = 0; k < lbf; ++k) G |= col[k];
            if (__builtin_popcount(low | G) > P.tb) fail(PTSBE_ERR_UNSUPPORTED, "frame plan: output bit wider than a tile");
            close_frame_stage(P, c, low | G, e, e, col, true, lbf);
        }
        for (int q = 0; q < n; ++q) col[q] = entry[q] = 1u << q;
    };
    for (size_t i = 0; i < nops; ++i) {
        uint32_t d = frame_dirs(c, i, col);
        if (__builtin_popcount(U | d) > P.tb) {
            if (__builtin_popcount(low | d) > P.tb) {
                // the permutation spread this operator's directions wider than a tile: go back
                // to logical order (directions are single bits again)
                close_logical((uint32_t)i);
                d = frame_dirs(c, i, col);
            } else {
                close_frame_stage(P, c, U, begin, (uint32_t)i, entry, false, 0);
                for (int q = 0; q < n; ++q) entry[q] = col[q];
            }
            begin = (uint32_t)i;
            U = low | d;
        } else {
            U |= d;
        }
        frame_linear(c, i, col);
    }
    close_logical((uint32_t)nops);
    return P;
}

}  // namespace

Plan make_frame_plan(const Circuit& c, int tile_bits) {
    const int n = (int)c.n;
    uint32_t id[kMaxQubits];
    for (int q = 0; q < kMaxQubits; ++q) id[q] = q < 32 ? 1u << q : 0u;
    Plan P = frame_plan_from(c, tile_bits, id);
    if (!(P.stages.size() == 1 && P.fstages[0].sparse_final)) return P;
    // One stage from |0...0>: the stored amplitudes only ever move along the mixing directions,
    // so they stay in the span V of those vectors. Entering the stage in a layout T with
    // T V = span(e_0 .. e_{D-1}) puts every nonzero amplitude at a tile address below 2^D, which
    // lets the kernel hold the support in a small buffer.
    uint32_t col[kMaxQubits], ech[kMaxQubits], dv[4];
    int piv[kMaxQubits], D = 0;
    for (int q = 0; q < n; ++q) col[q] = 1u << q;
    for (size_t i = 0; i < c.ops.size(); ++i) {
        const int k = frame_dir_vectors(c, i, col, dv);
        for (int j = 0; j < k; ++j) {
            uint32_t x = dv[j];
            for (int t = 0; t < D; ++t) if ((x >> piv[t]) & 1u) x ^= ech[t];
            if (!x) continue;
            if (D == kMaxQubits) break;
            ech[D] = x; piv[D] = __builtin_ctz(x); ++D;
        }
        frame_linear(c, i, col);
    }
    if (D > kSmallSupportBits) return P;
    // columns of V: the echelon vectors, then the unit vectors of the non-pivot bits; T = V^-1
    uint32_t V[kMaxQubits], R[kMaxQubits], T[kMaxQubits];
    uint32_t used = 0;
    for (int t = 0; t < D; ++t) { V[t] = ech[t]; used |= 1u << piv[t]; }
    int m = D;
    for (int x = 0; x < n; ++x) if (!((used >> x) & 1u)) V[m++] = 1u << x;
    invert_cols(n, V, R);                                  // rows of V^-1
    for (int q = 0; q < n; ++q) {                          // column q of V^-1
        uint32_t v = 0;
        for (int x = 0; x < n; ++x) if ((R[x] >> q) & 1u) v |= 1u << x;
        T[q] = v;
    }
    for (int q = n; q < kMaxQubits; ++q) T[q] = 0;
    Plan Q = frame_plan_from(c, tile_bits, T);
    if (!(Q.stages.size() == 1 && Q.fstages[0].sparse_final)) return P;
    Q.fstages[0].sbits = (uint32_t)std::max(D, 1);
    return Q;
}

}  // namespace ptsbe
