// Adjoint backward of the fixed-set estimator L = (1/N) sum_a mult_a <psi~_a|O|psi~_a> / q_a.
//
// For a set a, phi_T = B_T ... B_1 |0...0> (B_t the fused blocks with the set's Kraus variants,
// unitary-mixture variants applied as U_k with the scale s^2 = prod q_k kept on the host) and
// f = s^2 <phi_T|O|phi_T>. With mu_T = O phi_T and mu_{t-1} = B_t^dag mu_t, a parameter theta of
// block t contributes df/dtheta = 2 s^2 Re sum_{rc} G_t[r][c] (dB_t/dtheta)[r][c], where
// G_t[r][c] = sum over the other qubits of conj(mu_t[r]) phi_{t-1}[c] (the block's outer product).
//
// One thread-block cluster per set (persistent: cluster `slot` takes sets slot, slot + nslots, ...).
// phi and mu of the set live in the cluster's shared memory; the plan's swap steps exchange bit
// positions between CTAs through distributed shared memory so every block acts on local bits.
// Forward: apply each block to phi, storing phi first when the block cannot be inverted (or every
// ckpt_every blocks). Backward: walk the blocks in reverse, un-computing phi with B^-1 (or reloading
// the stored copy), accumulating G_t and updating mu, in one shared-memory pass per block.
// Blocks without a Kraus entry of the set share their derivative matrices across sets, so their
// G_t are summed with the set weights into per-slot accumulators and contracted once at the end;
// blocks that hold an entry of the set are contracted right away with that set's variants.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace ptsbe {
namespace {

constexpr int kBwThreads = 256;       // 8 warps of up to 255 registers: 4x4 blocks, inverses and outer products in registers
constexpr int kBwWarps = kBwThreads / 32;
constexpr int kSwapPer = ((1 << (kBwLocalBits - 1)) + kBwThreads - 1) / kBwThreads;   // half a slice per thread
constexpr int kFinThreads = 256;      // the finishing kernel
constexpr int kFinWarps = kFinThreads / 32;

struct ErrEnt {
    uint32_t item, member, k;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {    // a b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cjfma(float2 a, float2 b, float2 c) {   // conj(a) b + c
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ uint32_t ins0(uint32_t i, int p) { return ((i >> p) << (p + 1)) | (i & ((1u << p) - 1u)); }

// ---- block passes -------------------------------------------------------------------------------
// Index of the 2^nq amplitudes of coset i: matrix index 2 bit(p0) + bit(p1) (two qubits), bit(p0) (one).
template <int D>
__device__ __forceinline__ void coset(uint32_t i, int p0, int p1, uint32_t (&l)[D]) {
    if constexpr (D == 2) {
        l[0] = ins0(i, p0);
        l[1] = l[0] | (1u << p0);
    } else {
        const int lo = p0 < p1 ? p0 : p1, hi = p0 < p1 ? p1 : p0;
        const uint32_t b = ins0(ins0(i, lo), hi);
        l[0] = b; l[1] = b | (1u << p1); l[2] = b | (1u << p0); l[3] = b | (1u << p0) | (1u << p1);
    }
}

template <int D>
__device__ void fwd_pass(float2* v, int nl, int p0, int p1, const float2* M) {
    float2 m[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) m[i] = M[i];
    const uint32_t cnt = 1u << (nl - (D == 2 ? 1 : 2));
    for (uint32_t i = threadIdx.x; i < cnt; i += kBwThreads) {
        uint32_t l[D];
        coset<D>(i, p0, p1, l);
        float2 x[D];
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = v[l[c]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float2 y = cmul(m[r * D], x[0]);
#pragma unroll
            for (int c = 1; c < D; ++c) y = cfma(m[r * D + c], x[c], y);
            v[l[r]] = y;
        }
    }
}

// phi <- B^-1 phi (or the stored copy ck), G += conj(mu) (x) phi, mu <- B^dag mu.
template <int D, bool DIFF>
__device__ void bwd_pass(float2* phi, float2* mu, int nl, int p0, int p1, const float2* Bm, const float2* Bim,
                         const float2* ck, float (&g)[2 * D * D]) {
    float2 b[D * D], bi[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) { b[i] = Bm[i]; bi[i] = ck ? make_float2(0.f, 0.f) : Bim[i]; }
    const uint32_t cnt = 1u << (nl - (D == 2 ? 1 : 2));
    for (uint32_t i = threadIdx.x; i < cnt; i += kBwThreads) {
        uint32_t l[D];
        coset<D>(i, p0, p1, l);
        float2 x[D], y[D], xp[D];
#pragma unroll
        for (int c = 0; c < D; ++c) { x[c] = phi[l[c]]; y[c] = mu[l[c]]; }
        if (ck) {
#pragma unroll
            for (int c = 0; c < D; ++c) xp[c] = ck[l[c]];
        } else {
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float2 s = cmul(bi[r * D], x[0]);
#pragma unroll
                for (int c = 1; c < D; ++c) s = cfma(bi[r * D + c], x[c], s);
                xp[r] = s;
            }
        }
        if constexpr (DIFF) {
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float2 t = cjfma(y[r], xp[c], make_float2(g[2 * (r * D + c)], g[2 * (r * D + c) + 1]));
                    g[2 * (r * D + c)] = t.x; g[2 * (r * D + c) + 1] = t.y;
                }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < D; ++r) s = cjfma(b[r * D + c], y[r], s);
            phi[l[c]] = xp[c];
            mu[l[c]] = s;
        }
    }
}

// Sums each of the K values over the warp; lane l ends with the total of value l >> (5 - log2 K).
template <int K>
__device__ __forceinline__ float warp_vec_sum(float (&v)[K], int lane) {
    int len = K;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (len > 1) {
            const bool up = (lane & o) != 0;
            const int h = len >> 1;
#pragma unroll
            for (int j = 0; j < K / 2; ++j)
                if (j < h) {
                    const float send = up ? v[j] : v[j + h];
                    const float keep = up ? v[j + h] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
                }
            len = h;
        } else {
            v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], o);
        }
    }
    return v[0];
}

// Exchanges local position pa with rank position pg (bit pg - nl of the CTA rank) for phi (and mu).
template <int CL>
__device__ void swap_positions(float2* phi, float2* mu, int nl, int pa, int pg, int rank) {
    if constexpr (CL > 1) {
        cg::cluster_group cl = cg::this_cluster();
        const int gb = pg - nl;
        const uint32_t rb = (uint32_t)(rank >> gb) & 1u;
        const int partner = rank ^ (1 << gb);
        const float2* rphi = cl.map_shared_rank(phi, partner);
        const float2* rmu = mu ? cl.map_shared_rank(mu, partner) : nullptr;
        const uint32_t half = 1u << (nl - 1);
        float2 bp[kSwapPer], bm[kSwapPer];
        // own amplitudes whose bit pa differs from the rank bit receive the partner's amplitude at
        // the index with bit pa flipped (the two positions exchange their bits)
#pragma unroll
        for (int c = 0; c < kSwapPer; ++c) {
            const uint32_t i = threadIdx.x + (uint32_t)c * kBwThreads;
            if (i < half) {
                const uint32_t l = ins0(i, pa) | ((1u - rb) << pa);
                bp[c] = rphi[l ^ (1u << pa)];
                if (mu) bm[c] = rmu[l ^ (1u << pa)];
            }
        }
        cl.sync();
#pragma unroll
        for (int c = 0; c < kSwapPer; ++c) {
            const uint32_t i = threadIdx.x + (uint32_t)c * kBwThreads;
            if (i < half) {
                const uint32_t l = ins0(i, pa) | ((1u - rb) << pa);
                phi[l] = bp[c];
                if (mu) mu[l] = bm[c];
            }
        }
        cl.sync();
    }
}

// Product of an item's member variants (k from the set's entries ents[0..ne), sorted by member;
// other members variant 0) and of their inverses in reverse order, by lanes 0 .. d^2 - 1 of one
// warp, into shared Bs / Bis. *sing: some chosen variant cannot be inverted.
__device__ void build_item(const BwArgs& a, const BwItem& it, const ErrEnt* ents, int ne, float2* Bs, float2* Bis,
                           int* sing, int lane) {
    const int d = it.nq == 2 ? 4 : 2, dd = d * d;
    const int e = lane & (dd - 1), r = e / d, c = e % d;
    const bool act = lane < dd;
    if (act) { Bs[e] = make_float2(r == c ? 1.f : 0.f, 0.f); Bis[e] = Bs[e]; }
    int s = 0, p = 0;
    for (uint32_t m = it.mbeg; m < it.mend; ++m) {
        uint32_t k = 0;
        if (p < ne && ents[p].member == m) k = ents[p++].k;
        const BwMember M = a.members[m];
        s |= (int)((M.sing >> k) & 1u);
        const float2* A = a.pool + (size_t)(M.mat + k) * 16;
        const float2* Ai = a.pool + (size_t)(M.inv + k) * 16;
        __syncwarp();
        float2 nb = make_float2(0.f, 0.f), ni = make_float2(0.f, 0.f);
        for (int t = 0; t < d; ++t) {
            nb = cfma(A[r * d + t], Bs[t * d + c], nb);
            ni = cfma(Bis[r * d + t], Ai[t * d + c], ni);
        }
        __syncwarp();
        if (act) { Bs[e] = nb; Bis[e] = ni; }
    }
    __syncwarp();
    if (lane == 0) *sing = s;
}

// FP64 contraction of one item by one warp: for every differentiable member j (variants from
// ents, sorted by member), val = 2 Re sum_{uv} D[u][v] H_j[u][v] with H_j = S_j^T G P_j^T,
// P_j = A_{j-1} ... A_0, S_j = A_{M-1} ... A_{j+1}; out[dslot] += w val. G: 32 doubles (re, im).
// sc: 4 x 16 double2 of shared scratch.
__device__ void contract_item(const BwArgs& a, const BwItem& it, const ErrEnt* ents, int ne, const double* G, double w,
                              double* out, double2* sc, int lane) {
    const int d = it.nq == 2 ? 4 : 2, dd = d * d;
    const int e = lane & (dd - 1), r = e / d, c = e % d;
    const bool act = lane < dd;
    double2* Y = sc;
    double2* Pm = sc + 16;
    const int M = (int)(it.mend - it.mbeg);
    auto A64 = [&](uint32_t blk, int i) { const double* q = a.pool64 + (size_t)blk * 32 + 2 * i; return make_double2(q[0], q[1]); };
    auto variant = [&](uint32_t m) {
        for (int t = 0; t < ne; ++t)
            if (ents[t].member == m) return ents[t].k;
        return 0u;
    };
    if (act) Y[e] = make_double2(G[2 * e], G[2 * e + 1]);
    __syncwarp();
    for (int j = M - 1; j >= 0; --j) {
        const uint32_t m = it.mbeg + (uint32_t)j;
        const BwMember Mb = a.members[m];
        const uint32_t k = variant(m);
        if (Mb.nd) {
            if (act) Pm[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
            __syncwarp();
            for (int i = 0; i < j; ++i) {
                const uint32_t mi = it.mbeg + (uint32_t)i;
                const BwMember Mi = a.members[mi];
                const uint32_t blk = Mi.m64 + variant(mi);
                double2 s = make_double2(0.0, 0.0);
                for (int t = 0; t < d; ++t) {
                    const double2 x = A64(blk, r * d + t), y = Pm[t * d + c];
                    s.x += x.x * y.x - x.y * y.y; s.y += x.x * y.y + x.y * y.x;
                }
                __syncwarp();
                if (act) Pm[e] = s;
                __syncwarp();
            }
            // H[r][c] = sum_t Y[r][t] P[c][t]
            double2 h = make_double2(0.0, 0.0);
            for (int t = 0; t < d; ++t) {
                const double2 x = Y[r * d + t], y = Pm[c * d + t];
                h.x += x.x * y.x - x.y * y.y; h.y += x.x * y.y + x.y * y.x;
            }
            const int nder = Mb.noise ? 1 : Mb.nd;
            for (int jj = 0; jj < nder; ++jj) {
                const uint32_t dblk = Mb.d64 + (Mb.noise ? k : (uint32_t)jj);
                const double2 D = A64(dblk, e);
                double v = act ? 2.0 * (D.x * h.x - D.y * h.y) : 0.0;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                if (lane == 0) out[Mb.dslot + jj] += w * v;
            }
            __syncwarp();
        }
        // Y <- A_j^T Y
        const uint32_t blk = Mb.m64 + k;
        double2 s = make_double2(0.0, 0.0);
        for (int t = 0; t < d; ++t) {
            const double2 x = A64(blk, t * d + r), y = Y[t * d + c];
            s.x += x.x * y.x - x.y * y.y; s.y += x.x * y.y + x.y * y.x;
        }
        __syncwarp();
        if (act) Y[e] = s;
        __syncwarp();
    }
}

template <int CL>
__global__ void __launch_bounds__(kBwThreads, 1) k_backward(BwArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ float red[2][kBwWarps][32];
    __shared__ float2 Bs[16], Bis[16];
    __shared__ ErrEnt errs[kBwMaxErr];
    __shared__ uint32_t egs[kBwMaxErr];     // gslots of the set's differentiable error items
    __shared__ int s_nerr, s_negs, s_sing;
    __shared__ double s_part[kBwWarps];
    __shared__ double s_E;
    __shared__ double2 s_sc[32];
    __shared__ double s_G[32];
    const int nl = a.nl;
    const uint32_t L = 1u << nl;
    float2* phi = sm;
    float2* mu = sm + L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
    const uint32_t slot = blockIdx.x / CL;
    const size_t slice = (size_t)rank << nl;
    for (uint32_t al = slot; al < a.count; al += a.nslots) {
        if (tid == 0) {
            const uint32_t e0 = a.ebeg[al], e1 = a.ebeg[al + 1];
            int ne = 0;
            for (uint32_t x = e0; x < e1 && ne < kBwMaxErr; ++x) {
                const uint32_t s = a.ent_site[x];
                const ErrEnt v{a.site_item[s], a.site_mem[s], (uint32_t)a.ent_k[x]};
                int j = ne++;
                while (j > 0 && (errs[j - 1].item > v.item || (errs[j - 1].item == v.item && errs[j - 1].member > v.member))) {
                    errs[j] = errs[j - 1];
                    --j;
                }
                errs[j] = v;
            }
            int ng = 0;
            for (int j = 0; j < ne; ++j)
                if ((j == 0 || errs[j - 1].item != errs[j].item) && a.items[errs[j].item].diff) egs[ng++] = a.items[errs[j].item].gslot;
            s_nerr = ne;
            s_negs = ng;
        }
        for (uint32_t l = tid; l < L; l += kBwThreads) phi[l] = make_float2((rank == 0 && l == 0) ? 1.f : 0.f, 0.f);
        __syncthreads();
        const int nerr = s_nerr;
        // ---- forward ------------------------------------------------------------------------------
        int ep = 0;
        uint32_t ck = 0;
        for (uint32_t st = 0; st < a.nsteps; ++st) {
            const BwStep S = a.steps[st];
            if (S.kind == 1) { swap_positions<CL>(phi, nullptr, nl, (int)S.a, (int)S.g, rank); continue; }
            const uint32_t b = S.item;
            const BwItem it = a.items[b];
            int e1 = ep;
            while (e1 < nerr && errs[e1].item == b) ++e1;
            const float2* Bm = a.pool + (size_t)it.def * 16;
            bool sing = it.defsing != 0;
            if (e1 > ep) {
                if (warp == 0) build_item(a, it, errs + ep, e1 - ep, Bs, Bis, &s_sing, lane);
                __syncthreads();
                Bm = Bs;
                sing = s_sing != 0;
            }
            ep = e1;
            if (sing || it.ckpt || (a.ckpt_every && b % a.ckpt_every == 0)) {
                if (ck < a.maxck) {   // the host sizes maxck for every set; the test only guards memory
                    float2* dst = a.ckpt + ((((size_t)slot * a.maxck + ck) << a.n) | slice);
                    for (uint32_t l = tid; l < L; l += kBwThreads) dst[l] = phi[l];
                }
                ++ck;
                __syncthreads();
            }
            if (it.nq == 1) fwd_pass<2>(phi, nl, it.p0, 0, Bm);
            else fwd_pass<4>(phi, nl, it.p0, it.p1, Bm);
            __syncthreads();
        }
        // ---- observable: E = <phi|O|phi>, mu = O phi ------------------------------------------------
        double ev = 0;
        for (uint32_t l = tid; l < L; l += kBwThreads) {
            const uint32_t X = (uint32_t)slice | l;
            double o = 0;
            if (a.diag) {
                uint32_t x = 0;
                for (int q = 0; q < a.n; ++q) x |= ((X >> a.pos_final[q]) & 1u) << q;
                o = a.diag[x];
            }
            for (uint32_t t = 0; t < a.nterms; ++t) o += (__popc(X & a.pmask[t]) & 1) ? -a.coeff[t] : a.coeff[t];
            const float2 v = phi[l];
            ev += o * ((double)v.x * v.x + (double)v.y * v.y);
            mu[l] = make_float2((float)(o * (double)v.x), (float)(o * (double)v.y));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) ev += __shfl_xor_sync(0xFFFFFFFFu, ev, o);
        if (lane == 0) s_part[warp] = ev;
        __syncthreads();
        if (tid == 0) {
            double t = 0;
            for (int w = 0; w < kBwWarps; ++w) t += s_part[w];
            s_E = t;
        }
        if constexpr (CL > 1) cg::this_cluster().sync();
        else __syncthreads();
        // ---- backward -----------------------------------------------------------------------------
        ep = nerr;
        int gbuf = 0;
        double* Ga = a.Ga + ((size_t)slot * CL + rank) * a.ngs * 32;
        for (int st = (int)a.nsteps - 1; st >= (int)a.first_diff_step; --st) {
            const BwStep S = a.steps[st];
            if (S.kind == 1) { swap_positions<CL>(phi, mu, nl, (int)S.a, (int)S.g, rank); continue; }
            const uint32_t b = S.item;
            const BwItem it = a.items[b];
            int e0 = ep;
            while (e0 > 0 && errs[e0 - 1].item == b) --e0;
            const float2* Bm = a.pool + (size_t)it.def * 16;
            const float2* Bim = a.pool + (size_t)it.definv * 16;
            bool sing = it.defsing != 0;
            if (e0 < ep) {
                if (warp == 0) build_item(a, it, errs + e0, ep - e0, Bs, Bis, &s_sing, lane);
                __syncthreads();
                Bm = Bs; Bim = Bis;
                sing = s_sing != 0;
            }
            ep = e0;
            const float2* ckp = nullptr;
            if (sing || it.ckpt || (a.ckpt_every && b % a.ckpt_every == 0)) {
                --ck;   // forward counted every block, backward visits a suffix: ck stays >= 0
                if (ck < a.maxck) ckp = a.ckpt + ((((size_t)slot * a.maxck + ck) << a.n) | slice);
            }
            if (it.nq == 1) {
                float g[8] = {};
                if (it.diff) {
                    bwd_pass<2, true>(phi, mu, nl, it.p0, 0, Bm, Bim, ckp, g);
                    const float v = warp_vec_sum<8>(g, lane);
                    if ((lane & 3) == 0) red[gbuf][warp][lane >> 2] = v;
                } else {
                    bwd_pass<2, false>(phi, mu, nl, it.p0, 0, Bm, Bim, ckp, g);
                }
            } else {
                float g[32] = {};
                if (it.diff) {
                    bwd_pass<4, true>(phi, mu, nl, it.p0, it.p1, Bm, Bim, ckp, g);
                    const float v = warp_vec_sum<32>(g, lane);
                    red[gbuf][warp][lane] = v;
                } else {
                    bwd_pass<4, false>(phi, mu, nl, it.p0, it.p1, Bm, Bim, ckp, g);
                }
            }
            __syncthreads();
            if (it.diff && warp == 0) {
                const int K = it.nq == 1 ? 8 : 32;
                if (lane < K) {
                    double s = 0;
                    for (int w = 0; w < kBwWarps; ++w) s += (double)red[gbuf][w][lane];
                    Ga[(size_t)it.gslot * 32 + lane] = s;
                }
            }
            if (it.diff) gbuf ^= 1;
        }
        __syncthreads();
        // ---- weights ------------------------------------------------------------------------------
        const double W = a.W[al];
        {
            double* Gbar = a.Gbar + ((size_t)slot * CL + rank) * a.ngs * 32;
            const int ng = s_negs;
            for (uint32_t x = tid; x < a.ngs * 32; x += kBwThreads) {
                const uint32_t gs = x >> 5;
                bool skip = false;
                for (int j = 0; j < ng; ++j) skip |= egs[j] == gs;
                if (!skip) Gbar[x] += W * Ga[x];
            }
        }
        if constexpr (CL > 1) cg::this_cluster().sync();
        if (rank == 0) {
            if (warp == 0) {
                // blocks holding entries of this set: contract now with the set's variants
                int j = 0;
                while (j < nerr) {
                    int j1 = j + 1;
                    while (j1 < nerr && errs[j1].item == errs[j].item) ++j1;
                    const BwItem it = a.items[errs[j].item];
                    if (it.diff) {
                        double s = 0;
                        for (int rr = 0; rr < CL; ++rr) s += a.Ga[(((size_t)slot * CL + rr) * a.ngs + it.gslot) * 32 + lane];
                        s_G[lane] = s;
                        __syncwarp();
                        contract_item(a, it, errs + j, j1 - j, s_G, W, a.acc_err + (size_t)slot * a.ndslots, s_sc, lane);
                        __syncwarp();
                    }
                    j = j1;
                }
            }
            if (tid == 32) {
                double E = s_E;
                if constexpr (CL > 1) {
                    cg::cluster_group cl = cg::this_cluster();
                    E = 0;
                    for (int rr = 0; rr < CL; ++rr) E += *cl.map_shared_rank(&s_E, rr);
                }
                a.acc_loss[slot] += W * E;
                if (a.per_set) a.per_set[al] = a.s2q[al] * E;
                for (int c = 0; c < a.nch; ++c) a.acc_mix[(size_t)slot * a.nch + c] += W * E * a.gmix[(size_t)al * a.nch + c];
            }
        }
        if constexpr (CL > 1) cg::this_cluster().sync();
        else __syncthreads();
    }
}

// Default blocks: sum the per-slot accumulators, contract with the variant-0 derivatives; then add
// the per-set contractions and the unitary-mixture terms, and scatter to the outputs.
__global__ void __launch_bounds__(kFinThreads) k_backward_finish(BwArgs a) {
    __shared__ double2 sc[kFinWarps][32];
    __shared__ double Gs[kFinWarps][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t d = tid; d < a.ndslots; d += blockDim.x) a.dtot[d] = 0;
    __syncthreads();
    for (uint32_t b = warp; b < a.nitems; b += kFinWarps) {
        const BwItem it = a.items[b];
        if (!it.diff) continue;
        double s = 0;
        for (uint32_t sl = 0; sl < a.nslots; ++sl)
            for (int rr = 0; rr < a.cl; ++rr) s += a.Gbar[(((size_t)sl * a.cl + rr) * a.ngs + it.gslot) * 32 + lane];
        Gs[warp][lane] = s;
        __syncwarp();
        contract_item(a, it, nullptr, 0, Gs[warp], 1.0, a.dtot, sc[warp], lane);
        __syncwarp();
    }
    __syncthreads();
    for (uint32_t d = tid; d < a.ndslots; d += blockDim.x) {
        double s = a.dtot[d];
        for (uint32_t sl = 0; sl < a.nslots; ++sl) s += a.acc_err[(size_t)sl * a.ndslots + d];
        a.dtot[d] = s;
    }
    __syncthreads();
    if (a.grad_params) {
        for (uint32_t i = tid; i < 3 * a.n_ops; i += blockDim.x) a.grad_params[i] = 0;
        __syncthreads();
        for (uint32_t d = tid; d < a.ndslots; d += blockDim.x)
            if (!(a.dslot_out[d] & 0x80000000u)) a.grad_params[a.dslot_out[d]] = a.dtot[d];
    }
    if (a.grad_noise)
        for (int c = tid; c < a.nch; c += blockDim.x) {
            double s = 0;
            for (uint32_t d = 0; d < a.ndslots; ++d)
                if (a.dslot_out[d] == (0x80000000u | (uint32_t)c)) s += a.dtot[d];
            for (uint32_t sl = 0; sl < a.nslots; ++sl) s += a.acc_mix[(size_t)sl * a.nch + c];
            a.grad_noise[c] = s;
        }
    if (a.loss && tid == 0) {
        double s = 0;
        for (uint32_t sl = 0; sl < a.nslots; ++sl) s += a.acc_loss[sl];
        *a.loss = s;
    }
}

size_t bw_smem(int nl) { return 2 * sizeof(float2) * ((size_t)1 << nl); }

template <int CL>
void configure() {
    // thread-safe once: two contexts may be driven from two host threads
    static const bool done = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_backward<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bw_smem(kBwLocalBits)));
        return true;
    }();
    (void)done;
}

template <int CL>
uint32_t slots_for(int nl, int n_sm) {
    configure<CL>();
    const size_t smem = bw_smem(nl);
    if constexpr (CL == 1) {
        int nb = 0;
        PTSBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_backward<1>, kBwThreads, smem));
        return (uint32_t)std::max(1, nb) * (uint32_t)std::max(1, n_sm);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CL, 1, 1);
        cfg.blockDim = dim3(kBwThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr; cfg.numAttrs = 1;
        int nc = 0;
        PTSBE_CUDA(cudaOccupancyMaxActiveClusters(&nc, k_backward<CL>, &cfg));
        return (uint32_t)std::max(1, nc);
    }
}

template <int CL>
void launch_main(const BwArgs& a, cudaStream_t s) {
    configure<CL>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nslots * CL, 1, 1);
    cfg.blockDim = dim3(kBwThreads, 1, 1);
    cfg.dynamicSmemBytes = bw_smem(a.nl);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr; cfg.numAttrs = 1;
    PTSBE_CUDA(cudaLaunchKernelEx(&cfg, k_backward<CL>, a));
    count_launch();
}

}  // namespace

uint32_t backward_slots(int n, uint32_t count, int n_sm) {
    const int nl = n < kBwLocalBits ? n : kBwLocalBits;
    uint32_t s = 1;
    switch (n - nl) {
    case 0: s = slots_for<1>(nl, n_sm); break;
    case 1: s = slots_for<2>(nl, n_sm); break;
    case 2: s = slots_for<4>(nl, n_sm); break;
    case 3: s = slots_for<8>(nl, n_sm); break;
    default: fail(PTSBE_ERR_UNSUPPORTED, "backward handles at most 16 qubits");
    }
    return std::max<uint32_t>(1, std::min(s, count));
}

void launch_backward(const BwArgs& a, cudaStream_t s) {
    if (a.count > 0) {
        switch (a.cl) {
        case 1: launch_main<1>(a, s); break;
        case 2: launch_main<2>(a, s); break;
        case 4: launch_main<4>(a, s); break;
        case 8: launch_main<8>(a, s); break;
        default: fail(PTSBE_ERR_UNSUPPORTED, "backward cluster size");
        }
    }
    k_backward_finish<<<1, kFinThreads, 0, s>>>(a);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace ptsbe
