// Traditional trajectory simulation, one prepared state per shot (Algorithm 1), as the comparison
// path for PTSBE on the same GPU with the same tile machinery.
//
// At noise site s shot j draws u = U53(Philox(seed; s, j_lo, j_hi, 3)). A unitary mixture picks k
// by its fixed probabilities and applies U_k. A general channel needs the branch probabilities
// p_i = <psi|K_i^dag K_i|psi> of the current state: when the state is one tile they are reduced in
// the CTA; otherwise the plan starts a new stage at every general site and the previous stage's
// epilogue leaves per-tile partials (FP64), which every tile of the shot sums in the same order, so
// all tiles pick the same k. The chosen K_k is applied and the state divided by sqrt(p_k).
#include "internal.h"
#include "philox.h"
#include "tile_ops.cuh"

namespace ptsbe {

namespace {
using namespace tile;

// Re <v|M|v> over this thread's share of the tile for a Hermitian M on one or two tile positions.
__device__ double tile_expect(const float2* s, int tb, int nt, int pa, int pb, const float2* __restrict__ M) {
    double acc = 0.0;
    if (nt == 1) {
        const float2 m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
        const uint32_t half = 1u << (tb - 1), bit = 1u << pa;
        for (uint32_t i = threadIdx.x; i < half; i += blockDim.x) {
            const uint32_t i0 = ins0(i, pa), i1 = i0 | bit;
            const float2 x = s[i0], y = s[i1];
            const float2 mx = cmul2(m00, x, m01, y), my = cmul2(m10, x, m11, y);
            acc += (double)(x.x * mx.x + x.y * mx.y + y.x * my.x + y.y * my.y);
        }
    } else {
        const uint32_t q = 1u << (tb - 2);
        for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
            const uint32_t b = ins00(i, pa, pb);
            const uint32_t idx[4] = {b, b | (1u << pb), b | (1u << pa), b | (1u << pa) | (1u << pb)};
            float2 v[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) v[l] = s[idx[l]];
            float re = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float2 mv = cmul(M[4 * r], v[0]);
#pragma unroll
                for (int l = 1; l < 4; ++l) {
                    const float2 t = cmul(M[4 * r + l], v[l]);
                    mv.x += t.x; mv.y += t.y;
                }
                re += v[r].x * mv.x + v[r].y * mv.y;
            }
            acc += (double)re;
        }
    }
    return acc;
}

__device__ void t_scale(float2* s, int tb, float f) {
    for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x) { s[l].x *= f; s[l].y *= f; }
}

__global__ void __launch_bounds__(1024) k_pershot_stage(PershotArgs a, int stage_idx) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevStage st;
    __shared__ double red[33];
    __shared__ double pk[kMaxKraus];
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    float2* tile = reinterpret_cast<float2*>(smem);
    uint32_t* hi = reinterpret_cast<uint32_t*>(tile + (1u << tb));
    if (threadIdx.x == 0) st = a.stages[stage_idx];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (1u << (tb - lb)); i += blockDim.x) hi[i] = a.hi[st.hi_off + i];
    const uint32_t node = blockIdx.y, tau = blockIdx.x;
    const uint64_t j = a.first_shot + node;
    uint64_t outer = 0;
    for (int b = 0; b < ob; ++b)
        if ((tau >> b) & 1u) outer |= 1ull << st.outer_q[b];
    float2* g = a.states + ((size_t)node << n);
    __syncthreads();
    if (stage_idx == 0) {
        for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x)
            tile[l] = make_float2((l == 0 && tau == 0) ? 1.0f : 0.0f, 0.0f);
    } else {
        tile_load(tile, g, tb, lb, hi, outer);
    }
    __syncthreads();

    __shared__ DevOp sops[kOpChunk];
    OpWindow win{sops};
    for (uint32_t op = st.op_begin; op < st.op_end; ++op) {
        const DevOp o = win.at(a.ops, op, st.op_end);
        if (o.kind != DOP_NOISE) {
            if (o.kind != DOP_NOP) {
                apply_micro(tile, tb, o.kind, st.pos[o.q0], st.pos[o.q1], a.mats + o.mat);
                __syncthreads();
            }
            continue;
        }
        const DevChannel& ch = a.chans[o.ch];
        const int nk = ch.nk;
        const double u = uniform53(a.seed, o.site, (uint32_t)j, (uint32_t)(j >> 32), kDomPershotKraus);
        int k;
        float scale = 1.0f;
        if (ch.mixture) {
            double acc = 0.0;
            k = nk - 1;
            for (int kk = 0; kk < nk; ++kk) { acc += ch.q[kk]; if (u < acc) { k = kk; break; } }
        } else {
            if (ob == 0) {
                for (int kk = 0; kk < nk; ++kk) {
                    const double e = cta_sum(tile_expect(tile, tb, o.nt, st.pos[o.q0], st.pos[o.q1], a.mats + ch.herm_mat[kk]), red);
                    if (threadIdx.x == 0) pk[kk] = e;
                }
            } else if (threadIdx.x == 0) {
                // the previous stage left per-tile partials for this site (it opens this stage); the
                // partials are double-buffered by stage parity so this stage's epilogue cannot
                // overwrite them while other tiles of the shot still read them
                const double* part = a.part + ((size_t)((stage_idx + 1) & 1) * gridDim.y + node) * ((size_t)kMaxKraus << ob);
                for (int kk = 0; kk < nk; ++kk) {
                    double e = 0.0;
                    for (uint32_t t = 0; t < (1u << ob); ++t) e += part[(size_t)t * kMaxKraus + kk];
                    pk[kk] = e;
                }
            }
            __syncthreads();
            double acc = 0.0;
            k = nk - 1;
            for (int kk = 0; kk < nk; ++kk) { acc += pk[kk]; if (u < acc) { k = kk; break; } }
            while (k > 0 && !(pk[k] > 0.0)) --k;       // rounding fallback landed on an impossible branch
            scale = pk[k] > 0.0 ? (float)(1.0 / sqrt(pk[k])) : 0.0f;
        }
        for (uint32_t mu = ch.micro_off[k]; mu < ch.micro_off[k + 1]; ++mu) {
            const DevMicro mi = a.micro[mu];
            apply_micro(tile, tb, mi.kind, st.pos[mi.operand == 1 ? o.q1 : o.q0], st.pos[o.q1], a.mats + mi.mat);
            __syncthreads();
        }
        if (scale != 1.0f) {
            t_scale(tile, tb, scale);
            __syncthreads();
        }
        if (a.kraus && threadIdx.x == 0 && tau == 0) a.kraus[(size_t)node * a.n_sites + o.site] = (uint8_t)k;
    }

    if (st.flags & 1u) {
        // branch-probability partials of the general site that opens the next stage
        const DevOp P = a.ops[st.probe_op];
        const DevChannel& ch = a.chans[P.ch];
        double* part = a.part + ((size_t)(stage_idx & 1) * gridDim.y + node) * ((size_t)kMaxKraus << ob) + (size_t)tau * kMaxKraus;
        for (int kk = 0; kk < ch.nk; ++kk) {
            const double e = cta_sum(tile_expect(tile, tb, P.nt, st.pos[P.q0], st.pos[P.q1], a.mats + ch.herm_mat[kk]), red);
            if (threadIdx.x == 0) part[kk] = e;
        }
    }
    tile_store(tile, g, tb, lb, hi, outer, 1.0f);
}

}  // namespace

void launch_pershot_stage(const PershotArgs& a, int stage, uint32_t batch, cudaStream_t s) {
    if (batch == 0) return;
    const size_t smem_max = ((size_t)8 << kTileMax) + ((size_t)4 << (kTileMax - 1));
    // thread-safe once: two contexts may be driven from two host threads
    static const bool configured = [&] {
        PTSBE_CUDA(cudaFuncSetAttribute(k_pershot_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        return true;
    }();
    (void)configured;
    const size_t smem = ((size_t)8 << a.tb) + ((size_t)4 << (a.tb - a.lb));
    int threads = (1 << a.tb) / 16;
    if (threads < 64) threads = 64;
    if (threads > 1024) threads = 1024;
    const uint32_t tiles = 1u << (a.n - a.tb);
    k_pershot_stage<<<dim3(tiles, batch), threads, smem, s>>>(a, stage);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace ptsbe
