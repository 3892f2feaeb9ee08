// Batched state preparation for PTSBE (Sec. 3: each Kraus set alpha is prepared once).
//
// One CTA owns one tile (2^tb complex64 amplitudes, shared memory) of one state for one stage of
// the plan. It gathers the tile from HBM (segments of 2^lb contiguous amplitudes), applies every
// op of the stage in shared memory -- gates, and at each noise site the Kraus operator that the
// state's set alpha selects (operator 0 where alpha lists nothing) -- and scatters the tile back.
// When the whole state fits one tile (n <= tb) the entire circuit runs in a single launch and the
// final renormalisation and branch weight are fused into the same CTA.
//
// Renormalisation (Sec. 2.2) is deferred to the end: the branch weight is the squared norm of
// the unnormalised state times the unitary-mixture probabilities, and dividing once at the end
// gives the same normalised state as dividing after every general Kraus operator.
//
// Prefix reuse: when set beta extends set alpha of the same batch, alpha writes its tile into
// beta's output slot just before alpha reaches beta's first extra site; beta later resumes from
// that op. Generations (depth in the prefix tree) run one after the other.
#include <cstdio>

#include "internal.h"

namespace ptsbe {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a*b + c*d
__device__ __forceinline__ float2 cmul2(float2 a, float2 b, float2 c, float2 d) {
    float2 r = cmul(c, d);
    r.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, r.x));
    r.y = fmaf(a.x, b.y, fmaf(a.y, b.x, r.y));
    return r;
}
__device__ __forceinline__ uint32_t ins0(uint32_t i, int p) { return ((i >> p) << (p + 1)) | (i & ((1u << p) - 1u)); }

// --- shared-memory micro kernels: every thread of the CTA calls them ------------------------------

__device__ void t_g1(float2* s, int tb, int p, const float2* __restrict__ m) {
    const float2 m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
    const uint32_t half = 1u << (tb - 1), bit = 1u << p;
    for (uint32_t i = threadIdx.x; i < half; i += blockDim.x) {
        const uint32_t i0 = ins0(i, p), i1 = i0 | bit;
        const float2 a = s[i0], b = s[i1];
        s[i0] = cmul2(m00, a, m01, b);
        s[i1] = cmul2(m10, a, m11, b);
    }
}

__device__ void t_d1(float2* s, int tb, int p, const float2* __restrict__ m) {
    const float2 d0 = m[0], d1 = m[1];
    const uint32_t half = 1u << (tb - 1), bit = 1u << p;
    if (d0.x == 1.0f && d0.y == 0.0f) {
        for (uint32_t i = threadIdx.x; i < half; i += blockDim.x) {
            const uint32_t i1 = ins0(i, p) | bit;
            s[i1] = cmul(d1, s[i1]);
        }
    } else {
        for (uint32_t i = threadIdx.x; i < half; i += blockDim.x) {
            const uint32_t i0 = ins0(i, p), i1 = i0 | bit;
            s[i0] = cmul(d0, s[i0]);
            s[i1] = cmul(d1, s[i1]);
        }
    }
}

// [[0, a], [b, 0]]
__device__ void t_x1(float2* s, int tb, int p, const float2* __restrict__ m) {
    const float2 a = m[0], b = m[1];
    const uint32_t half = 1u << (tb - 1), bit = 1u << p;
    const bool plain = a.x == 1.0f && a.y == 0.0f && b.x == 1.0f && b.y == 0.0f;
    for (uint32_t i = threadIdx.x; i < half; i += blockDim.x) {
        const uint32_t i0 = ins0(i, p), i1 = i0 | bit;
        const float2 v0 = s[i0], v1 = s[i1];
        if (plain) { s[i0] = v1; s[i1] = v0; }
        else { s[i0] = cmul(a, v1); s[i1] = cmul(b, v0); }
    }
}

__device__ __forceinline__ uint32_t ins00(uint32_t i, int pa, int pb) {
    const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
    return ins0(ins0(i, lo), hi);
}

__device__ void t_cx(float2* s, int tb, int pc, int pt) {
    const uint32_t q = 1u << (tb - 2);
    for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const uint32_t b = ins00(i, pc, pt) | (1u << pc);
        const float2 v0 = s[b], v1 = s[b | (1u << pt)];
        s[b] = v1; s[b | (1u << pt)] = v0;
    }
}

__device__ void t_cz(float2* s, int tb, int pa, int pb) {
    const uint32_t q = 1u << (tb - 2);
    for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const uint32_t b = ins00(i, pa, pb) | (1u << pa) | (1u << pb);
        const float2 v = s[b];
        s[b] = make_float2(-v.x, -v.y);
    }
}

__device__ void t_swap(float2* s, int tb, int pa, int pb) {
    const uint32_t q = 1u << (tb - 2);
    for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const uint32_t b = ins00(i, pa, pb);
        const uint32_t x = b | (1u << pa), y = b | (1u << pb);
        const float2 v0 = s[x], v1 = s[y];
        s[x] = v1; s[y] = v0;
    }
}

// 4x4 on local index 2*bit(pa) + bit(pb)
__device__ void t_g2(float2* s, int tb, int pa, int pb, const float2* __restrict__ m) {
    const uint32_t q = 1u << (tb - 2);
    for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const uint32_t b = ins00(i, pa, pb);
        const uint32_t idx[4] = {b, b | (1u << pb), b | (1u << pa), b | (1u << pa) | (1u << pb)};
        float2 v[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) v[l] = s[idx[l]];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float2 acc = cmul(m[4 * r], v[0]);
#pragma unroll
            for (int l = 1; l < 4; ++l) {
                const float2 t = cmul(m[4 * r + l], v[l]);
                acc.x += t.x; acc.y += t.y;
            }
            s[idx[r]] = acc;
        }
    }
}

__device__ __forceinline__ void apply_micro(float2* s, int tb, uint8_t kind, int pa, int pb, const float2* m) {
    switch (kind) {
    case DOP_G1: t_g1(s, tb, pa, m); break;
    case DOP_D1: t_d1(s, tb, pa, m); break;
    case DOP_X1: t_x1(s, tb, pa, m); break;
    case DOP_CX: t_cx(s, tb, pa, pb); break;
    case DOP_CZ: t_cz(s, tb, pa, pb); break;
    case DOP_SWAP: t_swap(s, tb, pa, pb); break;
    case DOP_G2: t_g2(s, tb, pa, pb, m); break;
    default: break;
    }
}

// --- tile movement ------------------------------------------------------------------------------------

__device__ __forceinline__ uint64_t gidx(uint32_t l, int lb, const uint32_t* hi, uint64_t outer) {
    return (uint64_t)(l & ((1u << lb) - 1u)) | (uint64_t)hi[l >> lb] | outer;
}

__device__ void tile_load(float2* tile, const float2* __restrict__ g, int tb, int lb, const uint32_t* hi, uint64_t outer) {
    const uint32_t nv = 1u << (tb - 1);
    for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const uint32_t l = 2 * v;
        reinterpret_cast<float4*>(tile)[v] = __ldg(reinterpret_cast<const float4*>(g + gidx(l, lb, hi, outer)));
    }
}

__device__ void tile_store(const float2* tile, float2* g, int tb, int lb, const uint32_t* hi, uint64_t outer, float scale) {
    const uint32_t nv = 1u << (tb - 1);
    for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const uint32_t l = 2 * v;
        float4 x = reinterpret_cast<const float4*>(tile)[v];
        if (scale != 1.0f) { x.x *= scale; x.y *= scale; x.z *= scale; x.w *= scale; }
        *reinterpret_cast<float4*>(g + gidx(l, lb, hi, outer)) = x;
    }
}

// Deterministic CTA sum in FP64 of per-thread values; every thread gets the result.
__device__ double cta_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += red[i];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

__device__ double tile_norm_partial(const float2* tile, int tb) {
    double acc = 0.0;
    for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x) {
        const float2 a = tile[l];
        acc += (double)fmaf(a.x, a.x, a.y * a.y);
    }
    return acc;
}

__global__ void __launch_bounds__(1024) k_evolve_stage(EvolveArgs a, int stage_idx, int last, const uint32_t* __restrict__ nodes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevStage st;
    __shared__ double red[33];
    const int tb = a.tb, lb = a.lb, n = a.n, ob = n - tb;
    float2* tile = reinterpret_cast<float2*>(smem);
    uint32_t* hi = reinterpret_cast<uint32_t*>(tile + (1u << tb));
    if (threadIdx.x == 0) st = a.stages[stage_idx];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (1u << (tb - lb)); i += blockDim.x) hi[i] = a.hi[st.hi_off + i];
    const uint32_t node = nodes[blockIdx.y];
    const uint32_t tau = blockIdx.x;
    uint64_t outer = 0;
    for (int b = 0; b < ob; ++b)
        if ((tau >> b) & 1u) outer |= 1ull << st.outer_q[b];
    float2* g = a.states + ((size_t)node << n);
    const uint32_t nstart = a.node_start[node];
    const uint32_t start = nstart > st.op_begin ? nstart : st.op_begin;
    __syncthreads();
    if (a.node_fresh[node] && stage_idx == 0) {
        for (uint32_t l = threadIdx.x; l < (1u << tb); l += blockDim.x)
            tile[l] = make_float2((l == 0 && tau == 0) ? 1.0f : 0.0f, 0.0f);
    } else {
        tile_load(tile, g, tb, lb, hi, outer);
    }
    uint32_t e = a.node_ebeg[node];
    const uint32_t ee = a.node_eend[node];
    while (e < ee && a.site_op[a.ent_site[e]] < start) ++e;
    uint32_t c = a.node_cbeg[node];
    const uint32_t ce = a.node_cend[node];
    while (c < ce && a.child_op[c] < start) ++c;
    __syncthreads();

    for (uint32_t op = start; op < st.op_end; ++op) {
        const DevOp o = a.ops[op];
        if (o.kind == DOP_NOISE) {
            if (c < ce && a.child_op[c] == op) {
                do {
                    tile_store(tile, a.states + ((size_t)a.child_node[c] << n), tb, lb, hi, outer, 1.0f);
                    ++c;
                } while (c < ce && a.child_op[c] == op);
                __syncthreads();
            }
            uint32_t k = 0;
            if (e < ee && a.ent_site[e] == o.site) { k = a.ent_k[e]; ++e; }
            const uint32_t u0 = a.chans[o.ch].micro_off[k], u1 = a.chans[o.ch].micro_off[k + 1];
            for (uint32_t u = u0; u < u1; ++u) {
                const DevMicro mi = a.micro[u];
                const int pa = st.pos[mi.operand == 1 ? o.q1 : o.q0];
                const int pb = st.pos[o.q1];
                apply_micro(tile, tb, mi.kind, pa, pb, a.mats + mi.mat);
                __syncthreads();
            }
        } else if (o.kind != DOP_NOP) {
            apply_micro(tile, tb, o.kind, st.pos[o.q0], st.pos[o.q1], a.mats + o.mat);
            __syncthreads();
        }
    }

    if (!last) {
        tile_store(tile, g, tb, lb, hi, outer, 1.0f);
        return;
    }
    const double part = cta_sum(tile_norm_partial(tile, tb), red);
    if (ob == 0) {
        const double w = a.wmix[node] * part;
        const bool null = !(part > 0.0) || w < 1e-6 * a.qalpha[node];
        const float scale = null ? 0.0f : (float)(1.0 / sqrt(part));
        tile_store(tile, g, tb, lb, hi, outer, scale);
        if (threadIdx.x == 0) {
            if (a.weights) a.weights[node] = w;
            if (a.status) a.status[node] = null ? 1 : 0;
        }
    } else {
        tile_store(tile, g, tb, lb, hi, outer, 1.0f);
        if (threadIdx.x == 0) a.part[((size_t)node << ob) + tau] = part;
    }
}

// Per node: total squared norm from the tile partials (fixed order), weight, null flag, scale.
__global__ void k_evolve_reduce(EvolveArgs a, float* scale_out) {
    __shared__ double red[33];
    const uint32_t node = blockIdx.x;
    const int ob = a.n - a.tb;
    const double* p = a.part + ((size_t)node << ob);
    double acc = 0.0;
    for (uint32_t i = threadIdx.x; i < (1u << ob); i += blockDim.x) acc += p[i];
    const double T = cta_sum(acc, red);
    if (threadIdx.x == 0) {
        const double w = a.wmix[node] * T;
        const bool null = !(T > 0.0) || w < 1e-6 * a.qalpha[node];
        scale_out[node] = null ? 0.0f : (float)(1.0 / sqrt(T));
        if (a.weights) a.weights[node] = w;
        if (a.status) a.status[node] = null ? 1 : 0;
    }
}

__global__ void k_evolve_scale(float2* states, int n, const float* __restrict__ scale) {
    const uint32_t node = blockIdx.y;
    const float s = scale[node];
    float4* v = reinterpret_cast<float4*>(states + ((size_t)node << n));
    const uint64_t nv = 1ull << (n - 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x) {
        float4 x = v[i];
        x.x *= s; x.y *= s; x.z *= s; x.w *= s;
        v[i] = x;
    }
}

int evolve_threads(int tb) {
    const int amps = 1 << tb;
    int t = amps / 16;
    if (t < 64) t = 64;
    if (t > 1024) t = 1024;
    return t;
}

}  // namespace

size_t evolve_smem_bytes(int tb, int lb) { return ((size_t)8 << tb) + ((size_t)4 << (tb - lb)); }

void launch_evolve_stage(const EvolveArgs& a, int stage, bool last, const uint32_t* d_nodes, uint32_t n_nodes,
                         cudaStream_t s) {
    if (n_nodes == 0) return;
    static bool configured = false;
    if (!configured) {
        PTSBE_CUDA(cudaFuncSetAttribute(k_evolve_stage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)evolve_smem_bytes(kTileMax, 1)));
        configured = true;
    }
    const size_t smem = evolve_smem_bytes(a.tb, a.lb);
    const int threads = evolve_threads(a.tb);
    const uint32_t tiles = 1u << (a.n - a.tb);
    for (uint32_t b = 0; b < n_nodes; b += 65535) {
        const uint32_t cnt = (n_nodes - b) < 65535u ? (n_nodes - b) : 65535u;
        k_evolve_stage<<<dim3(tiles, cnt), threads, smem, s>>>(a, stage, last ? 1 : 0, d_nodes + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

void launch_evolve_finalize(const EvolveArgs& a, uint32_t count, float* d_scale, cudaStream_t s) {
    if (a.n == a.tb || count == 0) return;
    k_evolve_reduce<<<count, 256, 0, s>>>(a, d_scale);
    PTSBE_CUDA(cudaGetLastError());
        count_launch();
    const uint64_t nv = 1ull << (a.n - 1);
    uint32_t blocks = (uint32_t)((nv + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    for (uint32_t b = 0; b < count; b += 65535) {
        const uint32_t cnt = (count - b) < 65535u ? (count - b) : 65535u;
        k_evolve_scale<<<dim3(blocks, cnt), 256, 0, s>>>(a.states + ((size_t)b << a.n), a.n, d_scale + b);
        PTSBE_CUDA(cudaGetLastError());
        count_launch();
    }
}

}  // namespace ptsbe
