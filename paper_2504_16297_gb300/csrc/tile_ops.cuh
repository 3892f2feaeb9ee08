// Shared-memory tile micro-kernels used by the tile passes of batched preparation and of the
// per-shot trajectories: every thread of the CTA calls them on the CTA's tile of 2^tb amplitudes.
#pragma once
#include <cstdint>

#include "internal.h"

namespace ptsbe {
namespace tile {
namespace {   // each translation unit gets its own copy

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

// monomial 4x4: out[l] = d[l] * in[perm_l] on local index 2*bit(pa) + bit(pb)
__device__ __forceinline__ float2 pick4(const float2 (&x)[4], int p) {
    return p == 0 ? x[0] : (p == 1 ? x[1] : (p == 2 ? x[2] : x[3]));
}
__device__ void t_m2(float2* s, int tb, int pa, int pb, const float2* __restrict__ m, uint32_t perm) {
    const uint32_t q = 1u << (tb - 2);
    const float2 d[4] = {m[0], m[1], m[2], m[3]};
    for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const uint32_t b = ins00(i, pa, pb);
        const uint32_t idx[4] = {b, b | (1u << pb), b | (1u << pa), b | (1u << pa) | (1u << pb)};
        float2 x[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) x[l] = s[idx[l]];
#pragma unroll
        for (int l = 0; l < 4; ++l) s[idx[l]] = cmul(d[l], pick4(x, (perm >> (2 * l)) & 3));
    }
}

__device__ __forceinline__ void apply_micro(float2* s, int tb, uint8_t kind, int pa, int pb, const float2* m,
                                            uint32_t perm = 0) {
    switch (kind) {
    case DOP_G1: t_g1(s, tb, pa, m); break;
    case DOP_D1: t_d1(s, tb, pa, m); break;
    case DOP_X1: t_x1(s, tb, pa, m); break;
    case DOP_CX: t_cx(s, tb, pa, pb); break;
    case DOP_CZ: t_cz(s, tb, pa, pb); break;
    case DOP_SWAP: t_swap(s, tb, pa, pb); break;
    case DOP_G2: t_g2(s, tb, pa, pb, m); break;
    case DOP_M2: t_m2(s, tb, pa, pb, m, perm); break;
    default: break;
    }
}

// --- staged operator lists -------------------------------------------------------------------------
// The per-operator kernels walk a stage's op list one op at a time; read from global memory each op
// costs a chain of dependent loads (descriptor, then its tables) for every CTA. OpWindow keeps a
// chunk of the list in shared memory and restages it when the walk leaves the chunk. Every thread
// must call at() with the same op (the walk is uniform over the CTA): restaging is a barrier.
constexpr uint32_t kOpChunk = 128;   // 32-byte descriptors: 4 KB of shared memory
struct OpWindow {
    DevOp* buf;
    uint32_t c0 = 1u, c1 = 0u;       // staged ops [c0, c1)
    __device__ DevOp at(const DevOp* __restrict__ ops, uint32_t op, uint32_t end) {
        if (op < c0 || op >= c1) {
            __syncthreads();
            c0 = op;
            c1 = op + kOpChunk < end ? op + kOpChunk : end;
            const uint32_t words = (c1 - c0) * (uint32_t)(sizeof(DevOp) / 4);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(ops + c0);
            uint32_t* dst = reinterpret_cast<uint32_t*>(buf);
            for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldg(src + w);
            __syncthreads();
        }
        return buf[op - c0];
    }
};
static_assert(sizeof(DevOp) % 4 == 0, "op descriptors are staged as 4-byte words");

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

// Deterministic CTA sum in FP64 of per-thread values; every thread gets the result. Blocks
// smaller than a warp add their values sequentially.
__device__ double cta_sum(double v, double* red) {
    if (blockDim.x < 32) {
        __syncthreads();
        red[threadIdx.x] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (uint32_t i = 0; i < blockDim.x; ++i) t += red[i];
            red[32] = t;
        }
        __syncthreads();
        return red[32];
    }
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


}  // namespace
}  // namespace tile
}  // namespace ptsbe
