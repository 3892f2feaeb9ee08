// Dense tile passes (dense.cuh): batched state preparation (Sec. 3) for states too large, or too
// densely mixed, for the deferred-frame kernel -- every amplitude streams through HBM once per pass
// and every gate and Kraus operator of the pass is applied on chip.
//
// One launch runs one pass for a list of nodes (a node = one Kraus set's state: where its tiles are
// read from, where they go, and the set's override blocks -- the fused blocks that contain one of
// its Kraus entries). Persistent CTAs walk the (node, tile) work items: a tile is loaded with
// 16-byte loads into XOR-swizzled shared memory, every register group of the pass loads its 16
// amplitudes per thread, applies its blocks in registers and writes them back, and the tile is
// stored in the pass's output order. The last pass also leaves each tile's FP64 squared norm.
#include <algorithm>

#include "dense.cuh"
#include "internal.h"

namespace ptsbe {

namespace {

using namespace dense;

constexpr int kDenseCtasPerSm = 2;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Copy of `bytes` (a multiple of 4) from global to shared memory by the whole CTA.
__device__ __forceinline__ void copy_words(void* dst, const void* src, uint32_t bytes) {
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = __ldg(s + i);
}

__global__ void __launch_bounds__(kThreads, kDenseCtasPerSm) k_dense_pass(DenseArgs a) {
    __shared__ __align__(16) float2 tile[1 << kT];
    __shared__ uint32_t hi[kHi];
    __shared__ uint16_t omap[kHi];
    __shared__ Pass P;
    __shared__ double red[kThreads / 32];
    extern __shared__ __align__(16) unsigned char stage[];
    const uint32_t tid = threadIdx.x;
    if (tid == 0) P = a.passes[a.pass];
    __syncthreads();
    for (uint32_t i = tid; i < (uint32_t)kHi; i += kThreads) {
        hi[i] = a.hi[P.hi_off + i];
        omap[i] = a.omap[P.omap_off + i];
    }
    // the pass's groups, blocks and default matrices: staged in shared memory when they fit
    const bool staged = P.stage_bytes != 0;
    const Group* groups = a.groups + P.group_begin;
    const Block* blocks = a.blocks + P.blk_begin;
    const float2* mats = a.mats + P.mat_begin;
    if (staged) {
        static_assert(sizeof(Group) % 4 == 0 && sizeof(Block) % 4 == 0, "staged tables move 4-byte words");
        copy_words(stage, a.groups + P.group_begin, (P.group_end - P.group_begin) * (uint32_t)sizeof(Group));
        const uint32_t bo = dense_stage_blocks_off(P), mo = dense_stage_mats_off(P);
        copy_words(stage + bo, a.blocks + P.blk_begin, (P.blk_end - P.blk_begin) * (uint32_t)sizeof(Block));
        copy_words(stage + mo, a.mats + P.mat_begin, (P.mat_end - P.mat_begin) * (uint32_t)sizeof(float2));
        groups = reinterpret_cast<const Group*>(stage);
        blocks = reinterpret_cast<const Block*>(stage + bo);
        mats = reinterpret_cast<const float2*>(stage + mo);
    }
    const uint32_t ngroups = P.group_end - P.group_begin;
    const int ob = a.n - kT;
    const uint64_t items = (uint64_t)a.n_nodes << ob;
    const uint64_t tmask = (1ull << ob) - 1;
    constexpr int kVec = (1 << (kT - 1)) / kThreads;   // float4 (two amplitudes) per thread per tile
    static_assert(kVec % 8 == 0, "tile loads go in rounds of eight");
    for (uint64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const uint32_t ni = (uint32_t)(w >> ob);
        const uint64_t tau = w & tmask;
        const Node nd = a.nodes[ni];
        const uint64_t outer = outer_offset(P, tau);
        __syncthreads();   // the previous item's store has read the tile; tables and stage are loaded
        if (nd.src == nullptr && tau != 0) {
            // a state starting from |0...0>: every other tile is zero and stays zero in this pass
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < kVec; ++i) {
                const uint32_t L = 2u * (i * kThreads + tid);
                __stcs(reinterpret_cast<float4*>(nd.dst + outer + (L & 15u) + hi[L >> kC]), z);
            }
            if (a.last && tid == 0) a.part[((size_t)nd.part << ob) + tau] = 0.0;
            continue;
        }
        if (nd.src == nullptr) {
#pragma unroll
            for (int i = 0; i < (1 << kT) / kThreads; ++i) tile[i * kThreads + tid] = make_float2(0.f, 0.f);
            __syncthreads();
            if (tid == 0) tile[0] = make_float2(1.f, 0.f);
        } else {
            // eight 16-byte loads in flight per thread, twice
#pragma unroll
            for (int h = 0; h < kVec; h += 8) {
                float4 x[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t t = 2u * ((h + i) * kThreads + tid);
                    x[i] = __ldcs(reinterpret_cast<const float4*>(nd.src + outer + (t & 15u) + hi[t >> kC]));
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t t = 2u * ((h + i) * kThreads + tid);
                    const uint32_t s = swz(t);
                    const float4 y = (s & 1u) ? make_float4(x[i].z, x[i].w, x[i].x, x[i].y) : x[i];
                    *reinterpret_cast<float4*>(tile + (s & ~1u)) = y;
                }
            }
        }
        __syncthreads();
        // the set's override blocks in this pass, in execution order
        uint32_t ov = nd.ov_begin;
        while (ov < nd.ov_end && a.ovr[ov].block < P.blk_begin) ++ov;
        uint32_t next_ov = ov < nd.ov_end ? a.ovr[ov].block : 0xFFFFFFFFu;
        for (uint32_t g = 0; g < ngroups; ++g) {
            const Group& G = groups[g];
            const uint32_t base = group_base(G, tid);
            float2 v[kAmps];
#pragma unroll
            for (int j = 0; j < kAmps; ++j) v[j] = tile[base ^ G.roff[j]];
            const uint32_t b1 = G.blk_end - P.blk_begin;
            for (uint32_t b = G.blk_begin - P.blk_begin; b < b1; ++b) {
                const Block B = blocks[b];
                const float2* m = mats + (B.mat - P.mat_begin);
                if (B.id == next_ov) {
                    m = a.opool + a.ovr[ov].mat;
                    ++ov;
                    next_ov = ov < nd.ov_end ? a.ovr[ov].block : 0xFFFFFFFFu;
                }
                apply_block(v, B.code, m);
            }
#pragma unroll
            for (int j = 0; j < kAmps; ++j) tile[base ^ G.roff[j]] = v[j];
            __syncthreads();
        }
        double nrm = 0.0;
        const uint32_t o1 = P.olow[1];
#pragma unroll
        for (int i = 0; i < kVec; ++i) {
            const uint32_t L = 2u * (i * kThreads + tid);
            const uint32_t t0 = omap[L >> kC] ^ P.olow[L & 15u];
            const float2 p0 = tile[swz(t0)], p1 = tile[swz(t0 ^ o1)];
            __stcs(reinterpret_cast<float4*>(nd.dst + outer + (L & 15u) + hi[L >> kC]), make_float4(p0.x, p0.y, p1.x, p1.y));
            if (a.last) nrm += (double)(p0.x * p0.x + p0.y * p0.y) + (double)(p1.x * p1.x + p1.y * p1.y);
        }
        if (a.last) {
            nrm = warp_sum(nrm);
            if ((tid & 31) == 0) red[tid >> 5] = nrm;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int i = 0; i < kThreads / 32; ++i) s += red[i];
                a.part[((size_t)nd.part << ob) + tau] = s;
            }
        }
    }
}

}  // namespace

int dense_ctas_per_sm() { return kDenseCtasPerSm; }

void launch_dense_pass(const DenseArgs& a, int n_sm, cudaStream_t s) {
    if (a.n_nodes == 0) return;
    if (a.n <= kT || a.n > kMaxQ) fail(PTSBE_ERR_UNSUPPORTED, "dense passes need 12 < n <= 32");
    const uint64_t items = (uint64_t)a.n_nodes << (a.n - kT);
    const uint64_t cap = (uint64_t)std::max(1, n_sm) * kDenseCtasPerSm;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(items, cap);
    static bool configured = false;
    if (!configured) {
        PTSBE_CUDA(cudaFuncSetAttribute(k_dense_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageMax));
        configured = true;
    }
    k_dense_pass<<<grid, kThreads, a.stage_bytes, s>>>(a);
    PTSBE_CUDA(cudaGetLastError());
    count_launch();
}

}  // namespace ptsbe
